"""B300-native one-site TDVP projector-splitting (TDVP-PS) for Frenkel-Holstein chains.

The time evolution runs in ``libtdvp.so`` (hand-written CUDA for sm_103a behind a C ABI, see
``include/tdvp.h``); this package only loads the library and marshals arguments.  There is no
CPU path: if the library is missing, ``Engine`` raises.
"""
from ._lib import (Engine, TDVPError, load_library, library_path, lq_noalloc, zgemm_ozaki,
                   zgemm_ozaki_workspace, zgemm_ozaki_status, PREC_FP64, PREC_TF32,
                   PREC_TF32X3, PREC_BF16, PREC_BF16X3, PREC_TF32_3M, PREC_BF16_3M, MIXED_PRECISIONS,
                   PHASES, KRYLOV_ADAPTIVE, KRYLOV_LEARNED, MLP_NPARAM, OPT_RANK_RTOL, OPT_KRYLOV_CHECK_ALL, OPT_QR_KERNEL, OPT_GRAPH, OPT_PDL, OPT_FUSED_LANCZOS, OPT_STALL_TEST, OPT_LANCZOS_CHUNKS, OPT_ENV_FP64,
                   EXPORTED_SYMBOLS)
from .build import build

__all__ = ["Engine", "TDVPError", "load_library", "library_path", "lq_noalloc", "zgemm_ozaki",
           "zgemm_ozaki_workspace", "zgemm_ozaki_status", "build", "PREC_FP64", "PREC_TF32", "PREC_TF32X3",
           "PREC_BF16", "PREC_BF16X3", "PREC_TF32_3M", "PREC_BF16_3M", "MIXED_PRECISIONS", "PHASES",
           "KRYLOV_ADAPTIVE", "KRYLOV_LEARNED", "MLP_NPARAM", "OPT_RANK_RTOL", "OPT_KRYLOV_CHECK_ALL", "OPT_QR_KERNEL", "OPT_GRAPH", "OPT_PDL", "OPT_FUSED_LANCZOS", "OPT_STALL_TEST", "OPT_LANCZOS_CHUNKS", "OPT_ENV_FP64",
           "EXPORTED_SYMBOLS"]
