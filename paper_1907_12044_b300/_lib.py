"""ctypes binding of libtdvp (argument marshalling only; every step runs in the CUDA library)."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

PREC_FP64 = 0
PREC_TF32 = 1
PREC_TF32X3 = 2
PREC_BF16 = 3
PREC_BF16X3 = 4
PREC_TF32_3M = 5
PREC_BF16_3M = 6
MIXED_PRECISIONS = (PREC_TF32, PREC_TF32X3, PREC_BF16, PREC_BF16X3, PREC_TF32_3M, PREC_BF16_3M)
KRYLOV_ADAPTIVE = 0
KRYLOV_LEARNED = 1
MLP_NPARAM = 4866

ERRORS = {
    -1: "invalid argument", -2: "CUDA error", -3: "out of device memory",
    -4: "Krylov solve stopped at kmax above the tolerance", -5: "device wait timed out",
    -6: "non-finite value", -7: "call out of order",
}

EXPORTED_SYMBOLS = [
    "tdvp_create", "tdvp_build_mpo", "tdvp_init_mps", "tdvp_init_mps_tensors", "tdvp_ps_step",
    "tdvp_observables", "tdvp_chain_info", "tdvp_get_site", "tdvp_move_center",
    "tdvp_center_to_zero", "tdvp_apply_heff", "tdvp_debug_qr", "tdvp_debug_expm", "tdvp_stats",
    "tdvp_reset_stats", "tdvp_last_error", "tdvp_destroy", "tdvp_set_profiling",
    "tdvp_lq_noalloc", "tdvp_apply_h0", "tdvp_set_option", "tdvp_autotune",
    "tdvp_controller_set_weights", "tdvp_controller_get_weights", "tdvp_controller_logging",
    "tdvp_controller_log", "tdvp_controller_train", "tdvp_controller_loss_grad",
    "tdvp_zgemm_ozaki_workspace", "tdvp_zgemm_ozaki", "tdvp_zgemm_ozaki_status",
]


class TDVPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libtdvp error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class FHParamsC(C.Structure):
    _fields_ = [("n_el", C.c_int), ("E", C.POINTER(C.c_double)), ("J", C.POINTER(C.c_double)),
                ("n_modes", C.POINTER(C.c_int)), ("omega", C.POINTER(C.c_double)),
                ("g", C.POINTER(C.c_double)), ("n_levels", C.POINTER(C.c_int)),
                ("el_order", C.POINTER(C.c_int)), ("energy_offset", C.c_double),
                ("include_zpe", C.c_int)]


NCAT = 7
CATEGORIES = ["gemm", "wapply", "lanczos_vec", "tridiag", "qr", "other", "tc_gemm"]
# the paper's sub-step labels of the time cost of a step (Sec. III.B), in TDVP_PH_* order
NPHASE = 7
PHASES = ["Deriv-Forward", "Deriv-Backward", "Krylov", "QR", "MatMul-QR", "Get Env", "other"]
OPT_RANK_RTOL = 1
OPT_KRYLOV_CHECK_ALL = 2
OPT_QR_KERNEL = 3
OPT_GRAPH = 4
OPT_PDL = 5
OPT_FUSED_LANCZOS = 6
OPT_STALL_TEST = 7
OPT_LANCZOS_CHUNKS = 8
OPT_ENV_FP64 = 9


class StatsC(C.Structure):
    _fields_ = [("steps", C.c_longlong), ("site_updates", C.c_longlong), ("matvecs", C.c_longlong),
                ("krylov_solves", C.c_longlong), ("krylov_dim_sum", C.c_longlong),
                ("krylov_dim_max", C.c_int), ("host_syncs", C.c_longlong),
                ("kernel_launches", C.c_longlong), ("not_converged", C.c_longlong),
                ("tri_evals", C.c_longlong),
                ("prof_ms", C.c_double * NCAT), ("prof_launches", C.c_longlong * NCAT),
                ("prof_flops", C.c_double * NCAT), ("prof_bytes", C.c_double * NCAT),
                ("prof_phase_ms", C.c_double * NPHASE), ("prof_phase_launches", C.c_longlong * NPHASE)]


def library_path():
    return os.path.join(HERE, "libtdvp.so")


_LIB = None


def load_library():
    """Load libtdvp.so from the package directory (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_1907_12044_b300.build()")
    lib = C.CDLL(path)
    P = C.c_void_p
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int)
    lib.tdvp_create.argtypes = [C.POINTER(P), C.c_int, P, C.c_int, C.c_int]
    lib.tdvp_build_mpo.argtypes = [P, C.c_int, C.POINTER(FHParamsC)]
    lib.tdvp_init_mps.argtypes = [P, C.c_int, C.c_int, C.c_int]
    lib.tdvp_init_mps_tensors.argtypes = [P, C.c_int, ip, dp]
    lib.tdvp_ps_step.argtypes = [P, C.c_double, C.c_int, C.c_int, C.c_int, C.c_double]
    lib.tdvp_observables.argtypes = [P, C.c_int, dp, dp, dp]
    lib.tdvp_chain_info.argtypes = [P, C.c_int, ip, ip, ip, ip]
    lib.tdvp_get_site.argtypes = [P, C.c_int, C.c_int, dp]
    lib.tdvp_move_center.argtypes = [P, C.c_int, C.c_int]
    lib.tdvp_center_to_zero.argtypes = [P, C.c_int]
    lib.tdvp_apply_heff.argtypes = [P, C.c_int, C.c_int, C.c_int, dp, dp]
    lib.tdvp_apply_h0.argtypes = [P, C.c_int, C.c_int, C.c_int, dp, dp]
    lib.tdvp_debug_qr.argtypes = [P, C.c_int, C.c_int, dp, dp, dp]
    lib.tdvp_debug_expm.argtypes = [P, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, dp, dp, ip]
    lib.tdvp_stats.argtypes = [P, C.POINTER(StatsC)]
    lib.tdvp_set_profiling.argtypes = [P, C.c_int]
    lib.tdvp_set_option.argtypes = [P, C.c_int, C.c_double]
    lib.tdvp_autotune.argtypes = [P]
    fp = C.POINTER(C.c_float)
    lib.tdvp_controller_set_weights.argtypes = [P, fp, C.c_int]
    lib.tdvp_controller_get_weights.argtypes = [P, fp, C.c_int]
    lib.tdvp_controller_logging.argtypes = [P, C.c_longlong]
    lib.tdvp_controller_log.argtypes = [P, fp, C.c_longlong, C.POINTER(C.c_longlong)]
    lib.tdvp_controller_train.argtypes = [P, C.c_int, C.c_int, C.c_float, fp]
    lib.tdvp_controller_loss_grad.argtypes = [P, C.c_int, fp, fp, C.c_int, fp, fp]
    lib.tdvp_lq_noalloc.argtypes = [C.c_int, C.c_int, P, P, P, P]
    lib.tdvp_zgemm_ozaki_workspace.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int]
    lib.tdvp_zgemm_ozaki_workspace.restype = C.c_size_t
    lib.tdvp_zgemm_ozaki.argtypes = [C.c_int, C.c_int, C.c_int, P, P, P, C.c_int, P, C.c_size_t, P]
    lib.tdvp_zgemm_ozaki_status.argtypes = [P, P]
    lib.tdvp_reset_stats.argtypes = [P]
    lib.tdvp_reset_stats.restype = None
    lib.tdvp_last_error.argtypes = [P]
    lib.tdvp_last_error.restype = C.c_char_p
    lib.tdvp_destroy.argtypes = [P]
    lib.tdvp_destroy.restype = None
    _LIB = lib
    return lib


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _fptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


class Engine:
    """One libtdvp context: ``n_realisations`` trajectories on one GPU and one CUDA stream.

    ``stream`` is a raw cudaStream_t value (int); by default the current PyTorch stream of the
    device is used.
    """

    def __init__(self, n_realisations=1, kmax=64, device=0, stream=None):
        self.lib = load_library()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        self._h = C.c_void_p()
        self.R = n_realisations
        rc = self.lib.tdvp_create(C.byref(self._h), device, C.c_void_p(stream), n_realisations, kmax)
        if rc != 0:
            raise TDVPError(rc, "tdvp_create failed")
        self._keep = []
        self.n_el = None

    def _check(self, rc):
        if rc != 0:
            raise TDVPError(rc, self.lib.tdvp_last_error(self._h).decode())
        return rc

    def close(self):
        if self._h:
            self.lib.tdvp_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- set-up -----------------------------------------------------------------------------
    def build_mpo(self, r, params):
        """``params``: an object with ``.flat()`` (dict of E, J, n_modes, omega, g, n_levels,
        el_order), ``energy_offset`` and ``include_zpe``."""
        f = params.flat()
        arrs = {k: np.ascontiguousarray(v, dtype=np.int32 if k in ("n_modes", "n_levels", "el_order") else np.float64)
                for k, v in f.items()}
        p = FHParamsC(len(arrs["E"]), _dptr(arrs["E"]), _dptr(arrs["J"]), _iptr(arrs["n_modes"]),
                      _dptr(arrs["omega"]), _dptr(arrs["g"]), _iptr(arrs["n_levels"]), _iptr(arrs["el_order"]),
                      float(params.energy_offset), int(bool(params.include_zpe)))
        self._check(self.lib.tdvp_build_mpo(self._h, r, C.byref(p)))
        self.n_el = len(arrs["E"])

    def init_mps(self, r, D, exciton_site):
        self._check(self.lib.tdvp_init_mps(self._h, r, int(D), int(exciton_site)))

    def init_mps_tensors(self, r, tensors):
        bd = [1] + [int(t.shape[2]) for t in tensors]
        bd = np.asarray(bd, dtype=np.int32)
        flat = np.concatenate([np.ascontiguousarray(t, dtype=np.complex128).reshape(-1) for t in tensors])
        buf = np.ascontiguousarray(flat.view(np.float64))
        self._check(self.lib.tdvp_init_mps_tensors(self._h, r, _iptr(bd), _dptr(buf)))

    # -- time evolution -----------------------------------------------------------------------
    def step(self, dt_fs, n_steps=1, precision=PREC_FP64, krylov_mode=KRYLOV_ADAPTIVE, tol=1e-12):
        self._check(self.lib.tdvp_ps_step(self._h, float(dt_fs), int(n_steps), int(precision),
                                          int(krylov_mode), float(tol)))

    def observables(self, r=0):
        pops = np.zeros(self.n_el)
        e = C.c_double()
        n = C.c_double()
        self._check(self.lib.tdvp_observables(self._h, r, _dptr(pops), C.byref(e), C.byref(n)))
        return pops, e.value, n.value

    # -- inspection and components ----------------------------------------------------------
    def chain_info(self, r=0):
        n = C.c_int()
        self._check(self.lib.tdvp_chain_info(self._h, r, C.byref(n), None, None, None))
        N = n.value
        d = np.zeros(N, np.int32)
        bd = np.zeros(N + 1, np.int32)
        w = np.zeros(N + 1, np.int32)
        self._check(self.lib.tdvp_chain_info(self._h, r, C.byref(n), _iptr(d), _iptr(bd), _iptr(w)))
        return d, bd, w

    def get_site(self, r, i):
        d, bd, _ = self.chain_info(r)
        out = np.zeros((bd[i], d[i], bd[i + 1]), dtype=np.complex128)
        self._check(self.lib.tdvp_get_site(self._h, r, i, _dptr(out.view(np.float64))))
        return out

    def get_mps(self, r=0):
        d, _, _ = self.chain_info(r)
        return [self.get_site(r, i) for i in range(len(d))]

    def move_center(self, r, site):
        self._check(self.lib.tdvp_move_center(self._h, r, site))

    def center_to_zero(self, r):
        self._check(self.lib.tdvp_center_to_zero(self._h, r))

    def apply_heff(self, r, i, x, precision=PREC_FP64):
        x = np.ascontiguousarray(x, dtype=np.complex128)
        y = np.zeros_like(x)
        self._check(self.lib.tdvp_apply_heff(self._h, r, i, int(precision), _dptr(x.view(np.float64)),
                                             _dptr(y.view(np.float64))))
        return y

    def apply_h0(self, r, i, x, precision=PREC_FP64):
        x = np.ascontiguousarray(x, dtype=np.complex128)
        y = np.zeros_like(x)
        self._check(self.lib.tdvp_apply_h0(self._h, r, i, int(precision), _dptr(x.view(np.float64)),
                                           _dptr(y.view(np.float64))))
        return y

    def debug_qr(self, Cm):
        Cm = np.ascontiguousarray(Cm, dtype=np.complex128)
        m, n = Cm.shape
        Q = np.zeros((m, n), np.complex128)
        R = np.zeros((n, n), np.complex128)
        self._check(self.lib.tdvp_debug_qr(self._h, m, n, _dptr(Cm.view(np.float64)), _dptr(Q.view(np.float64)),
                                           _dptr(R.view(np.float64))))
        return Q, R

    def debug_expm(self, r, i, z, tol, v):
        v = np.ascontiguousarray(v, dtype=np.complex128)
        out = np.zeros_like(v)
        k = C.c_int()
        self._check(self.lib.tdvp_debug_expm(self._h, r, i, float(np.real(z)), float(np.imag(z)), float(tol),
                                             _dptr(v.view(np.float64)), _dptr(out.view(np.float64)), C.byref(k)))
        return out, k.value

    def stats(self):
        s = StatsC()
        self._check(self.lib.tdvp_stats(self._h, C.byref(s)))
        out = {}
        for k, _ in StatsC._fields_:
            v = getattr(s, k)
            if k.startswith("prof_phase"):
                out[k] = {c: v[i] for i, c in enumerate(PHASES)}
            elif k.startswith("prof_"):
                out[k] = {c: v[i] for i, c in enumerate(CATEGORIES)}
            else:
                out[k] = v
        return out

    # -- learned Krylov controller ------------------------------------------------------------
    def controller_set_weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        self._check(self.lib.tdvp_controller_set_weights(self._h, _fptr(w), w.size))

    def controller_get_weights(self):
        w = np.zeros(MLP_NPARAM, np.float32)
        self._check(self.lib.tdvp_controller_get_weights(self._h, _fptr(w), w.size))
        return w

    def controller_logging(self, capacity):
        self._check(self.lib.tdvp_controller_logging(self._h, int(capacity)))

    def controller_log(self, max_rows=1 << 22):
        n = C.c_longlong()
        self._check(self.lib.tdvp_controller_log(self._h, None, 0, C.byref(n)))
        k = min(n.value, max_rows)
        out = np.zeros((k, 9), np.float32)
        if k:
            self._check(self.lib.tdvp_controller_log(self._h, _fptr(out), k, C.byref(n)))
        return out

    def controller_train(self, epochs=20, batch=1024, lr=1e-3):
        """Both training stages; returns (mean-squared error of k, logistic loss of acceptance)."""
        loss = np.zeros(2, np.float32)
        self._check(self.lib.tdvp_controller_train(self._h, int(epochs), int(batch), float(lr), _fptr(loss)))
        return float(loss[0]), float(loss[1])

    def controller_loss_grad(self, X, t, head=0):
        X = np.ascontiguousarray(X, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        loss = C.c_float()
        g = np.zeros(MLP_NPARAM, np.float32)
        self._check(self.lib.tdvp_controller_loss_grad(self._h, int(head), _fptr(X), _fptr(t), X.shape[0],
                                                       C.byref(loss), _fptr(g)))
        return loss.value, g

    def autotune(self):
        self._check(self.lib.tdvp_autotune(self._h))

    def set_option(self, option, value):
        self._check(self.lib.tdvp_set_option(self._h, int(option), float(value)))

    def set_profiling(self, on=True):
        self._check(self.lib.tdvp_set_profiling(self._h, 1 if on else 0))

    def reset_stats(self):
        self.lib.tdvp_reset_stats(self._h)


def zgemm_ozaki_workspace(m, n, k, slices):
    """Bytes of device workspace tdvp_zgemm_ozaki needs (0: sizes out of its limits)."""
    return int(load_library().tdvp_zgemm_ozaki_workspace(int(m), int(n), int(k), int(slices)))


def zgemm_ozaki(m, n, k, a_ptr, b_ptr, c_ptr, slices, ws_ptr, ws_bytes, stream):
    """C = A B (complex FP64, device pointers as ints) emulated on the BF16 tensor cores with
    `slices` 7-bit slices per operand; see tdvp_zgemm_ozaki in include/tdvp.h.  Asynchronous."""
    rc = load_library().tdvp_zgemm_ozaki(int(m), int(n), int(k), C.c_void_p(a_ptr), C.c_void_p(b_ptr),
                                         C.c_void_p(c_ptr), int(slices), C.c_void_p(ws_ptr), int(ws_bytes),
                                         C.c_void_p(stream))
    if rc != 0:
        raise TDVPError(rc, "tdvp_zgemm_ozaki failed")


def zgemm_ozaki_status(ws_ptr, stream):
    """Synchronise the stream; raise TDVPError if a device wait of the last call gave up."""
    rc = load_library().tdvp_zgemm_ozaki_status(C.c_void_p(ws_ptr), C.c_void_p(stream))
    if rc != 0:
        raise TDVPError(rc, "tdvp_zgemm_ozaki: device wait timed out")


def lq_noalloc(n, m, x_ptr, q_ptr, l_ptr, stream):
    """X = L Q on device buffers (raw device pointers as ints) with no device allocation.

    For callers that must not allocate device memory; see tdvp_lq_noalloc in include/tdvp.h.
    Raises TDVPError on a non-zero status.
    """
    lib = load_library()
    rc = lib.tdvp_lq_noalloc(int(n), int(m), C.c_void_p(x_ptr), C.c_void_p(q_ptr), C.c_void_p(l_ptr),
                             C.c_void_p(stream))
    if rc != 0:
        raise TDVPError(rc, "tdvp_lq_noalloc failed")
