/*
 * tdvp.h -- C ABI of the B300 one-site TDVP projector-splitting (TDVP-PS) library.
 *
 * The library advances matrix product states (MPS) of Frenkel-Holstein chains in
 * time with the one-site TDVP-PS integrator of Li, Ren, Shuai (arXiv:1907.12044,
 * Sec. II.A.2 "TDVP-PS"): every time step is the symmetric second-order split of
 * Eq. ps_trotter, i.e. a left-to-right half sweep with tau/2 (forward site
 * evolution Eq. tdvp2_C, QR gauge shift Eq. QR, backward bond evolution
 * Eq. tdvp2_D, absorption C_{i+1} = D_i R_{i+1}), the last site with tau, and the
 * mirror right-to-left half sweep.  Each local exponential is a Lanczos Krylov
 * exponential.  All arithmetic of a step runs in CUDA kernels on one GPU.
 *
 * Conventions shared by every entry point
 *  - Return value: TDVP_OK (0) or a negative TDVP_ERR_* code.  No C++ exception
 *    crosses the ABI.  tdvp_last_error() gives a message for the last failure.
 *  - Host arrays passed in are owned by the caller and copied before return.
 *  - The context owns all device memory it allocates (cudaMalloc on the device
 *    given at creation) and frees it in tdvp_destroy().
 *  - Work is enqueued on the caller's CUDA stream (cudaStream_t passed as void*;
 *    NULL = legacy default stream).  Entry points that return host data
 *    synchronise that stream; tdvp_ps_step() may synchronise it to read Krylov
 *    convergence flags.
 *  - Complex numbers are interleaved (re, im) doubles.  A site tensor A[l][s][r]
 *    of bond dims (Dl, Dr) and local dimension d is stored row-major with r
 *    fastest: element (l, s, r) at offset 2*((l*d + s)*Dr + r).
 *  - Units: energies and frequencies in cm^-1, times in fs (hbar = 1, phase
 *    2*pi*c*E*t with 2*pi*c = 1.883651567e-4 rad/(cm^-1 fs)).
 *  - A context is not thread-safe: one host thread at a time.
 */
#ifndef TDVP_H
#define TDVP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tdvp_ctx tdvp_ctx;

/* Frenkel-Holstein Hamiltonian, Eq. holstein (Sec. II.C):
 *   H = sum_m (E_m - energy_offset) n_m + sum_{m!=n} J_mn a_m^+ a_n
 *     + sum_{m,l} w_ml (b^+ b [+ 1/2 if include_zpe])
 *     + sum_{m,l} g_ml w_ml (b^+ + b) n_m
 * Electronic sites are two-level (|0>, |1>); mode (m, l) has n_levels levels.
 * Chain order: for m in el_order, electronic site m followed by its modes in the
 * order given (the paper's layout, Sec. II.C).  All pointers are host memory. */
typedef struct {
  int n_el;                /* number of electronic sites, >= 1 */
  const double* E;         /* [n_el] site energies (cm^-1) */
  const double* J;         /* [n_el*n_el] row-major couplings (cm^-1); must be symmetric; diagonal ignored */
  const int* n_modes;      /* [n_el] number of modes attached to each electronic site */
  const double* omega;     /* [sum n_modes] mode frequencies (cm^-1), site 0's modes first */
  const double* g;         /* [sum n_modes] dimensionless couplings (Huang-Rhys S = g^2) */
  const int* n_levels;     /* [sum n_modes] phonon levels of each mode, >= 1 */
  const int* el_order;     /* [n_el] permutation of 0..n_el-1: chain order of electronic sites */
  double energy_offset;    /* subtracted from every E_m (keeps the shifted spectrum small) */
  int include_zpe;         /* 1: add w/2 per mode; 0: omit the zero-point constant */
} tdvp_fh_params;

/* Status codes. */
#define TDVP_OK                        0
#define TDVP_ERR_INVALID_ARG          -1  /* bad size, pointer, index or mismatched structure */
#define TDVP_ERR_CUDA                 -2  /* a CUDA runtime call failed */
#define TDVP_ERR_OOM                  -3  /* cudaMalloc failed */
#define TDVP_ERR_KRYLOV_NOT_CONVERGED -4  /* Lanczos hit k_max above the tolerance (result still written) */
#define TDVP_ERR_DEVICE_TIMEOUT       -5  /* a bounded device-side wait gave up */
#define TDVP_ERR_NAN                  -6  /* a non-finite norm was met */
#define TDVP_ERR_STATE                -7  /* call out of order (e.g. step before init) */

/* Arithmetic of the contractions of a step: the Lanczos matvecs H_eff.A (Eq. tdvp2_C) and H0.D
 * (Eq. tdvp2_D) and, in the mixed precisions, the environment updates (Eq. tdvp1_h1i,
 * tdvp1_hiN).  The Lanczos orthogonalisation, the tridiagonal exponential, the gauge-shift QR and
 * the absorption are FP64 in every mode.  Every mixed mode accumulates in FP32 on the tcgen05
 * tensor cores.  "4M": a complex product as 4 real products (re re - im im, re im + im re);
 * "3M" (Gauss): as 3 real products re re, im im, (re + im)(re + im), combined in FP32; "x3": each
 * operand split into a rounded high part and the rounded remainder, the terms hi hi + hi lo +
 * lo hi of the 4M form accumulated (compensated products). */
#define TDVP_PREC_FP64    0   /* complex double on the FP64 pipe */
#define TDVP_PREC_TF32    1   /* kind::tf32, TF32 operands (11 significant bits), 4M */
#define TDVP_PREC_TF32X3  2   /* TF32 hi/lo split, 4M, x3 (~FP32-level products) */
#define TDVP_PREC_BF16    3   /* kind::f16, BF16 operands (8 significant bits), 4M */
#define TDVP_PREC_BF16X3  4   /* BF16 hi/lo split, 4M, x3 (~16 significant bits) */
#define TDVP_PREC_TF32_3M 5   /* TF32 operands, 3M */
#define TDVP_PREC_BF16_3M 6   /* BF16 operands, 3M */
#define TDVP_PREC_LAST    6

/* Krylov dimension control. */
#define TDVP_KRYLOV_ADAPTIVE 0   /* grow k until the a-posteriori estimate meets the tolerance */
#define TDVP_KRYLOV_LEARNED  1   /* the learned controller predicts k after the first Lanczos step;
                                    convergence is tested from that k on, and the adaptive test
                                    (the same estimate and tolerance) decides when to stop */

/* Create a context on CUDA device `device` working on `cuda_stream`, holding
 * `n_realisations` independent trajectories (>= 1) that share one chain layout,
 * with at most `kmax` (1..128) Krylov vectors per local exponential. */
int tdvp_create(tdvp_ctx** ctx, int device, void* cuda_stream, int n_realisations, int kmax);

/* Build the MPO of Eq. holstein (Eq. mpo, finite-state construction with bond
 * dimension 2 + 2*min(k_left, k_right) (+1 inside a mode block), k = electronic
 * sites on each side) for realisation r and upload it.  Every realisation must
 * have the same chain layout (n_el, modes, levels, order); values may differ. */
int tdvp_build_mpo(tdvp_ctx* ctx, int r, const tdvp_fh_params* p);

/* Initial state of Sec. II.C for realisation r: exciton on electronic site
 * `exciton_site`, every mode in its ground level, embedded at bond dims
 * D_b = min(D, prod d left, prod d right).  Site i viewed as a Dl x (d*Dr)
 * matrix gets row 0 = the occupied path and rows j >= 1 = the standard basis
 * vectors at the successive (s, r) positions other than (occupied, 0), ordered by
 * r first and s second, which makes it right-canonical (Eq. rcanon).  Builds all right
 * environments h[i+1:N] (Eq. tdvp1_hiN).  Requires tdvp_build_mpo first. */
int tdvp_init_mps(tdvp_ctx* ctx, int r, int D, int exciton_site);   /* 1 <= D <= 256 */

/* Explicit initial tensors for realisation r: bond_dims[0..N] (bond_dims[0] =
 * bond_dims[N] = 1) and re_im = all site tensors concatenated in site order,
 * each in the layout above.  The state is right-canonicalised on the device by
 * LQ from the last site (Eq. QR, "RQ" direction), the new centre normalised after
 * each absorbed factor (only the normalised state is kept, and the norm of a product
 * of generic tensors grows or shrinks geometrically with the chain length), and the
 * right environments are built.  Tensors need not be canonical or normalised. */
int tdvp_init_mps_tensors(tdvp_ctx* ctx, int r, const int* bond_dims, const double* re_im);

/* Advance every realisation by n_steps steps of dt_fs with Eq. ps_trotter.
 * precision: TDVP_PREC_*; krylov_mode: TDVP_KRYLOV_*; krylov_tol: absolute
 * tolerance on the a-posteriori Lanczos estimate ||v|| beta_k |[exp(zT_k)e_1]_k|
 * (e.g. 1e-12).  On return the state is right-canonical with the centre at site 0.
 * Returns TDVP_ERR_KRYLOV_NOT_CONVERGED if some exponential stopped at kmax (the
 * step is still complete). */
int tdvp_ps_step(tdvp_ctx* ctx, double dt_fs, int n_steps, int precision, int krylov_mode,
                 double krylov_tol);

/* Observables of realisation r (synchronises the stream):
 *   pops[n_el]: exciton populations P^(n) = <n_n>/<Psi|Psi> by electronic label (Eq. error);
 *   energy: <Psi|H|Psi>/<Psi|Psi> in the shifted frame (cm^-1);  norm: ||Psi||.
 * Any output pointer may be NULL. */
int tdvp_observables(tdvp_ctx* ctx, int r, double* pops, double* energy, double* norm);

/* Chain layout: n_sites; phys_dims[n_sites]; bond_dims[n_sites+1] of realisation
 * r; mpo_dims[n_sites+1].  Array pointers may be NULL. */
int tdvp_chain_info(tdvp_ctx* ctx, int r, int* n_sites, int* phys_dims, int* bond_dims,
                    int* mpo_dims);

/* Copy site tensor i of realisation r to the host (Dl*d*Dr complex, layout above). */
int tdvp_get_site(tdvp_ctx* ctx, int r, int i, double* re_im);

/* Move the gauge centre of realisation r from site 0 to site `site` by QR
 * (Eq. QR) and build the left environments h[1:i-1] on the way; the state must
 * have its centre at site 0 (after init or a step).  Used to probe H_eff at
 * interior sites.  Call tdvp_center_to_zero() before the next tdvp_ps_step(). */
int tdvp_move_center(tdvp_ctx* ctx, int r, int site);
int tdvp_center_to_zero(tdvp_ctx* ctx, int r);

/* y = H[i] x for the effective Hamiltonian of Eq. tdvp1_H at site i of
 * realisation r, with the stored environments (valid at the current centre), in the
 * arithmetic `precision` (TDVP_PREC_*).  x, y: host arrays of Dl*d*Dr complex. */
int tdvp_apply_heff(tdvp_ctx* ctx, int r, int i, int precision, const double* x, double* y);

/* y = H0 x for the zero-site Hamiltonian of Eq. tdvp2_D on the bond (i, i+1):
 * sum_w h[1:i]_w x h[i+1:N]_w^T with the stored left environment of site i+1 and right
 * environment of site i.  x, y: host arrays of D*D complex (D = bond dimension). */
int tdvp_apply_h0(tdvp_ctx* ctx, int r, int i, int precision, const double* x, double* y);

/* Gauge-shift decomposition of Eq. QR on the device, exposed for testing:
 * C (m x n, m >= n, row-major complex, host) = Q R with Q orthonormal columns
 * and R upper triangular; rank-deficient columns (residual <= rtol*||C||_F after
 * two Gram-Schmidt passes) get R[j][j] = 0 and Q[:,j] completed from the first
 * standard basis vector at distance >= 1/2 from the span so far. */
int tdvp_debug_qr(tdvp_ctx* ctx, int m, int n, const double* C, double* Q, double* R);

/* Lanczos exponential exp(z H) v with H = H[i] of realisation r at the current
 * centre (same requirements as tdvp_apply_heff), z = z_re + i z_im.  Exposed for
 * testing; k_out receives the Krylov dimension used. */
int tdvp_debug_expm(tdvp_ctx* ctx, int r, int i, double z_re, double z_im, double tol,
                    const double* v, double* out, int* k_out);

/* Kernel categories of the optional per-launch timing (tdvp_set_profiling). */
#define TDVP_CAT_GEMM    0   /* contraction GEMMs: H_eff stages 1/3, environments, H0, absorption */
#define TDVP_CAT_WAPPLY  1   /* sparse MPO middle stage of H_eff and the environments */
#define TDVP_CAT_LZVEC   2   /* Lanczos orthogonalisation (dots, two Gram-Schmidt passes), start, combination */
#define TDVP_CAT_TRIDIAG 3   /* tridiagonal exponential, convergence test, next Krylov vector */
#define TDVP_CAT_QR      4   /* gauge-shift QR/LQ and its transposes */
#define TDVP_CAT_OTHER   5
#define TDVP_CAT_TC      6   /* tcgen05 complex GEMMs of the mixed-precision matvecs */
#define TDVP_NCAT        7

/* Sub-steps of a TDVP-PS step under the paper's own time-cost labels (Sec. III.B, Fig. of the
 * time cost per sub-step), for the per-launch timing: every launch of a step is booked under
 * the sub-step it serves. */
#define TDVP_PH_DERIV_FWD 0   /* "Deriv-Forward": H_eff.C matvecs of the forward site exponentials
                                 (Eq. tdvp2_C, Eq. tdvp1_H) and their operand packing */
#define TDVP_PH_DERIV_BWD 1   /* "Deriv-Backward": H0.D matvecs of the backward bond exponentials
                                 (Eq. tdvp2_D) and their operand packing */
#define TDVP_PH_KRYLOV    2   /* "Krylov": Lanczos vectors, tridiagonal exponential, combination */
#define TDVP_PH_QR        3   /* "QR": gauge-shift QR / LQ (Eq. QR) */
#define TDVP_PH_MATMUL_QR 4   /* "MatMul-QR": absorption of the bond factor into the neighbour,
                                 C_{i+1} = D_i R_{i+1} */
#define TDVP_PH_GET_ENV   5   /* "Get Env": environment updates (Eq. tdvp1_h1i, tdvp1_hiN) */
#define TDVP_PH_OTHER     6   /* observables and set-up */
#define TDVP_NPHASE       7

typedef struct {
  long long steps;             /* completed time steps (per realisation) */
  long long site_updates;      /* forward site evolutions, all realisations (2N-1 per step each) */
  long long matvecs;           /* H_eff and H0 applications, all realisations */
  long long krylov_solves;     /* local exponentials */
  long long krylov_dim_sum;    /* sum of Krylov dimensions over those solves */
  int krylov_dim_max;
  long long host_syncs;        /* stream synchronisations made inside tdvp_ps_step */
  long long kernel_launches;   /* kernels enqueued by this context */
  long long not_converged;     /* solves that stopped at kmax above tolerance */
  long long tri_evals;         /* tridiagonal exponentials evaluated (convergence tests), all realisations */
  /* filled only while profiling is on: per category, summed CUDA-event time of each launch
   * (recorded on the context stream right before and after it), launch count, the
   * algorithmic real flops of the contraction GEMMs (8 per complex multiply-add), and the
   * algorithmic bytes of the Lanczos vector kernels (TDVP_CAT_LZVEC): per solve of dimension k
   * on vectors of n complex elements, 16 n (2 k (k+1) + 10 k + 5) -- iteration j reads
   * V_0..V_j four times (dot and update of each of the two Gram-Schmidt passes) and moves w,
   * V_{j+1} and x nine times; start and combination add k + 5 vectors -- and their FP64 flops,
   * 16 n k (k+1) per solve (the two passes). */
  double prof_ms[TDVP_NCAT];
  long long prof_launches[TDVP_NCAT];
  double prof_flops[TDVP_NCAT];
  double prof_bytes[TDVP_NCAT];
  /* the same per-launch times booked by sub-step (TDVP_PH_*) */
  double prof_phase_ms[TDVP_NPHASE];
  long long prof_phase_launches[TDVP_NPHASE];
} tdvp_stats_t;

/* Turn per-launch CUDA-event timing on (1) or off (0).  While on, every kernel launch is
 * bracketed by two events on the context stream; the times are collected into tdvp_stats at
 * the end of each tdvp_ps_step (which then synchronises the stream). */
int tdvp_set_profiling(tdvp_ctx* ctx, int on);

int tdvp_stats(tdvp_ctx* ctx, tdvp_stats_t* out);
void tdvp_reset_stats(tdvp_ctx* ctx);

/* Right-to-left gauge shift without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that must not allocate device memory themselves or have
 * it allocated for them, e.g. code running inside a framework that owns every byte of device
 * memory through its own pool, or a latency-critical path where the implicit device
 * synchronisation of cudaMalloc/cudaFree is not acceptable.
 *
 * Computes X = L Q for X (n x m, row-major complex, interleaved, device memory), with Q
 * (n x m, device) having orthonormal rows and L (n x n, device) lower triangular, by the same
 * rule as the library's gauge shift: rows orthogonalised in order by Gram-Schmidt with one
 * re-orthogonalisation pass; a row whose residual is <= 1e-13 ||X||_F gets L[j][j] = 0 and is
 * replaced by the first unit vector at distance >= 1/2 from the rows so far.  No context is
 * needed; the work runs on the current device and `cuda_stream`, and the call returns after it
 * has finished (it synchronises the stream).
 *
 * Limits: 1 <= n <= 256, n <= m <= 16384; anything else returns TDVP_ERR_INVALID_ARG without
 * touching the device.  X, Q and L must not overlap (checked on the host: TDVP_ERR_INVALID_ARG).
 *
 * Memory: the scratch space (partial sums, column norms, barrier words; about 0.9 MB) is one
 * static device array of fixed size in the library, held by every GPU that loads the library
 * until the process exits.  The first call on a device (and the first after the device's context
 * was replaced, e.g. by cudaDeviceReset) looks up its address (cudaGetSymbolAddress) and the
 * co-resident block count; make that first call before any stream capture.  Every device-side
 * barrier wait gives up after 1 s of wall-clock time.  All calls on a device share that one array, so calls that overlap on the
 * GPU (other streams, other host threads) race and give wrong results; serialise them.
 * Returns TDVP_ERR_DEVICE_TIMEOUT if a bounded device-side wait gave up. */
int tdvp_lq_noalloc(int n, int m, const double* X, double* Q, double* L, void* cuda_stream);

/* FP64 complex GEMM emulated on the BF16 tensor cores (Ozaki splitting).  The paper's FP64
 * contractions (Eq. tdvp1_H, the absorption C_{i+1} = D_i R_{i+1} after Eq. QR) are complex GEMMs
 * on B300's FP64 pipe, which is far slower than its tensor cores; this computes the same product
 * from exact BF16 pieces of the operands.
 *
 * C = A B with A (m x k), B (k x n), C (m x n): complex, row-major, interleaved (re, im) doubles,
 * device memory, 16-byte aligned.  Method: the complex product as the real product
 * [[Ar, -Ai], [Ai, Ar]] [Br; Bi]; every row of the left factor and column of the right one scaled
 * by a power of two below 1 in magnitude and cut into `slices` (1..8) integer slices of 7 bits
 * (exact in BF16); the slice products of total order < slices accumulated exactly in FP32 tensor
 * memory over windows of 128 K values and summed in a float-float register pair.  Error per
 * element <= 2k (slices + 3) 2^(-7 slices) 2^(eR + fc) + ~2^-47 k 2^(eR + fc), where 2^eR and
 * 2^fc are the powers of two just above max|A row| and max|B column| (slices = 8: ~1e-14 of
 * k max|A_r| max|B_c|).  Operands whose parts are integers of magnitude below 128 give the exact
 * product with slices = 1 (as long as its elements stay below 2^24).
 *
 * Workspace: `workspace` (device, 1024-byte aligned, at least tdvp_zgemm_ozaki_workspace(m, n, k,
 * slices) bytes; 0 means invalid sizes) holds the slices, the scale exponents and an error word;
 * it is owned by the caller, who must not share it between calls in flight.  No allocation.
 * Asynchronous on `cuda_stream`; the buffers must not overlap (checked on the host).
 * Limits: 1 <= m, k <= 2^21, 1 <= n <= 2^28, 4 m k <= 2^36, 2 k n <= 2^36, 1 <= slices <= 8;
 * otherwise TDVP_ERR_INVALID_ARG without touching the device.  Every device-side wait is bounded
 * (1 s); tdvp_zgemm_ozaki_status() synchronises the stream and returns TDVP_ERR_DEVICE_TIMEOUT if a
 * wait of the last call on this workspace gave up (C is then not written), else TDVP_OK. */
size_t tdvp_zgemm_ozaki_workspace(int m, int n, int k, int slices);
int tdvp_zgemm_ozaki(int m, int n, int k, const double* A, const double* B, double* C, int slices,
                     void* workspace, size_t workspace_bytes, void* cuda_stream);
int tdvp_zgemm_ozaki_status(const void* workspace, void* cuda_stream);

/* Learned Krylov controller (not in the paper): a two-layer MLP, 8 features -> 64 -> 64, ReLU,
 * FP32, with two heads on the second hidden layer: the Krylov dimension y (linear) and the logit a
 * of the acceptance of the dimension kp = floor(y) clamped to [1, 126] (logistic: will the residual
 * test pass at kp).  MLP_NPARAM = 4866 floats laid out W1[8][64], b1[64], W2[64][64], b2[64],
 * W3[64], b3 (head 1), W4[64], b4 (head 2).
 * Features of a local exponential, known after its first Lanczos step: log10(1 + |tau| ||H v||),
 * kind (site 0 / bond 1), previous k of the same site and kind / 32, site / (N-1),
 * log2(vector length) / 20, log10|tau| / 4, -log10(tol) / 12, log10(1 + |tau| |alpha_0|).
 * With TDVP_KRYLOV_LEARNED the Lanczos iterations run without any convergence test up to kp, or up
 * to kp - 1 when a >= 0 (a predicted pass at kp means the solve may have converged earlier, and an
 * iteration past convergence costs a whole matvec while a failed test costs one tridiagonal
 * exponential); from there the adaptive test (same estimate, same tolerance) decides where the
 * solve stops, so a wrong prediction costs iterations or tests, never accuracy. */
int tdvp_controller_set_weights(tdvp_ctx* ctx, const float* w, int n);   /* n = 4866, host array */
int tdvp_controller_get_weights(tdvp_ctx* ctx, float* w, int n);
/* Log every finished exponential (features, k) into a device buffer of `capacity` rows; 0 stops. */
int tdvp_controller_logging(tdvp_ctx* ctx, long long capacity);
/* Copy up to max_rows log rows (9 floats each) to the host; rows receives the logged count. */
int tdvp_controller_log(tdvp_ctx* ctx, float* out, long long max_rows, long long* rows);
/* Training on the log, on the GPU, in two stages of `epochs` passes over mini-batches of `batch`
 * rows, Adam (beta 0.9/0.999, moments reset per stage): (1) trunk and head 1 by the mean-squared
 * error of k; (2) head 2 alone (trunk frozen) by the logistic loss of [k <= kp].  final_loss[0],
 * final_loss[1] receive each stage's mean loss over its last epoch (final_loss may be NULL). */
int tdvp_controller_train(tdvp_ctx* ctx, int epochs, int batch, float lr, float* final_loss);
/* Loss and gradient (all MLP_NPARAM entries) of head `head` (0: squared error of k over trunk and
 * head 1; 1: logistic loss of the acceptance over head 2) of the current weights on B rows
 * X[B][8] with final dimensions t[B] (host), for checking. */
int tdvp_controller_loss_grad(tdvp_ctx* ctx, int head, const float* X, const float* t, int B, float* loss,
                              float* grad);

/* Autotuner: for every distinct gauge-shift QR shape of the chain, time the cooperative-grid QR
 * kernel with several block counts per realisation and the cluster QR kernel with several
 * cluster sizes, each on a random full-rank plus a random rank-deficient matrix placed in the QR
 * scratch (the state is not touched), and keep the fastest for the following steps.  Requires every
 * realisation to be initialised; synchronises the stream. */
int tdvp_autotune(tdvp_ctx* ctx);

/* Options of a context (take effect from the next call):
 *   TDVP_OPT_RANK_RTOL: relative rank threshold of the gauge-shift QR (default 1e-13); a column
 *     whose residual after two Gram-Schmidt passes is <= value * ||C||_F is replaced by the
 *     completion vector.  From a product start most bonds are rank deficient and this threshold
 *     decides which directions are completed; raising it (e.g. to 1e-6) makes those decisions
 *     insensitive to arithmetic noise of the mixed-precision matvecs.
 *   TDVP_OPT_KRYLOV_CHECK_ALL: 1 = test Lanczos convergence at every k, 0 (default) = from the
 *     last Krylov dimension of the same site minus 2 on.
 *   TDVP_OPT_QR_KERNEL: which kernel runs the gauge-shift QR.  -1 (default): the autotuned
 *     choice, else the cooperative-grid kernel; -2: the cluster kernel with the largest cluster
 *     the shape fits, else the cooperative-grid kernel; 0: the
 *     cooperative-grid kernel (blocked Gram-Schmidt with Cholesky-QR panels); 1, 2, 4, 8, 16: the
 *     cluster kernel with that many CTAs per realisation (a shape that does not fit its shared
 *     memory fails with TDVP_ERR_INVALID_ARG).  All compute the same decomposition.
 *   TDVP_OPT_GRAPH: 1 = tdvp_ps_step captures one whole step (every realisation) into a CUDA
 *     graph and replays it n_steps times.  Each Lanczos exponential is a conditional while node
 *     whose body is one iteration; the device ends the loop, so a step needs no host round trip.
 *     Convergence tests start from each realisation's previous Krylov dimension of the same
 *     (site, kind) minus 2 (or every k with TDVP_OPT_KRYLOV_CHECK_ALL, or at the learned
 *     prediction).  The graph is captured on the first call for a (dt, tolerance, precision,
 *     Krylov mode) and kept until build/init, autotune or any option change.  Ignored while
 *     profiling is on (per-launch timing needs the launch-by-launch path).  0 (default): launch
 *     by launch, one host flag read per exponential.
 *   TDVP_OPT_PDL: 1 (default) = kernels of the step are launched as programmatic dependents of
 *     their predecessor (they start while it finishes and wait for it before touching memory);
 *     0 = plain stream order.  Process-wide: it applies to every context.
 *   TDVP_OPT_FUSED_LANCZOS: 1 (default) = each Lanczos iteration after the matvec (dots, both
 *     Gram-Schmidt passes, tridiagonal step, next vector) is one cooperative launch whose phases
 *     are separated by bounded group barriers, whenever the vector chunks of every realisation fit
 *     co-resident on the GPU; 0 = four launches per iteration.  Both give bit-identical results.
 *   TDVP_OPT_STALL_TEST: for testing the failure path only.  A value t in (0, 1] (seconds) makes
 *     the first group barrier of every fused Lanczos iteration wait for one block more than the
 *     launch has (a participant that never arrives) and limits every wait of that kernel to t, so
 *     the waits run out and the step returns TDVP_ERR_DEVICE_TIMEOUT (nothing faults or hangs; the
 *     context stays usable, the state must be initialised again).  0 (default) = off.
 *   TDVP_OPT_ENV_FP64: 1 = in the mixed precisions the environment updates (Eq. tdvp1_h1i,
 *     tdvp1_hiN) stay FP64 and only the Lanczos matvecs run on the tensor cores; 0 (default) = the
 *     environment updates use the tensor cores too.  An environment error is seen by every H_eff
 *     of the following sweep, while a matvec error stays inside one Krylov space.
 *   TDVP_OPT_LANCZOS_CHUNKS: at most this many chunks (thread blocks) per Lanczos vector, 1..148
 *     (default 148); fewer chunks make the fused iteration's partial-sum reductions and group
 *     barriers shorter.  Results depend on it only through the summation order. */
#define TDVP_OPT_RANK_RTOL         1
#define TDVP_OPT_KRYLOV_CHECK_ALL  2
#define TDVP_OPT_QR_KERNEL         3
#define TDVP_OPT_GRAPH             4
#define TDVP_OPT_PDL               5
#define TDVP_OPT_FUSED_LANCZOS     6
#define TDVP_OPT_STALL_TEST        7
#define TDVP_OPT_LANCZOS_CHUNKS    8
#define TDVP_OPT_ENV_FP64          9
int tdvp_set_option(tdvp_ctx* ctx, int option, double value);

const char* tdvp_last_error(const tdvp_ctx* ctx);
void tdvp_destroy(tdvp_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* TDVP_H */
