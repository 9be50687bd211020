// Internal declarations shared by the CUDA translation units of libtdvp.
//
// Layout conventions (row-major, complex interleaved as double2):
//   site tensor        A[l][s][r]                   Dl*d*Dr
//   left environment   L[w][l'][l]   (sites < i)    Wl*Dl*Dl   (h[1:i-1] of Eq. tdvp1_h1i)
//   right environment  R[w][r'][r]   (sites > i)    Wr*Dr*Dr   (h[i+1:N] of Eq. tdvp1_hiN)
//   MPO                W[w][w'][s'][s]               (Eq. mpo; s' is the bra index)
//   contraction scratch T[c][x][s][y] with channel c, x = left bond, y = right bond.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

typedef double2 zc;

// Programmatic dependent launch: a kernel launched with launch_pdl may be scheduled while its
// predecessor in the stream is still running; it calls pdl_wait() before touching any memory and
// lets its own successor start early with pdl_trigger().  In a kernel launched without the
// attribute both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_enter() { pdl_wait(); pdl_trigger(); }

extern int g_tdvp_pdl;   // 1: launch_pdl sets the programmatic-serialization attribute

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = g_tdvp_pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

#define TDVP_KMAX_HARD 128        // largest Krylov dimension supported
#define TDVP_KFLAG_DONE (1 << 20) // finished-solve bit of a Krylov flag word: k | notconv << 16 | this
#define TDVP_VEC_THREADS 256      // threads of the Lanczos vector kernels
#define TDVP_MAX_VEC_BLOCKS 148   // chunks per vector: at most one block per SM, so that no SM
                                  // carries two chunks of one vector
#define TDVP_VEC_CHUNK 32         // elements per chunk before the cap, so that a 64 x 64 bond
                                  // vector also spreads over 128 SMs
#define TDVP_QR_THREADS 256

// Learned Krylov controller (kernels_mlp.cu): 8 features -> 64 -> 64 -> two heads, the Krylov
// dimension (linear) and the acceptance logit of that dimension (logistic)
#define MLP_NIN 8
#define MLP_NH 64
#define MLP_NPARAM_K (MLP_NIN * MLP_NH + MLP_NH + MLP_NH * MLP_NH + MLP_NH + MLP_NH + 1)   // trunk + k head
#define MLP_NPARAM (MLP_NPARAM_K + MLP_NH + 1)                                              // + acceptance head

__host__ __device__ __forceinline__ zc zmake(double re, double im) { return make_double2(re, im); }
__host__ __device__ __forceinline__ zc zadd(zc a, zc b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ zc zsub(zc a, zc b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ zc zconj(zc a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ zc zscale(zc a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ zc zmul(zc a, zc b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc + a*b
__host__ __device__ __forceinline__ zc zfma(zc a, zc b, zc acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
// acc + conj(a)*b
__host__ __device__ __forceinline__ zc zcfma(zc a, zc b, zc acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
  return acc;
}
// acc - a*b
__host__ __device__ __forceinline__ zc zfms(zc a, zc b, zc acc) {
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(-a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
  return acc;
}
__host__ __device__ __forceinline__ double zabs2(zc a) { return a.x * a.x + a.y * a.y; }

// Sparse MPO action used by the middle contraction stage:
//   out[co][x][so][y] = sum_e val[e] * in[ci[e]][x][si[e]][y],  e in row (co*d + so).
struct WCsr {
  const int* ptr;     // [n_out*d + 1]
  const int* ci;      // input channel
  const int* si;      // input local index
  const double* val;  // coefficient (the Hamiltonian is real)
};

// One site of one realisation.
struct SiteDev {
  zc* A;        // [Dl][d][Dr]
  zc* Lenv;     // [Wl][Dl][Dl]
  zc* Renv;     // [Wr][Dr][Dr]
  int Dl, d, Dr, Wl, Wr;
  WCsr fw;      // rows (w', s'), entries (w, s): used in H_eff.A and the left environment
  WCsr bw;      // rows (w, s'), entries (w', s): used in the right environment
};

// Krylov (Lanczos) state of one realisation for the exponential in flight.
struct KState {
  double alpha[TDVP_KMAX_HARD];
  double beta[TDVP_KMAX_HARD];
  zc coef[TDVP_KMAX_HARD];     // ||v|| * exp(z T_k) e_1 once done
  double nrm;                  // ||v|| of the start vector
  double inv_beta;             // 1/beta_j of the last accepted step
  double err;                  // last a-posteriori estimate
  int k;                       // Krylov dimension when done
  int done;                    // 1: the remaining iteration kernels of this solve are no-ops
  int kcap;                    // min(kmax, vector length)
  int n;                       // vector length of the solve
  int notconv;                 // stopped at kcap above tolerance
  int status;                  // 0 ok, TDVP_ERR_NAN ...
  int kpred;                   // Krylov dimension predicted by the learned controller (0: none)
  int jcur;                    // iteration index of a device-driven (graph) loop
  float feat[MLP_NIN];         // controller features of the solve in flight
  // counters of device-driven solves (read and cleared by the host after a graph replay)
  long long dim_sum;
  int dim_max, solves, nc_count, pad2;
};

// Per-realisation work buffers.
struct WorkDev {
  zc* x;        // matvec input (current Krylov vector)            [nmax]
  zc* w;        // matvec output / residual                        [nmax]
  zc* V;        // Krylov basis, V_t = V + t*ldV                   [kmax*ldV]
  long long ldV;
  zc* T1;       // contraction scratch                             [Wmax*nmax]
  zc* T2;       // contraction scratch                             [Wmax*nmax]
  zc* bond;     // bond matrix D                                   [Dmax*Dmax]
  zc* bond2;    // second square buffer (transfer matrices)        [Dmax*Dmax]
  zc* scratch;  // QR transpose buffer                             [nmax]
  zc* part;     // partial sums, 3 tables of [TDVP_MAX_VEC_BLOCKS][TDVP_KMAX_HARD+2]
  zc* qpart;    // QR partial sums [qr_blocks][Dmax+4] x 3
  zc* qhp;      // QR completion coefficients [Dmax]
  double* colsq;// QR column norms [d*Dmax]
  zc* qtail;    // QR rank-deficient tail: row backup [Dmax*d*Dmax], two coefficient tables
                // [Dmax][Dmax], per-block residual norms [Dmax][148] (as doubles)
  double* obs;  // observables: [n_el] <n>, then <Psi|Psi>, energy numerator
  KState* ks;
  // tensor-core operands (packed tiles, see kernels_tc.cu)
  char* tc_l;   // A operand: left environment stacked [(w l')][l]
  char* tc_r;   // B operand: right environment [r'][(w r)]
  char* tc_x;   // B operand: the Lanczos vector
  char* tc_t2;  // A operand of the third stage
  char* tc_e1;  // A operand of an environment update (site tensor, its conjugate or adjoint)
  char* tc_e2;  // B operand of an environment update (environment rows or the MPO stage)
  float* tc_t1; // first-stage output, planar FP32 (re plane, then im plane)
  long long tc_t1_plane;
  int* kprev;   // [2*N] last Krylov dimension per (site, kind)
  int* tri_count; // tridiagonal exponentials evaluated (convergence tests)
  unsigned* lzc;  // [0] blocks of the second orthogonalisation pass that have finished (reset by the
                  // last), [1] group-barrier word of the fused iteration kernel (both reset per solve)
  unsigned* bar;// [0]=count, [1]=generation of the QR group barrier
  int* err;     // device-side error flag of this realisation
};

// Operation selectors of the batched complex GEMM (descriptors are derived on the device).
enum GemmOp {
  OP_MV1 = 0,   // T1[w] = L_w x                     (H_eff stage 1)
  OP_MV3,       // w = sum_w' T2[w'] R_w'^T           (H_eff stage 3)
  OP_EL1,       // T1[w] = L_w A                     (left environment stage 1)
  OP_EL3,       // Lnew_w' = A^H T2[w']              (left environment stage 3)
  OP_ER1,       // T1[w'] = A R_w'^T                 (right environment stage 1)
  OP_ER3,       // Rnew_w = conj(A) T2[w]^T          (right environment stage 3)
  OP_Z1,        // T1[w] = Lb_w x                    (zero-site stage 1)
  OP_Z3,        // w = sum_w T1[w] Rb_w^T            (zero-site stage 2)
  OP_ABS_L,     // x = D A_{i+1}                     (gauge centre moves right)
  OP_ABS_R,     // x = A_{i-1} D                     (gauge centre moves left)
  OP_TR1,       // T1 = E A                          (transfer pass, norm/populations)
  OP_TR3,       // E' = A^H T1
  OP_HX1,       // T1[w] = L_w A  with x = site tensor (energy: H_eff C)
};

// Precision mode word of the tensor-core path (kernels_tc.cu): bit 0 hi/lo split operands
// (compensated products), bit 1 BF16 operands (kind::f16; else TF32, kind::tf32), bit 2 the
// three-product (Gauss, "3M") complex form.
#define TC_PM_SPLIT 1
#define TC_PM_BF16 2
#define TC_PM_GAUSS 4

// Tensor-core GEMMs of the mixed-precision matvecs.
// Tensor-core GEMMs: the Lanczos matvec stages (skipped once the solve is done) and the
// environment updates of the mixed-precision sweep.
enum TcOp { TC_MV1 = 0, TC_MV3 = 1, TC_Z1 = 2, TC_Z3 = 3, TC_EL1 = 4, TC_EL3 = 5, TC_ER1 = 6, TC_ER3 = 7 };

struct GemmDesc {
  const zc* A;
  const zc* B;
  zc* C;
  int M, N, K;
  int lda, ldb, ldc;
  int nz;                 // inner sum: C = sum_z op(A_z) op(B_z)
  long long sAz, sBz;
  int opA, opB;           // 0: as stored, 1: transpose, 2: conjugate transpose, 3: conjugate
  const int* skip;        // if non-null and *skip != 0 the block does nothing
  zc* ws;                 // workspace for split-K partials (null: split-K not allowed)
};

struct Ctx;  // host context (tdvp_ctx.cu)

// Kernel launchers (each returns the cudaError_t of the launch).
cudaError_t launch_gemm(int op, int site, const SiteDev* sd, const WorkDev* wk, int R, int N_sites,
                        int maxM, int maxN, int nbatch, int nsplit, cudaStream_t st);
cudaError_t launch_wapply(int dir, int site, int lanczos, const SiteDev* sd, const WorkDev* wk, int R,
                          int N_sites, int max_xy, int n_rows, cudaStream_t st);
cudaError_t launch_transpose_site(int to_scratch, int site, const SiteDev* sd, const WorkDev* wk, int R,
                                  int N_sites, int maxRows, int maxCols, cudaStream_t st);

// Lanczos (kind: 0 = site vector of `site`, 1 = bond matrix between `site` and `site+1`).
struct LzArgs {
  const SiteDev* sd;
  const WorkDev* wk;
  int R, N_sites, site, kind;
  int src;          // start vector: 0 = x buffer, 1 = site tensor, 2 = bond buffer
  int dst;          // result: 1 = site tensor, 2 = bond buffer, 3 = w buffer
  double theta;     // z = i*theta (purely imaginary exponent)
  double tol;
  int kmax;
  int jcheck;       // convergence is tested only once k >= jcheck
  int nblk;         // chunks per vector (max over realisations)
  int bcap;         // at most this many chunks per vector (<= TDVP_MAX_VEC_BLOCKS)
  int pack_pm;      // >= 0: also write each new Krylov vector as the packed tensor-core B operand
                    // of the next matvec (TC_PM_* mode word), so no separate pack launch is needed
  unsigned long long wait_ns;   // group-barrier wait limit of the fused iteration kernel
  int stall;        // test of the failure path: the first barrier of the fused iteration waits for
                    // one more block than the launch has, so every block's bounded wait runs out
  int* flags;       // [R] device: k | notconv << 16 | TDVP_KFLAG_DONE once a solve is done, -1 on failure
  const float* mlp; // learned controller weights (null: tests start at jcheck)
  float* log;       // solve log rows [8 features, k] (null: no logging)
  unsigned* log_count;
  long long log_cap;
  // device-driven loop (CUDA graph with a conditional while node per solve)
  int devj;                          // 1: the iteration index comes from KState::jcur
  cudaGraphConditionalHandle cond;   // loop condition set by lz_loop_ctl
  unsigned* loop_iters;              // [loop_id] body executions, for launch accounting
  int loop_id;
};

// Controller inference by the first MLP_NH threads of a block: returns the predicted Krylov
// dimension y (head 1) to every thread and the acceptance logit of that dimension (head 2) in
// *za.  `sm` holds at least 3*MLP_NH + MLP_NIN floats of shared memory.
__device__ __forceinline__ float mlp_infer(const float* feat, const float* w, float* sm, float* za) {
  float* x = sm;
  float* h1 = sm + MLP_NIN;
  float* h2 = h1 + MLP_NH;
  float* h4 = h2 + MLP_NH;
  const int j = threadIdx.x;
  if (j < MLP_NIN) x[j] = feat[j];
  __syncthreads();
  if (j < MLP_NH) {
    float z = w[MLP_NIN * MLP_NH + j];
    for (int i = 0; i < MLP_NIN; ++i) z = fmaf(x[i], w[i * MLP_NH + j], z);
    h1[j] = fmaxf(z, 0.f);
  }
  __syncthreads();
  const int ow2 = MLP_NIN * MLP_NH + MLP_NH, ob2 = ow2 + MLP_NH * MLP_NH, ow3 = ob2 + MLP_NH;
  const int ow4 = MLP_NPARAM_K;
  if (j < MLP_NH) {
    float z = w[ob2 + j];
    for (int i = 0; i < MLP_NH; ++i) z = fmaf(h1[i], w[ow2 + i * MLP_NH + j], z);
    const float h = fmaxf(z, 0.f);
    h2[j] = h * w[ow3 + j];
    h4[j] = h * w[ow4 + j];
  }
  __syncthreads();
  if (j == 0) {
    float y = w[ow3 + MLP_NH], a = w[ow4 + MLP_NH];
    for (int i = 0; i < MLP_NH; ++i) { y += h2[i]; a += h4[i]; }
    x[0] = y;
    x[1] = a;
  }
  __syncthreads();
  const float y = x[0];
  *za = x[1];
  __syncthreads();
  return y;
}
cudaError_t launch_lz_start(const LzArgs& a, cudaStream_t st);
cudaError_t launch_lz_iter_pre(const LzArgs& a, int j, cudaStream_t st);   // orthogonalisation
cudaError_t launch_lz_iter_post(const LzArgs& a, int j, cudaStream_t st);  // tridiagonal exp, next vector
cudaError_t launch_lz_combine(const LzArgs& a, cudaStream_t st);
// One whole Lanczos iteration in one cooperative launch (dots, both Gram-Schmidt passes, the
// tridiagonal step, the next vector), with bounded group barriers between its phases; every block
// of a realisation must be co-resident, so a.nblk * a.R <= lz_iter_capacity().
cudaError_t launch_lz_iter(const LzArgs& a, int j, cudaStream_t st);
int lz_iter_capacity(int device);
// loop control of a device-driven solve: which = 0 before the loop (condition = some solve not
// done), 1 at the end of the body (advance the iteration index of unfinished solves, count the
// body execution, condition = some solve not done)
cudaError_t launch_lz_loop_ctl(const LzArgs& a, int which, cudaStream_t st);

// QR of the gauge shift (dir 0: left-to-right on site tensor via transpose scratch, result
// L = Q in A[site], D = R in bond; dir 1: right-to-left LQ in place, D = L-factor in bond;
// dir 2: debug matrix in scratch (n x m rows), R to bond).
cudaError_t launch_row_qr(int dir, int site, const SiteDev* sd, const WorkDev* wk, int R, int N_sites,
                          int blocks_per_r, double rtol, int dbg_n, int dbg_m, cudaStream_t st);
int qr_max_coresident_blocks(int device);

// The same decomposition by one thread-block cluster of C CTAs per realisation with the matrix in
// shared memory (kernels_cqr.cu).  dir 0 works on A[site] through its transposed view (no
// transpose pass), dir 1 on A[site] in place, dir 2 on the debug matrix in scratch, dir 3 and 4
// on scratch with the right-to-left / left-to-right shape of the site (autotuning).  `smem` must
// be at least cqr_smem_bytes of the largest realisation's shape and at most TDVP_CQR_SMEM_MAX.
#define TDVP_CQR_SMEM_MAX (220 * 1024)
long long cqr_smem_bytes(int n, int m, int C);
cudaError_t cqr_setup(int device);
int cqr_max_clusters(int C, long long smem);
cudaError_t launch_cluster_qr(int dir, int site, const SiteDev* sd, const WorkDev* wk, int R, int N_sites, int C,
                              long long smem, double rtol, int dbg_n, int dbg_m, cudaStream_t st);

// Observables helpers.
cudaError_t launch_set_identity_bond2(const WorkDev* wk, int R, int n, cudaStream_t st);
cudaError_t launch_obs_local(int site, int slot, const SiteDev* sd, const WorkDev* wk, int R, int N_sites,
                             cudaStream_t st);
cudaError_t launch_obs_norm(int site, int slot, const WorkDev* wk, int R, cudaStream_t st);
cudaError_t launch_obs_energy(int slot, const SiteDev* sd, const WorkDev* wk, int R, int N_sites,
                              cudaStream_t st);
cudaError_t launch_copy_vec(int what, int site, const SiteDev* sd, const WorkDev* wk, int R, int N_sites,
                            int maxn, cudaStream_t st);
cudaError_t launch_reset_ks(const WorkDev* wk, int R, cudaStream_t st);

// Tensor-core path (kernels_tc.cu)
long long tc_pack_bytes(int rows_tile, long long rows, long long K);
cudaError_t tc_setup();
// maxM x maxN output over maxK bound every realisation's product; long-K products are split over
// a thread-block cluster (tc_splits)
int tc_splits(int tiles, int R, int maxK);
// S_force > 0: that many CTAs per output tile along K (a power of two <= 8, at most the K tiles),
// else the tc_splits heuristic
cudaError_t launch_tc_gemm(int op, int site, const SiteDev* sd, const WorkDev* wk, int R, int N_sites, int maxM,
                           int maxN, int maxK, int pm, cudaStream_t st, int S_force = 0);
cudaError_t launch_pack_env(int which, int site, const SiteDev* sd, const WorkDev* wk, int R, int N_sites,
                            long long max_elems, int pm, cudaStream_t st);
cudaError_t launch_pack_x(int kind, int site, const SiteDev* sd, const WorkDev* wk, int R, int N_sites,
                          long long max_elems, int pm, cudaStream_t st);
// Environment updates on the tensor cores (kernels_tc.cu).  which = 0: left (site i -> Lenv of
// i+1), 1: right (site i -> Renv of i-1).  Stage operands:
//   pack_site (kind 0) A^H as A operand [r'][(l s)]; (kind 1) A as A operand [(l s)][r];
//             (kind 2) conj(A) as A operand [l'][(s r)]; (kind 3) A as B operand [(s r)][l]
//   pack_renv_rows: R as B operand [(w' r')][r]
//   wapply_env (which 0) T2[(l' s')][(w' r)] as B operand [(w' r)][(l' s')];
//              (which 1) T2[w][(l s')][r'] as B operand [(w l)][(s' r')]
// Every pack covers the padded tiles (zeros outside the valid region).
cudaError_t launch_pack_site(int kind, int site, const SiteDev* sd, const WorkDev* wk, int R, int N_sites,
                             long long max_rows, long long max_k, int pm, cudaStream_t st);
cudaError_t launch_pack_renv_rows(int site, const SiteDev* sd, const WorkDev* wk, int R, int N_sites,
                                  long long max_rows, long long max_k, int pm, cudaStream_t st);
cudaError_t launch_wapply_env(int which, int site, const SiteDev* sd, const WorkDev* wk, int R, int N_sites,
                              long long max_rows, long long max_k, int pm, cudaStream_t st);
cudaError_t launch_wapply_tc(int site, const SiteDev* sd, const WorkDev* wk, int R, int N_sites, int max_xy,
                             int n_rows, int pm, cudaStream_t st);

// Controller training (kernels_mlp.cu).  head 0: mean-squared error of the Krylov dimension
// (gradient over the trunk and head 1); head 1: logistic loss of the acceptance of the predicted
// dimension (gradient over head 2 only, the trunk is frozen).  grad[MLP_NPARAM] receives the loss,
// which is also added to *loss_acc when that is non-null.  The Adam step updates params [p0, p1).
int mlp_partial_floats(int B);
cudaError_t launch_mlp_grad(int head, const float* data, long long idx0, int B, const float* w, float* partial,
                            float* grad, float* loss_acc, cudaStream_t st);
cudaError_t launch_mlp_adam(float* w, const float* g, float* m, float* v, float lr, int t, int p0, int p1,
                            cudaStream_t st);
