// Host side of libtdvp: context, MPO construction, initial states, the TDVP-PS sweep driver
// (Eq. ps_trotter), observables and the component entry points.  All arithmetic on the state is
// done by the kernels in kernels_*.cu; this file sizes buffers, builds the device tables and
// enqueues launches on the caller's stream.
#include "tdvp_internal.cuh"
#include "../../include/tdvp.h"

#include <algorithm>
#include <cmath>
#include <map>
#include <random>
#include <tuple>
#include <cstring>
#include <string>
#include <vector>

namespace {

constexpr double kPhasePerCmFs = 2.0 * 3.14159265358979323846 * 2.99792458e-5;   // 2 pi c
constexpr double kRankRtolDefault = 1e-13;

struct RealHost {
  bool mpo = false, mps = false;
  std::vector<int> bd;                 // bond dims, N+1
  std::vector<void*> mpo_allocs;       // CSR buffers
  std::vector<void*> mps_allocs;       // tensors, environments, work buffers
  std::vector<std::vector<double>> W;  // dense MPO per site [Wl][Wr][d][d]
};

}  // namespace

int g_tdvp_pdl = 1;

struct tdvp_ctx {
  int dev = 0;
  cudaStream_t st = nullptr;
  int R = 1;
  int kmax = 64;
  // chain layout (shared by all realisations)
  int N = 0, n_el = 0;
  std::vector<int> d, Wb, is_el, label;   // Wb: MPO bond dims N+1
  std::vector<int> n_modes, levels;        // layout check
  std::vector<int> el_order;
  std::vector<RealHost> rh;
  std::vector<SiteDev> h_sites;
  SiteDev* d_sites = nullptr;
  std::vector<WorkDev> h_work;
  WorkDev* d_work = nullptr;
  int* d_flags = nullptr;
  int* h_flags = nullptr;     // pinned
  int* d_err = nullptr;       // [R] device error words
  int* h_err = nullptr;       // pinned
  double* h_obs = nullptr;    // pinned, (n_el+4) per realisation
  std::vector<int> khist;     // last Krylov dim per (site, kind)
  std::vector<long long> ws_cap;   // elements of T1 (= T2) per realisation
  int qr_cap = 0;
  double rank_rtol = kRankRtolDefault;
  // (R, m, n) -> QR kernel: B > 0 grid kernel with B blocks per realisation, -C cluster kernel
  std::map<std::tuple<int, int, int>, int> qr_tuned;
  // (op, R, M, N, K) of a Lanczos-matvec tensor-core GEMM -> CTAs per output tile along K
  std::map<std::tuple<int, int, int, int, int>, int> tc_tuned;
  int qr_force = -1;          // TDVP_OPT_QR_KERNEL
  bool cqr_ok[17] = {};       // cluster size launchable with the largest shared-memory slab
  int check_every = 0;        // 1: test Lanczos convergence at every k (else from the last k - 2 on)
  int fused_lz = 1;           // TDVP_OPT_FUSED_LANCZOS: one cooperative launch per Lanczos iteration
  double stall_test = 0.0;    // TDVP_OPT_STALL_TEST: > 0 = failure-path test with this wait limit (s)
  int lz_chunks = TDVP_MAX_VEC_BLOCKS;   // TDVP_OPT_LANCZOS_CHUNKS: chunk cap per Lanczos vector
  int env_fp64 = 0;           // TDVP_OPT_ENV_FP64: environment updates in FP64 in the mixed precisions
  int lz_cap = 0;             // co-resident blocks of the fused iteration kernel
  // per-launch timing
  // learned Krylov controller
  float* d_mlp = nullptr;           // weights (MLP_NPARAM)
  float* d_mlp_m = nullptr;         // Adam moments
  float* d_mlp_v = nullptr;
  int mlp_ready = 0;
  int mlp_step = 0;
  float* d_log = nullptr;           // solve log [cap][MLP_NIN + 1]
  unsigned* d_log_count = nullptr;
  long long log_cap = 0;
  int logging = 0;
  int l_site = -1, r_site = -1;     // site whose environment is packed in tc_l / tc_r
  int l_pm = -1, r_pm = -1;
  int prof = 0;
  int krylov_mode = TDVP_KRYLOV_ADAPTIVE;
  // CUDA-graph execution of whole steps (TDVP_OPT_GRAPH)
  int graph_on = 0;
  bool capturing = false;
  cudaStream_t body_st = nullptr;      // captures the body of each Lanczos while-node
  cudaStream_t cap_st = nullptr;       // captures the step
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<double> gkey;            // configuration the graph was captured for
  unsigned* d_loop_iters = nullptr;    // [loop] body executions since the last read
  int loop_cap = 0, loop_n = 0;
  std::vector<int> loop_body_launches; // kernels per body execution of each loop
  long long graph_outer_launches = 0;  // kernels of one replay outside the loops
  int graph_nc = 0;                    // a replayed solve stopped at kmax above the tolerance
  std::vector<cudaEvent_t> ev;   // pairs
  std::vector<int> ev_cat;
  std::vector<int> ev_phase;
  int phase = TDVP_PH_OTHER;     // sub-step the launches being enqueued serve (TDVP_PH_*)
  size_t ev_used = 0;
  std::string err;
  tdvp_stats_t stats{};
};

namespace {

int fail(tdvp_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? TDVP_ERR_OOM : TDVP_ERR_CUDA,       \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                        \
  } while (0)

int prof_begin(tdvp_ctx* ctx, int cat);
int prof_end(tdvp_ctx* ctx);

#define LAUNCHC(cat, call)                                    \
  do {                                                        \
    if (ctx->prof) { int pr_ = prof_begin(ctx, cat); if (pr_) return pr_; } \
    CK(call);                                                 \
    if (ctx->prof) { int pr_ = prof_end(ctx); if (pr_) return pr_; }        \
    ctx->stats.kernel_launches++;                             \
  } while (0)
#define LAUNCH(call) LAUNCHC(TDVP_CAT_OTHER, call)

template <class T>
int dalloc(tdvp_ctx* ctx, std::vector<void*>& owner, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return fail(ctx, TDVP_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  cudaMemsetAsync(q, 0, std::max<size_t>(count, 1) * sizeof(T), ctx->st);
  owner.push_back(q);
  *p = static_cast<T*>(q);
  return TDVP_OK;
}

void free_all(std::vector<void*>& v) {
  for (void* p : v) cudaFree(p);
  v.clear();
}

int prof_begin(tdvp_ctx* ctx, int cat) {
  if (ctx->ev_used + 2 > ctx->ev.size()) {
    for (int q = 0; q < 512; ++q) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      ctx->ev.push_back(e);
    }
    ctx->ev_cat.resize(ctx->ev.size() / 2);
    ctx->ev_phase.resize(ctx->ev.size() / 2);
  }
  ctx->ev_cat[ctx->ev_used / 2] = cat;
  ctx->ev_phase[ctx->ev_used / 2] = ctx->phase;
  CK(cudaEventRecord(ctx->ev[ctx->ev_used], ctx->st));
  return TDVP_OK;
}

int prof_end(tdvp_ctx* ctx) {
  CK(cudaEventRecord(ctx->ev[ctx->ev_used + 1], ctx->st));
  ctx->ev_used += 2;
  return TDVP_OK;
}

// Fold the recorded event pairs into the statistics (synchronises the stream).
int prof_collect(tdvp_ctx* ctx) {
  if (ctx->ev_used == 0) return TDVP_OK;
  CK(cudaStreamSynchronize(ctx->st));
  for (size_t q = 0; q < ctx->ev_used; q += 2) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ctx->ev[q], ctx->ev[q + 1]));
    const int cat = ctx->ev_cat[q / 2];
    ctx->stats.prof_ms[cat] += ms;
    ctx->stats.prof_launches[cat]++;
    const int ph = ctx->ev_phase[q / 2];
    ctx->stats.prof_phase_ms[ph] += ms;
    ctx->stats.prof_phase_launches[ph]++;
  }
  ctx->ev_used = 0;
  return TDVP_OK;
}

// Books the launches enqueued while it lives under one sub-step (TDVP_PH_*), then restores the
// previous one.
struct PhaseScope {
  tdvp_ctx* ctx;
  int saved;
  PhaseScope(tdvp_ctx* c, int ph) : ctx(c), saved(c->phase) { c->phase = ph; }
  ~PhaseScope() { ctx->phase = saved; }
};

// ---------------------------------------------------------------------------------------------
// MPO of Eq. holstein as a finite-state machine (Eq. mpo).  Channel 0 of a cut = nothing placed,
// channel 1 = a complete term placed.  A cut with k electronic sites to its left (of M) carries
// 2*min(k, M-k) hopping channels, labelled by the left site while k <= M-k (an a^+ or a placed
// there, waiting for its partner), afterwards by the right site n (sum_m J a_m^+ or sum_m J a_m
// placed, waiting for a_n or a_n^+ at n).  Inside the mode block of electronic site m one more
// channel carries n_m waiting for (b^+ + b) on one of its modes.  The left end keeps only
// channel 0, the right end only channel 1.
struct MpoBuilder {
  int N, M;
  std::vector<int> d, is_el, label, elpos, nleft;   // elpos: position of label along el order
  std::vector<int> order;
  bool zpe;
  double off;
  const double *E, *J, *om, *gg;
  std::vector<int> mode_index;   // flat mode index of vib sites

  int regime_left(int k) const { return k <= M - k; }       // true: channels indexed by left sites
  int nhop(int k) const { return 2 * std::min(k, M - k); }
  bool has_ph(int cut) const { return cut > 0 && cut < N && !is_el[cut]; }
  int width(int cut) const {
    if (cut == 0 || cut == N) return 1;
    return 2 + nhop(nleft[cut]) + (has_ph(cut) ? 1 : 0);
  }
  // channel index; kind: 0 idle, 1 done, 2 cr(j), 3 an(j), 4 ph ; j = position along el order
  int chan(int cut, int kind, int j) const {
    if (cut == 0) return kind == 0 ? 0 : -1;
    if (cut == N) return kind == 1 ? 0 : -1;
    const int k = nleft[cut];
    if (kind <= 1) return kind;
    if (kind == 4) return has_ph(cut) ? 2 + nhop(k) : -1;
    int slot;
    if (regime_left(k)) { if (j < 0 || j >= k) return -1; slot = j; }
    else { if (j < k || j >= M) return -1; slot = j - k; }
    return 2 + 2 * slot + (kind == 2 ? 0 : 1);
  }
};

void add_op(std::vector<double>& T, int Wr, int dd, int wl, int wr, const std::vector<double>& op, double coef) {
  if (wl < 0 || wr < 0 || coef == 0.0) return;
  double* base = &T[((size_t)wl * Wr + wr) * dd * dd];
  for (int q = 0; q < dd * dd; ++q) base[q] += coef * op[q];
}

// drop a captured step graph (its shapes, options or tables may no longer hold)
void graph_reset(tdvp_ctx* ctx) {
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  ctx->gexec = nullptr;
  ctx->graph = nullptr;
  ctx->gkey.clear();
}

}  // namespace

// --------------------------------------------------------------------------------------------- ABI
extern "C" {

int tdvp_create(tdvp_ctx** out, int device, void* cuda_stream, int n_realisations, int kmax) {
  if (!out || n_realisations < 1 || kmax < 1 || kmax > TDVP_KMAX_HARD) return TDVP_ERR_INVALID_ARG;
  *out = nullptr;
  tdvp_ctx* ctx = new tdvp_ctx();
  ctx->dev = device;
  ctx->st = static_cast<cudaStream_t>(cuda_stream);
  ctx->R = n_realisations;
  ctx->kmax = kmax;
  ctx->rh.resize(n_realisations);
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) { delete ctx; return TDVP_ERR_CUDA; }
  if (cudaMalloc(&ctx->d_work, sizeof(WorkDev) * ctx->R) != cudaSuccess ||
      cudaMalloc(&ctx->d_flags, sizeof(int) * ctx->R) != cudaSuccess ||
      cudaMalloc(&ctx->d_err, sizeof(int) * ctx->R) != cudaSuccess ||
      cudaMallocHost(&ctx->h_flags, sizeof(int) * ctx->R) != cudaSuccess ||
      cudaMallocHost(&ctx->h_err, sizeof(int) * ctx->R) != cudaSuccess) {
    tdvp_destroy(ctx);
    return TDVP_ERR_OOM;
  }
  cudaMemsetAsync(ctx->d_err, 0, sizeof(int) * ctx->R, ctx->st);
  ctx->h_work.assign(ctx->R, WorkDev{});
  ctx->ws_cap.assign(ctx->R, 0);
  ctx->qr_cap = qr_max_coresident_blocks(device);
  ctx->lz_cap = lz_iter_capacity(device);
  if (tc_setup() != cudaSuccess) { tdvp_destroy(ctx); return TDVP_ERR_CUDA; }
  if (cqr_setup(device) != cudaSuccess) { tdvp_destroy(ctx); return TDVP_ERR_CUDA; }
  for (int C : {1, 2, 4, 8, 16}) ctx->cqr_ok[C] = cqr_max_clusters(C, TDVP_CQR_SMEM_MAX) >= 1;
  if (ctx->qr_cap < 1) { tdvp_destroy(ctx); return TDVP_ERR_CUDA; }
  *out = ctx;
  return TDVP_OK;
}

void tdvp_destroy(tdvp_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->dev);
  if (ctx->st) cudaStreamSynchronize(ctx->st); else cudaDeviceSynchronize();
  for (auto& r : ctx->rh) { free_all(r.mpo_allocs); free_all(r.mps_allocs); }
  cudaFree(ctx->d_sites);
  cudaFree(ctx->d_work);
  cudaFree(ctx->d_flags);
  cudaFree(ctx->d_err);
  cudaFreeHost(ctx->h_flags);
  cudaFreeHost(ctx->h_err);
  cudaFreeHost(ctx->h_obs);
  cudaFree(ctx->d_mlp);
  cudaFree(ctx->d_mlp_m);
  cudaFree(ctx->d_mlp_v);
  cudaFree(ctx->d_log);
  cudaFree(ctx->d_log_count);
  graph_reset(ctx);
  if (ctx->body_st) cudaStreamDestroy(ctx->body_st);
  if (ctx->cap_st) cudaStreamDestroy(ctx->cap_st);
  cudaFree(ctx->d_loop_iters);
  for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
  delete ctx;
}

const char* tdvp_last_error(const tdvp_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int tdvp_build_mpo(tdvp_ctx* ctx, int r, const tdvp_fh_params* p) {
  if (!ctx) return TDVP_ERR_INVALID_ARG;
  graph_reset(ctx);
  if (r < 0 || r >= ctx->R || !p || p->n_el < 1 || !p->E || !p->J || !p->n_modes || !p->el_order)
    return fail(ctx, TDVP_ERR_INVALID_ARG, "build_mpo: bad arguments");
  CK(cudaSetDevice(ctx->dev));
  const int M = p->n_el;
  int nm_tot = 0;
  for (int m = 0; m < M; ++m) {
    if (p->n_modes[m] < 0) return fail(ctx, TDVP_ERR_INVALID_ARG, "build_mpo: negative n_modes");
    nm_tot += p->n_modes[m];
  }
  if (nm_tot > 0 && (!p->omega || !p->g || !p->n_levels))
    return fail(ctx, TDVP_ERR_INVALID_ARG, "build_mpo: mode arrays missing");
  std::vector<int> seen(M, 0);
  for (int j = 0; j < M; ++j) {
    const int m = p->el_order[j];
    if (m < 0 || m >= M || seen[m]) return fail(ctx, TDVP_ERR_INVALID_ARG, "build_mpo: el_order is not a permutation");
    seen[m] = 1;
  }
  for (int m = 0; m < M; ++m)
    for (int n = 0; n < M; ++n)
      if (m != n && p->J[m * M + n] != p->J[n * M + m])
        return fail(ctx, TDVP_ERR_INVALID_ARG, "build_mpo: J must be symmetric");
  std::vector<int> mode_off(M, 0);
  for (int m = 1; m < M; ++m) mode_off[m] = mode_off[m - 1] + p->n_modes[m - 1];
  for (int q = 0; q < nm_tot; ++q)
    if (p->n_levels[q] < 1 || p->n_levels[q] > 64) return fail(ctx, TDVP_ERR_INVALID_ARG, "build_mpo: n_levels out of range");

  // chain layout
  MpoBuilder B;
  B.M = M; B.zpe = p->include_zpe != 0; B.off = p->energy_offset;
  B.E = p->E; B.J = p->J; B.om = p->omega; B.gg = p->g;
  B.order.assign(p->el_order, p->el_order + M);
  B.elpos.assign(M, 0);
  for (int j = 0; j < M; ++j) B.elpos[B.order[j]] = j;
  for (int j = 0; j < M; ++j) {
    const int m = B.order[j];
    B.d.push_back(2); B.is_el.push_back(1); B.label.push_back(m); B.mode_index.push_back(-1);
    for (int q = 0; q < p->n_modes[m]; ++q) {
      B.d.push_back(p->n_levels[mode_off[m] + q]); B.is_el.push_back(0); B.label.push_back(m);
      B.mode_index.push_back(mode_off[m] + q);
    }
  }
  B.N = (int)B.d.size();
  B.nleft.assign(B.N + 1, 0);
  for (int c = 1; c <= B.N; ++c) B.nleft[c] = B.nleft[c - 1] + B.is_el[c - 1];

  std::vector<int> nmv(p->n_modes, p->n_modes + M);
  std::vector<int> lev(p->n_levels, p->n_levels + nm_tot);
  if (ctx->N == 0) {
    ctx->N = B.N; ctx->n_el = M; ctx->d = B.d; ctx->is_el = B.is_el; ctx->label = B.label;
    ctx->n_modes = nmv; ctx->levels = lev; ctx->el_order = B.order;
    ctx->Wb.resize(B.N + 1);
    for (int c = 0; c <= B.N; ++c) ctx->Wb[c] = B.width(c);
    ctx->h_sites.assign((size_t)ctx->R * ctx->N, SiteDev{});
    CK(cudaMalloc(&ctx->d_sites, sizeof(SiteDev) * ctx->R * ctx->N));
    CK(cudaMallocHost(&ctx->h_obs, sizeof(double) * (M + 4) * ctx->R));
    ctx->khist.assign(2 * ctx->N, 0);
  } else if (ctx->n_el != M || ctx->n_modes != nmv || ctx->levels != lev || ctx->el_order != B.order) {
    return fail(ctx, TDVP_ERR_INVALID_ARG, "build_mpo: chain layout differs from realisation 0");
  }
  RealHost& H = ctx->rh[r];
  if (H.mps) return fail(ctx, TDVP_ERR_STATE, "build_mpo: realisation already initialised");
  free_all(H.mpo_allocs);
  H.W.assign(B.N, {});

  for (int i = 0; i < B.N; ++i) {
    const int dd = B.d[i], Wl = B.width(i), Wr = B.width(i + 1);
    std::vector<double>& T = H.W[i];
    T.assign((size_t)Wl * Wr * dd * dd, 0.0);
    // local operators, op[s'*dd + s]
    std::vector<double> I(dd * dd, 0.0);
    for (int s = 0; s < dd; ++s) I[s * dd + s] = 1.0;
    const int cl = i, cr = i + 1;
    add_op(T, Wr, dd, B.chan(cl, 0, 0), B.chan(cr, 0, 0), I, 1.0);
    add_op(T, Wr, dd, B.chan(cl, 1, 0), B.chan(cr, 1, 0), I, 1.0);
    if (B.is_el[i]) {
      const int m = B.label[i], jm = B.elpos[m];
      std::vector<double> cre(4, 0.0), ann(4, 0.0), num(4, 0.0);
      cre[1 * 2 + 0] = 1.0;   // |1><0|
      ann[0 * 2 + 1] = 1.0;   // |0><1|
      num[1 * 2 + 1] = 1.0;
      add_op(T, Wr, dd, B.chan(cl, 0, 0), B.chan(cr, 1, 0), num, B.E[m] - B.off);
      add_op(T, Wr, dd, B.chan(cl, 0, 0), B.chan(cr, 4, 0), num, 1.0);
      const int kL = B.nleft[cl], kR = B.nleft[cr];
      const bool leftL = B.regime_left(kL), leftR = B.regime_left(kR);
      // terms completed here (this site is the right partner)
      if (leftL) {
        for (int j = 0; j < kL; ++j) {
          const int src = B.order[j];
          add_op(T, Wr, dd, B.chan(cl, 2, j), B.chan(cr, 1, 0), ann, B.J[src * M + m]);
          add_op(T, Wr, dd, B.chan(cl, 3, j), B.chan(cr, 1, 0), cre, B.J[m * M + src]);
        }
      } else {
        add_op(T, Wr, dd, B.chan(cl, 2, jm), B.chan(cr, 1, 0), ann, 1.0);
        add_op(T, Wr, dd, B.chan(cl, 3, jm), B.chan(cr, 1, 0), cre, 1.0);
      }
      // terms opened here (this site is the left partner)
      if (leftR) {
        add_op(T, Wr, dd, B.chan(cl, 0, 0), B.chan(cr, 2, jm), cre, 1.0);
        add_op(T, Wr, dd, B.chan(cl, 0, 0), B.chan(cr, 3, jm), ann, 1.0);
      } else {
        for (int j = kR; j < M; ++j) {
          const int n = B.order[j];
          add_op(T, Wr, dd, B.chan(cl, 0, 0), B.chan(cr, 2, j), cre, B.J[m * M + n]);
          add_op(T, Wr, dd, B.chan(cl, 0, 0), B.chan(cr, 3, j), ann, B.J[n * M + m]);
        }
      }
      // pending terms passing through
      if (leftL && leftR) {
        for (int j = 0; j < kL; ++j) {
          add_op(T, Wr, dd, B.chan(cl, 2, j), B.chan(cr, 2, j), I, 1.0);
          add_op(T, Wr, dd, B.chan(cl, 3, j), B.chan(cr, 3, j), I, 1.0);
        }
      } else if (leftL && !leftR) {
        for (int j = 0; j < kL; ++j) {
          const int src = B.order[j];
          for (int q = kR; q < M; ++q) {
            const int n = B.order[q];
            add_op(T, Wr, dd, B.chan(cl, 2, j), B.chan(cr, 2, q), I, B.J[src * M + n]);
            add_op(T, Wr, dd, B.chan(cl, 3, j), B.chan(cr, 3, q), I, B.J[n * M + src]);
          }
        }
      } else {
        for (int q = kR; q < M; ++q) {
          add_op(T, Wr, dd, B.chan(cl, 2, q), B.chan(cr, 2, q), I, 1.0);
          add_op(T, Wr, dd, B.chan(cl, 3, q), B.chan(cr, 3, q), I, 1.0);
        }
      }
    } else {
      const int q = B.mode_index[i];
      const double w = B.om[q], g = B.gg[q];
      std::vector<double> nb(dd * dd, 0.0), xb(dd * dd, 0.0);
      for (int s = 0; s < dd; ++s) nb[s * dd + s] = s;
      for (int s = 1; s < dd; ++s) {
        const double v = std::sqrt((double)s);
        xb[(s - 1) * dd + s] = v;   // b
        xb[s * dd + (s - 1)] = v;   // b^+
      }
      add_op(T, Wr, dd, B.chan(cl, 0, 0), B.chan(cr, 1, 0), nb, w);
      if (B.zpe) add_op(T, Wr, dd, B.chan(cl, 0, 0), B.chan(cr, 1, 0), I, 0.5 * w);
      add_op(T, Wr, dd, B.chan(cl, 4, 0), B.chan(cr, 1, 0), xb, g * w);
      add_op(T, Wr, dd, B.chan(cl, 4, 0), B.chan(cr, 4, 0), I, 1.0);
      const int k = B.nleft[cl];
      const int lo = B.regime_left(k) ? 0 : k, hi = B.regime_left(k) ? k : M;
      for (int j = lo; j < hi; ++j) {
        add_op(T, Wr, dd, B.chan(cl, 2, j), B.chan(cr, 2, j), I, 1.0);
        add_op(T, Wr, dd, B.chan(cl, 3, j), B.chan(cr, 3, j), I, 1.0);
      }
    }
    // CSR of the middle stage: forward rows (w', s') and backward rows (w, s')
    std::vector<int> fptr(Wr * dd + 1, 0), bptr(Wl * dd + 1, 0);
    std::vector<int> fci, fsi, bci, bsi;
    std::vector<double> fval, bval;
    for (int wr = 0; wr < Wr; ++wr)
      for (int so = 0; so < dd; ++so) {
        for (int wl = 0; wl < Wl; ++wl)
          for (int s = 0; s < dd; ++s) {
            const double v = T[(((size_t)wl * Wr + wr) * dd + so) * dd + s];
            if (v != 0.0) { fci.push_back(wl); fsi.push_back(s); fval.push_back(v); }
          }
        fptr[wr * dd + so + 1] = (int)fval.size();
      }
    for (int wl = 0; wl < Wl; ++wl)
      for (int so = 0; so < dd; ++so) {
        for (int wr = 0; wr < Wr; ++wr)
          for (int s = 0; s < dd; ++s) {
            const double v = T[(((size_t)wl * Wr + wr) * dd + so) * dd + s];
            if (v != 0.0) { bci.push_back(wr); bsi.push_back(s); bval.push_back(v); }
          }
        bptr[wl * dd + so + 1] = (int)bval.size();
      }
    SiteDev& S = ctx->h_sites[(size_t)r * ctx->N + i];
    int *dfp, *dfc, *dfs, *dbp, *dbc, *dbs;
    double *dfv, *dbv;
    int rc;
    if ((rc = dalloc(ctx, H.mpo_allocs, &dfp, fptr.size()))) return rc;
    if ((rc = dalloc(ctx, H.mpo_allocs, &dfc, fci.size()))) return rc;
    if ((rc = dalloc(ctx, H.mpo_allocs, &dfs, fsi.size()))) return rc;
    if ((rc = dalloc(ctx, H.mpo_allocs, &dfv, fval.size()))) return rc;
    if ((rc = dalloc(ctx, H.mpo_allocs, &dbp, bptr.size()))) return rc;
    if ((rc = dalloc(ctx, H.mpo_allocs, &dbc, bci.size()))) return rc;
    if ((rc = dalloc(ctx, H.mpo_allocs, &dbs, bsi.size()))) return rc;
    if ((rc = dalloc(ctx, H.mpo_allocs, &dbv, bval.size()))) return rc;
    CK(cudaMemcpy(dfp, fptr.data(), fptr.size() * sizeof(int), cudaMemcpyHostToDevice));
    if (!fci.empty()) {
      CK(cudaMemcpy(dfc, fci.data(), fci.size() * sizeof(int), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(dfs, fsi.data(), fsi.size() * sizeof(int), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(dfv, fval.data(), fval.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    CK(cudaMemcpy(dbp, bptr.data(), bptr.size() * sizeof(int), cudaMemcpyHostToDevice));
    if (!bci.empty()) {
      CK(cudaMemcpy(dbc, bci.data(), bci.size() * sizeof(int), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(dbs, bsi.data(), bsi.size() * sizeof(int), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(dbv, bval.data(), bval.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    S.fw = WCsr{dfp, dfc, dfs, dfv};
    S.bw = WCsr{dbp, dbc, dbs, dbv};
    S.d = dd; S.Wl = Wl; S.Wr = Wr;
  }
  H.mpo = true;
  return TDVP_OK;
}

}  // extern "C"

// --------------------------------------------------------------------------------------------
// internal helpers
namespace {

inline int cdivi(long long a, long long b) { return (int)((a + b - 1) / b); }

struct Views {
  const SiteDev* sd;
  const WorkDev* wk;
  int R;
  int* flags;
  int r0;
};

// maxima over the realisations in [r0, r0+R)
struct Dims { int Dl, Dr; };
Dims maxdims(tdvp_ctx* ctx, int site, const Views& v) {
  Dims m{0, 0};
  for (int r = v.r0; r < v.r0 + v.R; ++r) {
    m.Dl = std::max(m.Dl, ctx->rh[r].bd[site]);
    m.Dr = std::max(m.Dr, ctx->rh[r].bd[site + 1]);
  }
  return m;
}

Views all_views(tdvp_ctx* ctx) { return Views{ctx->d_sites, ctx->d_work, ctx->R, ctx->d_flags, 0}; }
Views one_view(tdvp_ctx* ctx, int r) {
  return Views{ctx->d_sites + (size_t)r * ctx->N, ctx->d_work + r, 1, ctx->d_flags + r, r};
}

// tensor-core precision mode word (TC_PM_* bits) of a TDVP_PREC_* value (mixed precisions only)
int tc_mode(int P) {
  switch (P) {
    case TDVP_PREC_TF32X3: return TC_PM_SPLIT;
    case TDVP_PREC_BF16: return TC_PM_BF16;
    case TDVP_PREC_BF16X3: return TC_PM_BF16 | TC_PM_SPLIT;
    case TDVP_PREC_TF32_3M: return TC_PM_GAUSS;
    case TDVP_PREC_BF16_3M: return TC_PM_BF16 | TC_PM_GAUSS;
    default: return 0;   // TDVP_PREC_TF32
  }
}

// autotuned split-K of a tensor-core GEMM shape (0: the heuristic)
int tc_split_pick(tdvp_ctx* ctx, int op, int R, int M, int N, int K) {
  auto it = ctx->tc_tuned.find(std::make_tuple(op, R, M, N, K));
  return it == ctx->tc_tuned.end() ? 0 : it->second;
}

// algorithmic real flops of one batched GEMM launch (8 per complex multiply-add)
double gemm_flops(tdvp_ctx* ctx, const Views& v, int op, int site) {
  double f = 0;
  for (int r = v.r0; r < v.r0 + v.R; ++r) {
    const auto& bd = ctx->rh[r].bd;
    const double Dl = bd[site], Dr = bd[site + 1], d = ctx->d[site];
    const double Wl = ctx->Wb[site], Wr = ctx->Wb[site + 1];
    switch (op) {
      case OP_MV1: case OP_EL1: case OP_HX1: f += Wl * Dl * d * Dr * Dl; break;
      case OP_MV3: f += Wr * Dl * d * Dr * Dr; break;
      case OP_EL3: f += Wr * Dr * Dr * Dl * d; break;
      case OP_ER1: f += Wr * Dl * d * Dr * Dr; break;
      case OP_ER3: f += Wl * Dl * Dl * d * Dr; break;
      case OP_Z1: case OP_Z3: f += Wr * Dr * Dr * Dr; break;
      case OP_ABS_L: { const double Dn = bd[site + 2 <= (int)bd.size() - 1 ? site + 2 : site + 1];
                       f += Dr * Dr * ctx->d[site + 1] * Dn; break; }
      case OP_ABS_R: { const double Dp = bd[site - 1]; f += Dp * ctx->d[site - 1] * Dl * Dl; break; }
      case OP_TR1: f += Dl * Dl * d * Dr; break;
      case OP_TR3: f += Dr * Dr * Dl * d; break;
    }
  }
  return 8.0 * f;
}

// K splits for a GEMM with few output tiles: enough blocks to cover every SM twice, limited by the
// inner tile count and by the workspace (T1 or T2 of each realisation, ws_cap elements).
int split_for(tdvp_ctx* ctx, const Views& v, int op, int site, int M, int Nn, int nb) {
  const bool splittable = op == OP_MV3 || op == OP_EL3 || op == OP_ER3 || op == OP_Z1 || op == OP_Z3 || op == OP_TR3;
  if (!splittable) return 1;
  const long long tiles = (long long)cdivi(M, 32) * cdivi(Nn, 32) * nb * v.R;
  if (tiles >= 296) return 1;
  int K = 0, nz = 1;
  const Dims m = maxdims(ctx, site, v);
  switch (op) {
    case OP_MV3: K = m.Dr; nz = ctx->Wb[site + 1]; break;
    case OP_EL3: K = m.Dl * ctx->d[site]; break;
    case OP_ER3: K = ctx->d[site] * m.Dr; break;
    case OP_Z1: K = m.Dr; break;
    case OP_Z3: K = m.Dr; nz = ctx->Wb[site + 1]; break;
    case OP_TR3: K = m.Dl * ctx->d[site]; break;
  }
  const int kt = nz * cdivi(K, 16);
  int S = (int)std::min<long long>(cdivi(296, tiles), 16);
  S = std::min(S, kt);
  long long cap = 1LL << 62;
  for (int r = v.r0; r < v.r0 + v.R; ++r) cap = std::min(cap, ctx->ws_cap[r]);
  const long long need_per_split = (long long)nb * M * Nn;
  S = (int)std::min<long long>(S, cap / std::max(1LL, need_per_split));
  return std::max(1, S);
}

int g_op(tdvp_ctx* ctx, const Views& v, int op, int site, int M, int Nn, int nb) {
  const int S = split_for(ctx, v, op, site, M, Nn, nb);
  LAUNCHC(TDVP_CAT_GEMM, launch_gemm(op, site, v.sd, v.wk, v.R, ctx->N, M, Nn, nb, S, ctx->st));
  if (S > 1) ctx->stats.kernel_launches++;     // the split-K reduction
  if (ctx->prof) ctx->stats.prof_flops[TDVP_CAT_GEMM] += gemm_flops(ctx, v, op, site);
  return TDVP_OK;
}

int matvec_site(tdvp_ctx* ctx, const Views& v, int i, int first_op) {
  const Dims m = maxdims(ctx, i, v);
  const int d = ctx->d[i], Wl = ctx->Wb[i], Wr = ctx->Wb[i + 1];
  int rc;
  if ((rc = g_op(ctx, v, first_op, i, m.Dl, d * m.Dr, Wl))) return rc;
  LAUNCHC(TDVP_CAT_WAPPLY, launch_wapply(0, i, first_op == OP_MV1 ? 1 : 0, v.sd, v.wk, v.R, ctx->N, m.Dl * m.Dr, Wr * d, ctx->st));
  return g_op(ctx, v, OP_MV3, i, m.Dl * d, m.Dr, 1);
}

int matvec_bond(tdvp_ctx* ctx, const Views& v, int i) {
  const Dims m = maxdims(ctx, i, v);
  const int Wr = ctx->Wb[i + 1];
  int rc;
  if ((rc = g_op(ctx, v, OP_Z1, i, m.Dr, m.Dr, Wr))) return rc;
  return g_op(ctx, v, OP_Z3, i, m.Dr, m.Dr, 1);
}

// ---- mixed-precision matvecs on the tensor cores ----
// bytes of one packed tensor-core operand of realisation r (which: 0 L, 1 R, 2 x of a site
// solve, 3 x of a bond solve, 4 T2 of a site solve, 5 T of a bond solve)
long long used_bytes(tdvp_ctx* ctx, int r, int which, int site) {
  const auto& bd = ctx->rh[r].bd;
  const long long Dl = bd[site], Dr = bd[site + 1], d = ctx->d[site];
  const long long Wl = ctx->Wb[site], Wr = ctx->Wb[site + 1];
  switch (which) {
    case 0: return tc_pack_bytes(128, Wl * Dl, Dl);
    case 1: return tc_pack_bytes(64, Dr, Wr * Dr);
    case 2: return tc_pack_bytes(64, d * Dr, Dl);
    case 3: return tc_pack_bytes(64, Dr, Dr);
    case 4: return tc_pack_bytes(128, Dl * d, Wr * Dr);
    default: return tc_pack_bytes(128, Dr, Wr * Dr);
  }
}

// zero the used part of one tensor-core operand buffer in every realisation of the view
int memset_tc(tdvp_ctx* ctx, const Views& v, int field, int which, int site) {
  for (int r = v.r0; r < v.r0 + v.R; ++r) {
    const WorkDev& W = ctx->h_work[r];
    void* p = field == 0 ? (void*)W.tc_l : field == 1 ? (void*)W.tc_r : field == 2 ? (void*)W.tc_x : (void*)W.tc_t2;
    CK(cudaMemsetAsync(p, 0, (size_t)used_bytes(ctx, r, which, site), ctx->st));
  }
  return TDVP_OK;
}

int ensure_env_packs(tdvp_ctx* ctx, const Views& v, int lsite, int rsite, int pm);

// the left environment of `site` packed in tc_l (kept while it stays valid)
int ensure_l_pack(tdvp_ctx* ctx, const Views& v, int site, int pm) {
  if (ctx->l_site == site && ctx->l_pm == pm) return TDVP_OK;
  int rc = memset_tc(ctx, v, 0, 0, site);
  if (rc) return rc;
  const Dims m = maxdims(ctx, site, v);
  LAUNCH(launch_pack_env(0, site, v.sd, v.wk, v.R, ctx->N, (long long)ctx->Wb[site] * m.Dl * m.Dl, pm, ctx->st));
  ctx->l_site = site;
  ctx->l_pm = pm;
  return TDVP_OK;
}

// Left update on the tensor cores: T1 = L A (stage 1, as the matvec's), the MPO stage written as
// the B operand of the last stage, Lenv(i+1) = A^H T2.
int env_left_tc(tdvp_ctx* ctx, const Views& v, int i, int pm) {
  const Dims m = maxdims(ctx, i, v);
  const int d = ctx->d[i], Wl = ctx->Wb[i], Wr = ctx->Wb[i + 1];
  int rc;
  if ((rc = ensure_l_pack(ctx, v, i, pm))) return rc;
  LAUNCH(launch_pack_site(3, i, v.sd, v.wk, v.R, ctx->N, (long long)d * m.Dr, m.Dl, pm, ctx->st));
  LAUNCHC(TDVP_CAT_TC, launch_tc_gemm(TC_EL1, i, v.sd, v.wk, v.R, ctx->N, Wl * m.Dl, d * m.Dr, m.Dl, pm, ctx->st));
  LAUNCHC(TDVP_CAT_WAPPLY, launch_wapply_env(0, i, v.sd, v.wk, v.R, ctx->N, (long long)Wr * m.Dr, (long long)m.Dl * d,
                                             pm, ctx->st));
  LAUNCH(launch_pack_site(0, i, v.sd, v.wk, v.R, ctx->N, m.Dr, (long long)m.Dl * d, pm, ctx->st));
  LAUNCHC(TDVP_CAT_TC, launch_tc_gemm(TC_EL3, i, v.sd, v.wk, v.R, ctx->N, m.Dr, Wr * m.Dr, m.Dl * d, pm, ctx->st));
  if (ctx->l_site == i + 1) ctx->l_site = -1;
  if (ctx->prof) {
    double f = 0;
    for (int r = v.r0; r < v.r0 + v.R; ++r) {
      const auto& bd = ctx->rh[r].bd;
      const double Dl = bd[i], Dr = bd[i + 1];
      f += 8.0 * (Wl * Dl * d * Dr * Dl + Dr * Wr * Dr * Dl * d);
    }
    ctx->stats.prof_flops[TDVP_CAT_TC] += f;
  }
  return TDVP_OK;
}

// Right update on the tensor cores: T1 = A R^T (all w' at once), the backward MPO stage written as
// the B operand of the last stage, Renv(i-1) = conj(A) T2^T.
int env_right_tc(tdvp_ctx* ctx, const Views& v, int i, int pm) {
  const Dims m = maxdims(ctx, i, v);
  const int d = ctx->d[i], Wl = ctx->Wb[i], Wr = ctx->Wb[i + 1];
  LAUNCH(launch_pack_site(1, i, v.sd, v.wk, v.R, ctx->N, (long long)m.Dl * d, m.Dr, pm, ctx->st));
  LAUNCH(launch_pack_renv_rows(i, v.sd, v.wk, v.R, ctx->N, (long long)Wr * m.Dr, m.Dr, pm, ctx->st));
  LAUNCHC(TDVP_CAT_TC, launch_tc_gemm(TC_ER1, i, v.sd, v.wk, v.R, ctx->N, m.Dl * d, Wr * m.Dr, m.Dr, pm, ctx->st));
  LAUNCHC(TDVP_CAT_WAPPLY, launch_wapply_env(1, i, v.sd, v.wk, v.R, ctx->N, (long long)Wl * m.Dl, (long long)d * m.Dr,
                                             pm, ctx->st));
  LAUNCH(launch_pack_site(2, i, v.sd, v.wk, v.R, ctx->N, m.Dl, (long long)d * m.Dr, pm, ctx->st));
  LAUNCHC(TDVP_CAT_TC, launch_tc_gemm(TC_ER3, i, v.sd, v.wk, v.R, ctx->N, m.Dl, Wl * m.Dl, d * m.Dr, pm, ctx->st));
  if (ctx->r_site == i - 1) ctx->r_site = -1;
  if (ctx->prof) {
    double f = 0;
    for (int r = v.r0; r < v.r0 + v.R; ++r) {
      const auto& bd = ctx->rh[r].bd;
      const double Dl = bd[i], Dr = bd[i + 1];
      f += 8.0 * (Dl * d * Wr * Dr * Dr + Dl * Wl * Dl * d * Dr);
    }
    ctx->stats.prof_flops[TDVP_CAT_TC] += f;
  }
  return TDVP_OK;
}

int ensure_env_packs(tdvp_ctx* ctx, const Views& v, int lsite, int rsite, int pm) {
  if (ctx->l_site != lsite || ctx->l_pm != pm) {
    int rc = memset_tc(ctx, v, 0, 0, lsite);
    if (rc) return rc;
    const Dims m = maxdims(ctx, lsite, v);
    LAUNCH(launch_pack_env(0, lsite, v.sd, v.wk, v.R, ctx->N, (long long)ctx->Wb[lsite] * m.Dl * m.Dl, pm, ctx->st));
    ctx->l_site = lsite;
    ctx->l_pm = pm;
  }
  if (ctx->r_site != rsite || ctx->r_pm != pm) {
    int rc = memset_tc(ctx, v, 1, 1, rsite);
    if (rc) return rc;
    const Dims m = maxdims(ctx, rsite, v);
    LAUNCH(launch_pack_env(1, rsite, v.sd, v.wk, v.R, ctx->N, (long long)ctx->Wb[rsite + 1] * m.Dr * m.Dr, pm, ctx->st));
    ctx->r_site = rsite;
    ctx->r_pm = pm;
  }
  return TDVP_OK;
}

// clear the per-solve tensor-core operands (their geometry changes from solve to solve)
int prepare_tc_solve(tdvp_ctx* ctx, const Views& v, int kind, int site, int pm) {
  PhaseScope ps(ctx, kind == 0 ? TDVP_PH_DERIV_FWD : TDVP_PH_DERIV_BWD);
  int rc;
  if (kind == 0) {
    if ((rc = ensure_env_packs(ctx, v, site, site, pm))) return rc;
    if ((rc = memset_tc(ctx, v, 2, 2, site))) return rc;
    return memset_tc(ctx, v, 3, 4, site);
  }
  if ((rc = ensure_env_packs(ctx, v, site + 1, site, pm))) return rc;
  if ((rc = memset_tc(ctx, v, 2, 3, site))) return rc;
  return memset_tc(ctx, v, 3, 5, site);
}

// prepacked: the Lanczos kernels have already written x as the packed B operand
int matvec_site_tc(tdvp_ctx* ctx, const Views& v, int i, int pm, bool prepacked = false) {
  const Dims m = maxdims(ctx, i, v);
  const int d = ctx->d[i], Wl = ctx->Wb[i], Wr = ctx->Wb[i + 1];
  if (!prepacked) LAUNCH(launch_pack_x(0, i, v.sd, v.wk, v.R, ctx->N, (long long)m.Dl * d * m.Dr, pm, ctx->st));
  LAUNCHC(TDVP_CAT_TC, launch_tc_gemm(TC_MV1, i, v.sd, v.wk, v.R, ctx->N, Wl * m.Dl, d * m.Dr, m.Dl, pm, ctx->st,
                                      tc_split_pick(ctx, TC_MV1, v.R, Wl * m.Dl, d * m.Dr, m.Dl)));
  LAUNCHC(TDVP_CAT_WAPPLY, launch_wapply_tc(i, v.sd, v.wk, v.R, ctx->N, m.Dl * m.Dr, Wr * d, pm, ctx->st));
  LAUNCHC(TDVP_CAT_TC, launch_tc_gemm(TC_MV3, i, v.sd, v.wk, v.R, ctx->N, m.Dl * d, m.Dr, Wr * m.Dr, pm, ctx->st,
                                      tc_split_pick(ctx, TC_MV3, v.R, m.Dl * d, m.Dr, Wr * m.Dr)));
  if (ctx->prof) {
    double f = 0;
    for (int r = v.r0; r < v.r0 + v.R; ++r) {
      const auto& bd = ctx->rh[r].bd;
      const double Dl = bd[i], Dr = bd[i + 1];
      f += 8.0 * (Wl * Dl * d * Dr * Dl + Dl * d * Dr * Wr * Dr);
    }
    ctx->stats.prof_flops[TDVP_CAT_TC] += f;
  }
  return TDVP_OK;
}

int matvec_bond_tc(tdvp_ctx* ctx, const Views& v, int i, int pm, bool prepacked = false) {
  const Dims m = maxdims(ctx, i, v);
  const int Wb = ctx->Wb[i + 1];
  if (!prepacked) LAUNCH(launch_pack_x(1, i, v.sd, v.wk, v.R, ctx->N, (long long)m.Dr * m.Dr, pm, ctx->st));
  LAUNCHC(TDVP_CAT_TC, launch_tc_gemm(TC_Z1, i, v.sd, v.wk, v.R, ctx->N, Wb * m.Dr, m.Dr, m.Dr, pm, ctx->st,
                                      tc_split_pick(ctx, TC_Z1, v.R, Wb * m.Dr, m.Dr, m.Dr)));
  LAUNCHC(TDVP_CAT_TC, launch_tc_gemm(TC_Z3, i, v.sd, v.wk, v.R, ctx->N, m.Dr, m.Dr, Wb * m.Dr, pm, ctx->st,
                                      tc_split_pick(ctx, TC_Z3, v.R, m.Dr, m.Dr, Wb * m.Dr)));
  if (ctx->prof) {
    double f = 0;
    for (int r = v.r0; r < v.r0 + v.R; ++r) {
      const double Db = ctx->rh[r].bd[i + 1];
      f += 8.0 * 2.0 * Wb * Db * Db * Db;
    }
    ctx->stats.prof_flops[TDVP_CAT_TC] += f;
  }
  return TDVP_OK;
}

int env_left_tc(tdvp_ctx* ctx, const Views& v, int i, int pm);
int env_right_tc(tdvp_ctx* ctx, const Views& v, int i, int pm);

// Left environment of site i+1 from site i (Eq. tdvp1_h1i); FP64, or TF32 / TF32x3 on the
// tensor cores in the mixed-precision sweep.
int env_left(tdvp_ctx* ctx, const Views& v, int i, int P = TDVP_PREC_FP64) {
  PhaseScope ps(ctx, TDVP_PH_GET_ENV);
  if (P != TDVP_PREC_FP64 && !ctx->env_fp64) return env_left_tc(ctx, v, i, tc_mode(P));
  const Dims m = maxdims(ctx, i, v);
  const int d = ctx->d[i], Wl = ctx->Wb[i], Wr = ctx->Wb[i + 1];
  int rc;
  if (ctx->l_site == i + 1) ctx->l_site = -1;
  if ((rc = g_op(ctx, v, OP_EL1, i, m.Dl, d * m.Dr, Wl))) return rc;
  LAUNCHC(TDVP_CAT_WAPPLY, launch_wapply(0, i, 0, v.sd, v.wk, v.R, ctx->N, m.Dl * m.Dr, Wr * d, ctx->st));
  return g_op(ctx, v, OP_EL3, i, m.Dr, m.Dr, Wr);
}

// Right environment of site i-1 from site i (Eq. tdvp1_hiN); FP64 or on the tensor cores.
int env_right(tdvp_ctx* ctx, const Views& v, int i, int P = TDVP_PREC_FP64) {
  PhaseScope ps(ctx, TDVP_PH_GET_ENV);
  if (P != TDVP_PREC_FP64 && !ctx->env_fp64) return env_right_tc(ctx, v, i, tc_mode(P));
  const Dims m = maxdims(ctx, i, v);
  const int d = ctx->d[i], Wl = ctx->Wb[i], Wr = ctx->Wb[i + 1];
  int rc;
  if (ctx->r_site == i - 1) ctx->r_site = -1;
  if ((rc = g_op(ctx, v, OP_ER1, i, m.Dl * d, m.Dr, Wr))) return rc;
  LAUNCHC(TDVP_CAT_WAPPLY, launch_wapply(1, i, 0, v.sd, v.wk, v.R, ctx->N, m.Dl * m.Dr, Wl * d, ctx->st));
  return g_op(ctx, v, OP_ER3, i, m.Dl, m.Dl, Wl);
}

int qr_grid_default(tdvp_ctx* ctx, int R, int m) {
  int B = cdivi(m, 8);
  B = std::max(1, std::min(B, 148));
  return std::min(B, std::max(1, ctx->qr_cap / std::max(1, R)));
}

bool cqr_fits(tdvp_ctx* ctx, int C, int m, int n) {
  return C >= 1 && C <= 16 && ctx->cqr_ok[C] && C <= m && cqr_smem_bytes(n, m, C) <= TDVP_CQR_SMEM_MAX;
}

// QR kernel for an (n x m) shape over R realisations: B > 0 grid kernel, -C cluster kernel
int qr_mode(tdvp_ctx* ctx, int R, int m, int n) {
  if (ctx->qr_force == 0) return qr_grid_default(ctx, R, m);
  if (ctx->qr_force > 0) return -ctx->qr_force;
  if (ctx->qr_force == -2) {
    for (int C : {16, 8, 4, 2, 1})
      if (cqr_fits(ctx, C, m, n)) return -C;
    return qr_grid_default(ctx, R, m);
  }
  auto it = ctx->qr_tuned.find(std::make_tuple(R, m, n));
  if (it != ctx->qr_tuned.end()) return it->second;
  return qr_grid_default(ctx, R, m);
}

// One QR launch.  dir: 0 left-to-right on A[site], 1 right-to-left on A[site], 2 debug matrix,
// 3 / 4 autotune shapes on scratch (right-to-left / left-to-right).  (m, n) bound every
// realisation's shape.
int run_qr(tdvp_ctx* ctx, const Views& v, int dir, int i, int m, int n, int mode, double rtol, int dn, int dm) {
  if (mode < 0) {
    const int C = -mode;
    if (!cqr_fits(ctx, C, m, n)) return fail(ctx, TDVP_ERR_INVALID_ARG, "QR: shape does not fit the cluster kernel");
    CK(launch_cluster_qr(dir, i, v.sd, v.wk, v.R, ctx->N, C, cqr_smem_bytes(n, m, C), rtol, dn, dm, ctx->st));
    ctx->stats.kernel_launches++;
    return TDVP_OK;
  }
  const int gdir = dir == 4 ? 0 : dir;      // the grid kernel's left-to-right shape lives in scratch
  if (dir == 0) CK(launch_transpose_site(1, i, v.sd, v.wk, v.R, ctx->N, m, n, ctx->st));
  // the cooperative grid kernel needs every block it launches co-resident: realisations go in
  // groups of at most qr_cap / B per launch
  const int G = std::max(1, ctx->qr_cap / std::max(1, mode));
  for (int r0 = 0; r0 < v.R; r0 += G) {
    const int Rg = std::min(G, v.R - r0);
    CK(launch_row_qr(gdir, i, v.sd + (size_t)r0 * ctx->N, v.wk + r0, Rg, ctx->N, mode, rtol, dn, dm, ctx->st));
    ctx->stats.kernel_launches++;
  }
  if (dir == 0) CK(launch_transpose_site(0, i, v.sd, v.wk, v.R, ctx->N, m, n, ctx->st));
  ctx->stats.kernel_launches += dir == 0 ? 2 : 0;
  return TDVP_OK;
}

// run_qr inside one profiling interval of category `cat`
int run_qr_timed(tdvp_ctx* ctx, int cat, const Views& v, int dir, int i, int m, int n, int mode, double rtol,
                 int dn, int dm) {
  if (ctx->prof) { int pr = prof_begin(ctx, cat); if (pr) return pr; }
  const int rc = run_qr(ctx, v, dir, i, m, n, mode, rtol, dn, dm);
  if (rc) return rc;
  if (ctx->prof) { int pr = prof_end(ctx); if (pr) return pr; }
  return TDVP_OK;
}

// dir 0: C_i = L_i D (left-to-right), dir 1: C_i = D R_i (right-to-left); D lands in `bond`
// Runs of consecutive realisations of a view whose gauge-shift QR at site i (direction dir, 0 =
// left-to-right, else right-to-left) has the same (m, n) shape.  Ragged realisations differ in
// cost by ~(D_max/D_min)^3; one launch over all of them with one block count leaves most SMs idle
// while the largest finish, so every run gets its own launch and block count.
struct QrRun { int r0, R, m, n; };
std::vector<QrRun> qr_runs(tdvp_ctx* ctx, const Views& v, int i, int dir) {
  std::vector<QrRun> runs;
  const int d = ctx->d[i];
  for (int q = 0; q < v.R; ++q) {
    const auto& bd = ctx->rh[v.r0 + q].bd;
    const int m = dir == 0 ? bd[i] * d : d * bd[i + 1], n = dir == 0 ? bd[i + 1] : bd[i];
    if (!runs.empty() && runs.back().m == m && runs.back().n == n) runs.back().R++;
    else runs.push_back(QrRun{q, 1, m, n});
  }
  return runs;
}

Views sub_view(tdvp_ctx* ctx, const Views& v, int q0, int R) {
  return Views{v.sd + (size_t)q0 * ctx->N, v.wk + q0, R, v.flags + q0, v.r0 + q0};
}

int gauge_qr(tdvp_ctx* ctx, const Views& v, int i, int dir) {
  PhaseScope ps(ctx, TDVP_PH_QR);
  const int d = ctx->d[i];
  if (ctx->prof) {
    // algorithmic flops of the definition: two Gram-Schmidt passes (dots and updates) per row,
    // 2 n^2 m complex multiply-adds of 8 real flops
    double f = 0;
    for (int r = v.r0; r < v.r0 + v.R; ++r) {
      const auto& bd = ctx->rh[r].bd;
      const double n = dir == 0 ? bd[i + 1] : bd[i], mr = dir == 0 ? (double)bd[i] * d : (double)d * bd[i + 1];
      f += 16.0 * n * n * mr;
    }
    ctx->stats.prof_flops[TDVP_CAT_QR] += f;
  }
  for (const QrRun& run : qr_runs(ctx, v, i, dir)) {
    const Views sv = sub_view(ctx, v, run.r0, run.R);
    const int rc = run_qr_timed(ctx, TDVP_CAT_QR, sv, dir, i, run.m, run.n, qr_mode(ctx, run.R, run.m, run.n),
                                ctx->rank_rtol, 0, 0);
    if (rc) return rc;
  }
  (void)d;
  return TDVP_OK;
}

int nblk_for(long long n, int cap) {
  long long nb = (n + TDVP_VEC_CHUNK - 1) / TDVP_VEC_CHUNK;
  return (int)std::max(1LL, std::min<long long>(nb, cap));
}

// Lanczos arguments shared by the launch-by-launch and the graph-captured exponential.  The fused
// iteration kernel runs when every realisation's chunks fit co-resident (the chunk count per
// vector is capped at capacity / R for that) and that cap leaves at least 8 chunks per vector; the
// mixed precisions let the Lanczos kernels write each new Krylov vector as the packed
// tensor-core operand of the next matvec.
LzArgs lz_args(tdvp_ctx* ctx, const Views& v, int kind, int site, int src, int dst, double theta, double tol,
               int prec, bool* fused) {
  const Dims m = maxdims(ctx, site, v);
  const long long n = kind == 0 ? (long long)m.Dl * ctx->d[site] * m.Dr : (long long)m.Dr * m.Dr;
  LzArgs a{};
  a.sd = v.sd; a.wk = v.wk; a.R = v.R; a.N_sites = ctx->N; a.site = site; a.kind = kind;
  a.src = src; a.dst = dst; a.theta = theta; a.tol = tol; a.kmax = ctx->kmax;
  // fused only while every vector keeps at least 8 chunks (or all it needs) under the
  // co-residency cap: with many realisations one block per vector would leave most SMs idle
  const int want = nblk_for(n, ctx->lz_chunks);
  *fused = ctx->fused_lz && ctx->lz_cap / v.R >= std::min(8, want);
  a.bcap = *fused ? std::min(ctx->lz_chunks, ctx->lz_cap / v.R) : ctx->lz_chunks;
  a.nblk = nblk_for(n, a.bcap);
  a.pack_pm = prec != TDVP_PREC_FP64 ? tc_mode(prec) : -1;
  a.stall = ctx->stall_test > 0.0 ? 1 : 0;
  a.wait_ns = a.stall ? (unsigned long long)(ctx->stall_test * 1e9) : 1000000000ull;
  a.flags = v.flags;
  a.mlp = (ctx->krylov_mode == TDVP_KRYLOV_LEARNED && ctx->mlp_ready) ? ctx->d_mlp : nullptr;
  a.log = ctx->logging ? ctx->d_log : nullptr;
  a.log_count = ctx->d_log_count;
  a.log_cap = ctx->log_cap;
  return a;
}

// exp(i theta H) applied to the start vector `src` (0 = x, 1 = site tensor, 2 = bond) with
// H = H[site] (kind 0) or the zero-site H0 of bond (site, site+1) (kind 1); the result goes to
// `dst` (1 = site tensor, 2 = bond, 3 = w).  Returns TDVP_OK or an error; sets *notconv.
// The matvec of one Lanczos iteration (site or bond, FP64 or tensor cores).
int lanczos_matvec(tdvp_ctx* ctx, const Views& v, int kind, int site, int prec, int pm) {
  PhaseScope ps(ctx, kind == 0 ? TDVP_PH_DERIV_FWD : TDVP_PH_DERIV_BWD);
  if (prec != TDVP_PREC_FP64) {
    if (kind == 0) return matvec_site_tc(ctx, v, site, pm, true);
    return matvec_bond_tc(ctx, v, site, pm, true);
  }
  if (kind == 0) return matvec_site(ctx, v, site, OP_MV1);
  return matvec_bond(ctx, v, site);
}

// Lanczos exponential while a step is being captured into a CUDA graph: the iterations become
// the body of a conditional while node (condition default 1 at every launch, then set by
// lz_loop_ctl at the end of each body run), the iteration index lives on the device, the
// convergence tests start from the device copy of the previous Krylov dimension (or every k, or
// at the learned prediction), and results, counters and failures stay on the device until the
// host reads them after the replays.
int expm_graph(tdvp_ctx* ctx, const Views& v, int kind, int site, int src, int dst, double theta, double tol,
               int prec) {
  if (ctx->loop_n >= ctx->loop_cap) return fail(ctx, TDVP_ERR_STATE, "graph capture: too many Lanczos loops");
  bool fused = false;
  LzArgs a = lz_args(ctx, v, kind, site, src, dst, theta, tol, prec, &fused);
  a.jcheck = ctx->check_every ? 1 : 0;
  a.devj = 1;
  a.loop_iters = ctx->d_loop_iters;
  a.loop_id = ctx->loop_n++;
  CK(cudaMemsetAsync(v.flags, 0, sizeof(int) * v.R, ctx->st));
  const int pm = tc_mode(prec);
  int rc;
  if (prec != TDVP_PREC_FP64 && (rc = prepare_tc_solve(ctx, v, kind, site, pm))) return rc;
  LAUNCHC(TDVP_CAT_LZVEC, launch_lz_start(a, ctx->st));
  ctx->stats.kernel_launches++;     // two kernels
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(ctx->st, &cs, nullptr, &g, &deps, nullptr, &nd));
  if (cs != cudaStreamCaptureStatusActive) return fail(ctx, TDVP_ERR_STATE, "graph capture: stream not capturing");
  CK(cudaGraphConditionalHandleCreate(&a.cond, g, 1u, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = a.cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  CK(cudaStreamUpdateCaptureDependencies(ctx->st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  // the body: one iteration, captured from the second stream
  CK(cudaStreamBeginCaptureToGraph(ctx->body_st, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  const cudaStream_t main_st = ctx->st;
  const long long before = ctx->stats.kernel_launches;
  ctx->st = ctx->body_st;
  rc = lanczos_matvec(ctx, v, kind, site, prec, pm);
  if (!rc) {
    cudaError_t e = cudaSuccess;
    if (fused) {
      e = launch_lz_iter(a, 0, ctx->st);
    } else {
      e = launch_lz_iter_pre(a, 0, ctx->st);
      if (e == cudaSuccess) e = launch_lz_iter_post(a, 0, ctx->st);
    }
    if (e == cudaSuccess) e = launch_lz_loop_ctl(a, 1, ctx->st);
    if (e != cudaSuccess) rc = fail(ctx, TDVP_ERR_CUDA, cudaGetErrorString(e));
  }
  ctx->st = main_st;
  cudaGraph_t tmp = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(ctx->body_st, &tmp);
  if (rc) return rc;
  if (ee != cudaSuccess) return fail(ctx, TDVP_ERR_CUDA, cudaGetErrorString(ee));
  // kernels of one body run: the matvec's (counted while capturing) + the fused iteration, or
  // dots, two passes (the tridiagonal step inside the second) and next vector; loop control
  ctx->loop_body_launches.push_back((int)(ctx->stats.kernel_launches - before) + (fused ? 2 : 5));
  ctx->stats.kernel_launches = before;
  LAUNCHC(TDVP_CAT_LZVEC, launch_lz_combine(a, ctx->st));
  return TDVP_OK;
}

int check_device_errors(tdvp_ctx* ctx);

int expm(tdvp_ctx* ctx, const Views& v, int kind, int site, int src, int dst, double theta, double tol,
         int* notconv, int prec = TDVP_PREC_FP64) {
  PhaseScope ps(ctx, TDVP_PH_KRYLOV);
  if (ctx->capturing) return expm_graph(ctx, v, kind, site, src, dst, theta, tol, prec);
  bool fused = false;
  LzArgs a = lz_args(ctx, v, kind, site, src, dst, theta, tol, prec, &fused);
  int& kh = ctx->khist[2 * site + kind];
  const int guess = kh > 0 ? kh : 6;
  a.jcheck = ctx->check_every ? 1 : std::max(1, guess - 2);
  CK(cudaMemsetAsync(v.flags, 0, sizeof(int) * v.R, ctx->st));
  const int pm = tc_mode(prec);
  if (prec != TDVP_PREC_FP64) {
    int rc0 = prepare_tc_solve(ctx, v, kind, site, pm);
    if (rc0) return rc0;
  }
  LAUNCHC(TDVP_CAT_LZVEC, launch_lz_start(a, ctx->st));
  ctx->stats.kernel_launches++;     // two kernels
  int j = 0, batch = guess, rc;
  bool all_done = false;
  while (j < ctx->kmax && !all_done) {
    for (int q = 0; q < batch && j < ctx->kmax; ++q, ++j) {
      if ((rc = lanczos_matvec(ctx, v, kind, site, prec, pm))) return rc;
      if (fused) {
        LAUNCHC(TDVP_CAT_LZVEC, launch_lz_iter(a, j, ctx->st));        // the whole iteration
      } else {
        LAUNCHC(TDVP_CAT_LZVEC, launch_lz_iter_pre(a, j, ctx->st));    // three kernels (tridiagonal step inside)
        LAUNCHC(TDVP_CAT_LZVEC, launch_lz_iter_post(a, j, ctx->st));   // next vector
        ctx->stats.kernel_launches += 2;
      }
      ctx->stats.matvecs += v.R;
    }
    CK(cudaMemcpyAsync(ctx->h_flags + v.r0, v.flags, sizeof(int) * v.R, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    ctx->stats.host_syncs++;
    all_done = true;
    for (int r = 0; r < v.R; ++r) if (ctx->h_flags[v.r0 + r] == 0) all_done = false;
    batch = 2;
  }
  LAUNCHC(TDVP_CAT_LZVEC, launch_lz_combine(a, ctx->st));
  int kmaxr = 0;
  for (int r = 0; r < v.R; ++r) {
    const int f = ctx->h_flags[v.r0 + r];
    if (f < 0) return fail(ctx, TDVP_ERR_NAN, "Lanczos: non-finite value or unsupported exponent");
    if (f == 0) {
      const int de = check_device_errors(ctx);     // a timed-out wait leaves the solve unfinished
      if (de) return de;
      return fail(ctx, TDVP_ERR_KRYLOV_NOT_CONVERGED, "Lanczos: solve did not finish");
    }
    const int k = f & 0xffff;
    if ((f >> 16) & 1) { ctx->stats.not_converged++; if (notconv) *notconv = 1; }
    kmaxr = std::max(kmaxr, k);
    if (ctx->prof) {
      // algorithmic bytes of this solve's vector kernels (see tdvp_stats_t)
      const auto& bd = ctx->rh[v.r0 + r].bd;
      const double nr = kind == 0 ? (double)bd[site] * ctx->d[site] * bd[site + 1] : (double)bd[site + 1] * bd[site + 1];
      ctx->stats.prof_bytes[TDVP_CAT_LZVEC] += 16.0 * nr * (2.0 * k * (k + 1) + 10.0 * k + 5.0);
      // FP64 flops of the two classical Gram-Schmidt passes (dot and update against V_0..V_j in
      // each, 8 real flops per complex multiply-add): 32 n (j + 1) at iteration j
      ctx->stats.prof_flops[TDVP_CAT_LZVEC] += 16.0 * nr * k * (k + 1.0);
    }
    ctx->stats.krylov_dim_sum += k;
    ctx->stats.krylov_dim_max = std::max(ctx->stats.krylov_dim_max, k);
  }
  ctx->stats.krylov_solves += v.R;
  kh = kmaxr;
  return TDVP_OK;
}

int check_device_errors(tdvp_ctx* ctx) {
  CK(cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(int) * ctx->R, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  for (int r = 0; r < ctx->R; ++r)
    if (ctx->h_err[r] != 0) {
      const int code = ctx->h_err[r];
      cudaMemsetAsync(ctx->d_err, 0, sizeof(int) * ctx->R, ctx->st);
      return fail(ctx, code == -5 ? TDVP_ERR_DEVICE_TIMEOUT : ((code == -6 || code == -7) ? TDVP_ERR_NAN : TDVP_ERR_INVALID_ARG),
                  code == -5 ? "device barrier timed out"
                  : code == -6 ? "gauge-shift QR met a non-positive Gram pivot"
                  : code == -7 ? "Lanczos: non-finite value or unsupported exponent"
                               : "device kernel rejected its sizes");
    }
  return TDVP_OK;
}

int collect_tri_counts(tdvp_ctx* ctx) {
  for (int r = 0; r < ctx->R; ++r) {
    int cnt = 0;
    CK(cudaMemcpyAsync(&cnt, ctx->h_work[r].tri_count, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemsetAsync(ctx->h_work[r].tri_count, 0, sizeof(int), ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    ctx->stats.tri_evals += cnt;
  }
  return TDVP_OK;
}

int upload_tables(tdvp_ctx* ctx, int r) {
  CK(cudaMemcpyAsync(ctx->d_sites + (size_t)r * ctx->N, ctx->h_sites.data() + (size_t)r * ctx->N,
                     sizeof(SiteDev) * ctx->N, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->d_work + r, &ctx->h_work[r], sizeof(WorkDev), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return TDVP_OK;
}

// Allocate tensors, environments and work buffers of realisation r at bond dims bd.
int alloc_realisation(tdvp_ctx* ctx, int r, const std::vector<int>& bd) {
  RealHost& H = ctx->rh[r];
  free_all(H.mps_allocs);
  H.bd = bd;
  const int N = ctx->N;
  long long nmax = 1, Dmax = 1, mmax = 1;
  int Wmax = 1;
  for (int i = 0; i < N; ++i) {
    const long long n = (long long)bd[i] * ctx->d[i] * bd[i + 1];
    nmax = std::max(nmax, n);
    Dmax = std::max<long long>(Dmax, std::max(bd[i], bd[i + 1]));
    mmax = std::max<long long>(mmax, std::max<long long>((long long)bd[i] * ctx->d[i], (long long)ctx->d[i] * bd[i + 1]));
    Wmax = std::max(Wmax, std::max(ctx->Wb[i], ctx->Wb[i + 1]));
  }
  nmax = std::max(nmax, Dmax * Dmax);
  const long long ldV = (nmax + 31) / 32 * 32;
  int rc;
  for (int i = 0; i < N; ++i) {
    SiteDev& S = ctx->h_sites[(size_t)r * N + i];
    S.Dl = bd[i]; S.Dr = bd[i + 1];
    if ((rc = dalloc(ctx, H.mps_allocs, &S.A, (size_t)S.Dl * S.d * S.Dr))) return rc;
    if ((rc = dalloc(ctx, H.mps_allocs, &S.Lenv, (size_t)S.Wl * S.Dl * S.Dl))) return rc;
    if ((rc = dalloc(ctx, H.mps_allocs, &S.Renv, (size_t)S.Wr * S.Dr * S.Dr))) return rc;
  }
  WorkDev& W = ctx->h_work[r];
  W.ldV = ldV;
  if ((rc = dalloc(ctx, H.mps_allocs, &W.x, nmax))) return rc;
  if ((rc = dalloc(ctx, H.mps_allocs, &W.w, nmax))) return rc;
  if ((rc = dalloc(ctx, H.mps_allocs, &W.V, (size_t)ldV * ctx->kmax))) return rc;
  if ((rc = dalloc(ctx, H.mps_allocs, &W.T1, (size_t)Wmax * nmax))) return rc;
  ctx->ws_cap[r] = (long long)Wmax * nmax;
  if ((rc = dalloc(ctx, H.mps_allocs, &W.T2, (size_t)Wmax * nmax))) return rc;
  if ((rc = dalloc(ctx, H.mps_allocs, &W.bond, (size_t)Dmax * Dmax))) return rc;
  if ((rc = dalloc(ctx, H.mps_allocs, &W.bond2, (size_t)Dmax * Dmax))) return rc;
  if ((rc = dalloc(ctx, H.mps_allocs, &W.scratch, nmax))) return rc;
  if ((rc = dalloc(ctx, H.mps_allocs, &W.part, (size_t)3 * TDVP_MAX_VEC_BLOCKS * (TDVP_KMAX_HARD + 2)))) return rc;
  if ((rc = dalloc(ctx, H.mps_allocs, &W.qpart, (size_t)3 * 148 * (Dmax + 4)))) return rc;
  if ((rc = dalloc(ctx, H.mps_allocs, &W.qhp, Dmax))) return rc;
  if ((rc = dalloc(ctx, H.mps_allocs, &W.colsq, mmax))) return rc;
  // rank-deficient tail of the QR: row backup, two coefficient tables, residual norms
  // ([n][blocks] doubles, blocks <= 148)
  if ((rc = dalloc(ctx, H.mps_allocs, &W.qtail, (size_t)(nmax + 2 * Dmax * Dmax + Dmax * 74 + 16)))) return rc;
  if ((rc = dalloc(ctx, H.mps_allocs, &W.obs, ctx->n_el + 4))) return rc;
  if ((rc = dalloc(ctx, H.mps_allocs, &W.ks, 1))) return rc;
  {
    long long bl = 1, br = 1, bx = 1, bt2 = 1, bt1 = 1, be1 = 1, be2 = 1;
    for (int i = 0; i < N; ++i) {
      const long long Dl = bd[i], Dr = bd[i + 1], d = ctx->d[i], Wl = ctx->Wb[i], Wr = ctx->Wb[i + 1];
      bl = std::max(bl, tc_pack_bytes(128, Wl * Dl, Dl));
      br = std::max(br, tc_pack_bytes(64, Dr, Wr * Dr));
      bx = std::max(bx, std::max(tc_pack_bytes(64, d * Dr, Dl), tc_pack_bytes(64, Dr, Dr)));
      bt2 = std::max(bt2, std::max(tc_pack_bytes(128, Dl * d, Wr * Dr), tc_pack_bytes(128, Dr, Wr * Dr)));
      bt1 = std::max(bt1, std::max(Wl * Dl * d * Dr, Dl * d * Wr * Dr));
      be1 = std::max(be1, std::max(tc_pack_bytes(128, Dr, Dl * d),
                                   std::max(tc_pack_bytes(128, Dl * d, Dr), tc_pack_bytes(128, Dl, d * Dr))));
      be2 = std::max(be2, std::max(tc_pack_bytes(64, Wr * Dr, Dl * d),
                                   std::max(tc_pack_bytes(64, Wr * Dr, Dr), tc_pack_bytes(64, Wl * Dl, d * Dr))));
    }
    if ((rc = dalloc(ctx, H.mps_allocs, &W.tc_e1, (size_t)be1))) return rc;
    if ((rc = dalloc(ctx, H.mps_allocs, &W.tc_e2, (size_t)be2))) return rc;
    if ((rc = dalloc(ctx, H.mps_allocs, &W.tc_l, (size_t)bl))) return rc;
    if ((rc = dalloc(ctx, H.mps_allocs, &W.tc_r, (size_t)br))) return rc;
    if ((rc = dalloc(ctx, H.mps_allocs, &W.tc_x, (size_t)bx))) return rc;
    if ((rc = dalloc(ctx, H.mps_allocs, &W.tc_t2, (size_t)bt2))) return rc;
    if ((rc = dalloc(ctx, H.mps_allocs, &W.tc_t1, (size_t)(2 * bt1)))) return rc;
    W.tc_t1_plane = bt1;
  }
  if ((rc = dalloc(ctx, H.mps_allocs, &W.bar, 2 + 16))) return rc;   // root, generation, group counters
  if ((rc = dalloc(ctx, H.mps_allocs, &W.kprev, 2 * N))) return rc;
  if ((rc = dalloc(ctx, H.mps_allocs, &W.tri_count, 1))) return rc;
  if ((rc = dalloc(ctx, H.mps_allocs, &W.lzc, 2))) return rc;   // last-block counter, fused-iteration barrier
  CK(cudaMemsetAsync(W.lzc, 0, 2 * sizeof(unsigned), ctx->st));
  W.err = ctx->d_err + r;
  // boundary environments are the scalar 1
  const zc one = zmake(1.0, 0.0);
  CK(cudaMemcpyAsync(ctx->h_sites[(size_t)r * N].Lenv, &one, sizeof(zc), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->h_sites[(size_t)r * N + N - 1].Renv, &one, sizeof(zc), cudaMemcpyHostToDevice, ctx->st));
  return upload_tables(ctx, r);
}

int build_right_envs(tdvp_ctx* ctx, const Views& v) {
  for (int i = ctx->N - 1; i >= 1; --i) {
    int rc = env_right(ctx, v, i);
    if (rc) return rc;
  }
  return TDVP_OK;
}

bool all_ready(tdvp_ctx* ctx) {
  if (ctx->N == 0) return false;
  for (auto& h : ctx->rh) if (!h.mps) return false;
  return true;
}

// One TDVP-PS step of every realisation (Eq. ps_trotter): left-to-right half sweep with tau/2,
// the last site with tau, right-to-left half sweep with tau/2.
int enqueue_step(tdvp_ctx* ctx, const Views& v, double tau, double tol, int P, int* nc) {
  const int N = ctx->N;
  int rc;
  ctx->l_site = ctx->r_site = -1;
  if (N == 1) return expm(ctx, v, 0, 0, 1, 1, -tau, tol, nc, P);
  for (int i = 0; i < N - 1; ++i) {
    if ((rc = expm(ctx, v, 0, i, i == 0 ? 1 : 0, 1, -0.5 * tau, tol, nc, P))) return rc;
    if ((rc = gauge_qr(ctx, v, i, 0))) return rc;
    if ((rc = env_left(ctx, v, i, P))) return rc;
    if ((rc = expm(ctx, v, 1, i, 2, 2, 0.5 * tau, tol, nc, P))) return rc;
    const Dims m = maxdims(ctx, i + 1, v);
    PhaseScope ps(ctx, TDVP_PH_MATMUL_QR);
    if ((rc = g_op(ctx, v, OP_ABS_L, i, m.Dl, ctx->d[i + 1] * m.Dr, 1))) return rc;
  }
  if ((rc = expm(ctx, v, 0, N - 1, 0, 1, -tau, tol, nc, P))) return rc;
  for (int i = N - 1; i >= 1; --i) {
    if ((rc = gauge_qr(ctx, v, i, 1))) return rc;
    if ((rc = env_right(ctx, v, i, P))) return rc;
    if ((rc = expm(ctx, v, 1, i - 1, 2, 2, 0.5 * tau, tol, nc, P))) return rc;
    const Dims m = maxdims(ctx, i - 1, v);
    {
      PhaseScope ps(ctx, TDVP_PH_MATMUL_QR);
      if ((rc = g_op(ctx, v, OP_ABS_R, i, m.Dl * ctx->d[i - 1], m.Dr, 1))) return rc;
    }
    if ((rc = expm(ctx, v, 0, i - 1, 0, 1, -0.5 * tau, tol, nc, P))) return rc;
  }
  return TDVP_OK;
}

// n_steps replays of one captured step.  The graph is captured once per configuration (dt,
// tolerance, precision, Krylov mode and options) and kept until a state or option change.
int graph_steps(tdvp_ctx* ctx, const Views& v, double tau, double tol, int P, int n_steps) {
  const std::vector<double> key = {tau, tol, (double)P, (double)ctx->krylov_mode, (double)ctx->check_every,
                                   (double)ctx->mlp_ready, (double)ctx->logging, (double)ctx->log_cap};
  if (!ctx->gexec || ctx->gkey != key) {
    graph_reset(ctx);
    if (!ctx->body_st) CK(cudaStreamCreateWithFlags(&ctx->body_st, cudaStreamNonBlocking));
    const int need = 4 * ctx->N + 8;
    if (ctx->loop_cap < need) {
      cudaFree(ctx->d_loop_iters);
      ctx->d_loop_iters = nullptr;
      ctx->loop_cap = 0;
      CK(cudaMalloc(&ctx->d_loop_iters, sizeof(unsigned) * need));
      ctx->loop_cap = need;
    }
    CK(cudaMemsetAsync(ctx->d_loop_iters, 0, sizeof(unsigned) * ctx->loop_cap, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    ctx->loop_n = 0;
    ctx->loop_body_launches.clear();
    // captured on a private stream (the caller's may be the legacy default stream, which cannot
    // be captured); the graph is then launched on the caller's stream
    if (!ctx->cap_st) CK(cudaStreamCreateWithFlags(&ctx->cap_st, cudaStreamNonBlocking));
    const long long before = ctx->stats.kernel_launches;
    const cudaStream_t user_st = ctx->st;
    ctx->st = ctx->cap_st;
    cudaError_t e = cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) { ctx->st = user_st; return fail(ctx, TDVP_ERR_CUDA, cudaGetErrorString(e)); }
    ctx->capturing = true;
    int nc = 0;
    int rc = enqueue_step(ctx, v, tau, tol, P, &nc);
    ctx->capturing = false;
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(ctx->st, &g);
    ctx->st = user_st;
    ctx->graph_outer_launches = ctx->stats.kernel_launches - before;
    ctx->stats.kernel_launches = before;
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return fail(ctx, TDVP_ERR_CUDA, cudaGetErrorString(e));
    ctx->graph = g;
    CK(cudaGraphInstantiate(&ctx->gexec, g, 0));
    ctx->gkey = key;
  }
  // device counters of the Krylov solves start from zero
  for (int r = v.r0; r < v.r0 + v.R; ++r)
    CK(cudaMemsetAsync(&ctx->h_work[r].ks->dim_sum, 0, sizeof(long long) + 4 * sizeof(int), ctx->st));
  for (int s = 0; s < n_steps; ++s) CK(cudaGraphLaunch(ctx->gexec, ctx->st));
  // launches and Krylov statistics from the device counters
  std::vector<unsigned> iters(ctx->loop_n);
  if (ctx->loop_n) {
    CK(cudaMemcpyAsync(iters.data(), ctx->d_loop_iters, sizeof(unsigned) * ctx->loop_n, cudaMemcpyDeviceToHost,
                       ctx->st));
    CK(cudaMemsetAsync(ctx->d_loop_iters, 0, sizeof(unsigned) * ctx->loop_n, ctx->st));
  }
  struct { long long dim_sum; int dim_max, solves, nc_count, pad; } kc;
  long long launches = ctx->graph_outer_launches * n_steps;
  for (int q = 0; q < ctx->loop_n; ++q) launches += (long long)iters[q] * ctx->loop_body_launches[q];
  for (int r = v.r0; r < v.r0 + v.R; ++r) {
    CK(cudaMemcpyAsync(&kc, &ctx->h_work[r].ks->dim_sum, sizeof(kc), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    ctx->stats.krylov_dim_sum += kc.dim_sum;
    ctx->stats.krylov_dim_max = std::max(ctx->stats.krylov_dim_max, kc.dim_max);
    ctx->stats.krylov_solves += kc.solves;
    ctx->stats.not_converged += kc.nc_count;
    if (kc.nc_count) ctx->graph_nc = 1;
  }
  CK(cudaStreamSynchronize(ctx->st));
  ctx->stats.kernel_launches += launches;
  ctx->stats.host_syncs += 1;
  ctx->l_site = ctx->r_site = -1;
  return TDVP_OK;
}

}  // namespace

extern "C" {

int tdvp_init_mps(tdvp_ctx* ctx, int r, int D, int exciton_site) {
  if (!ctx) return TDVP_ERR_INVALID_ARG;
  graph_reset(ctx);
  if (r < 0 || r >= ctx->R || D < 1 || D > 256) return fail(ctx, TDVP_ERR_INVALID_ARG, "init_mps: bad r or D");
  if (!ctx->rh[r].mpo) return fail(ctx, TDVP_ERR_STATE, "init_mps: build_mpo first");
  if (exciton_site < 0 || exciton_site >= ctx->n_el) return fail(ctx, TDVP_ERR_INVALID_ARG, "init_mps: bad exciton site");
  CK(cudaSetDevice(ctx->dev));
  const int N = ctx->N;
  std::vector<int> bd(N + 1, 1);
  for (int b = 1; b < N; ++b) {
    double left = 1, right = 1;
    for (int i = 0; i < b; ++i) left = std::min(left * ctx->d[i], 1e12);
    for (int i = b; i < N; ++i) right = std::min(right * ctx->d[i], 1e12);
    bd[b] = (int)std::min<double>(D, std::min(left, right));
  }
  int rc;
  if ((rc = alloc_realisation(ctx, r, bd))) return rc;
  // right-canonical product state: row 0 = occupied path, rows j>=1 = successive unit vectors,
  // positions (s, r) ordered by r first, then s
  for (int i = 0; i < N; ++i) {
    const int Dl = bd[i], d = ctx->d[i], Dr = bd[i + 1];
    const int occ = (ctx->is_el[i] && ctx->label[i] == exciton_site) ? 1 : 0;
    std::vector<zc> A((size_t)Dl * d * Dr, zmake(0, 0));
    A[((size_t)0 * d + occ) * Dr + 0] = zmake(1, 0);
    int j = 1;
    for (int rr = 0; rr < Dr && j < Dl; ++rr)
      for (int s = 0; s < d && j < Dl; ++s) {
        if (s == occ && rr == 0) continue;
        A[((size_t)j * d + s) * Dr + rr] = zmake(1, 0);
        ++j;
      }
    CK(cudaMemcpyAsync(ctx->h_sites[(size_t)r * N + i].A, A.data(), A.size() * sizeof(zc), cudaMemcpyHostToDevice,
                       ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
  }
  ctx->l_site = ctx->r_site = -1;
  if ((rc = build_right_envs(ctx, one_view(ctx, r)))) return rc;
  CK(cudaStreamSynchronize(ctx->st));
  ctx->rh[r].mps = true;
  return check_device_errors(ctx);
}

int tdvp_init_mps_tensors(tdvp_ctx* ctx, int r, const int* bond_dims, const double* re_im) {
  if (!ctx) return TDVP_ERR_INVALID_ARG;
  graph_reset(ctx);
  if (r < 0 || r >= ctx->R || !bond_dims || !re_im) return fail(ctx, TDVP_ERR_INVALID_ARG, "init_mps_tensors: bad args");
  if (!ctx->rh[r].mpo) return fail(ctx, TDVP_ERR_STATE, "init_mps_tensors: build_mpo first");
  CK(cudaSetDevice(ctx->dev));
  const int N = ctx->N;
  std::vector<int> bd(bond_dims, bond_dims + N + 1);
  if (bd[0] != 1 || bd[N] != 1) return fail(ctx, TDVP_ERR_INVALID_ARG, "init_mps_tensors: open ends must be 1");
  for (int i = 0; i < N; ++i) {
    if (bd[i] < 1 || bd[i] > 256) return fail(ctx, TDVP_ERR_INVALID_ARG, "init_mps_tensors: bond dim out of range");
    if (i > 0 && bd[i] > ctx->d[i] * bd[i + 1]) return fail(ctx, TDVP_ERR_INVALID_ARG, "init_mps_tensors: Dl > d*Dr");
    if (bd[i + 1] > ctx->d[i] * bd[i]) return fail(ctx, TDVP_ERR_INVALID_ARG, "init_mps_tensors: Dr > Dl*d");
  }
  int rc;
  if ((rc = alloc_realisation(ctx, r, bd))) return rc;
  size_t off = 0;
  for (int i = 0; i < N; ++i) {
    const size_t n = (size_t)bd[i] * ctx->d[i] * bd[i + 1];
    CK(cudaMemcpyAsync(ctx->h_sites[(size_t)r * N + i].A, re_im + 2 * off, n * sizeof(zc), cudaMemcpyHostToDevice,
                       ctx->st));
    off += n;
  }
  const Views v = one_view(ctx, r);
  // right-canonicalise: C_i = D_i R_i from the last site, D_i absorbed into site i-1, which is
  // then normalised (x = C/||C||, C <- x): the norm of a generic product of site tensors grows or
  // shrinks geometrically with the chain length, and only the normalised state is wanted
  for (int i = N - 1; i >= 1; --i) {
    if ((rc = gauge_qr(ctx, v, i, 1))) return rc;
    const Dims m = maxdims(ctx, i - 1, v);
    if ((rc = g_op(ctx, v, OP_ABS_R, i, m.Dl * ctx->d[i - 1], m.Dr, 1))) return rc;
    LAUNCH(launch_copy_vec(1, i - 1, v.sd, v.wk, v.R, N, m.Dl * ctx->d[i - 1] * m.Dr, ctx->st));
    LzArgs a{};
    a.sd = v.sd; a.wk = v.wk; a.R = 1; a.N_sites = N; a.site = i - 1; a.kind = 0; a.src = 1; a.dst = 1;
    a.kmax = ctx->kmax; a.bcap = TDVP_MAX_VEC_BLOCKS; a.pack_pm = -1;
    a.nblk = nblk_for((long long)m.Dl * ctx->d[i - 1] * m.Dr, a.bcap); a.flags = v.flags;
    LAUNCH(launch_lz_start(a, ctx->st));
    ctx->stats.kernel_launches++;
    LAUNCH(launch_copy_vec(1, i - 1, v.sd, v.wk, 1, N, m.Dl * ctx->d[i - 1] * m.Dr, ctx->st));
  }
  if (N == 1) {
    LzArgs a{};
    const Dims m = maxdims(ctx, 0, v);
    a.sd = v.sd; a.wk = v.wk; a.R = 1; a.N_sites = N; a.site = 0; a.kind = 0; a.src = 1; a.dst = 1;
    a.kmax = ctx->kmax; a.bcap = TDVP_MAX_VEC_BLOCKS; a.pack_pm = -1;
    a.nblk = nblk_for((long long)m.Dl * ctx->d[0] * m.Dr, a.bcap); a.flags = v.flags;
    LAUNCH(launch_lz_start(a, ctx->st));
    ctx->stats.kernel_launches++;
    LAUNCH(launch_copy_vec(1, 0, v.sd, v.wk, 1, N, m.Dl * ctx->d[0] * m.Dr, ctx->st));
  }
  ctx->l_site = ctx->r_site = -1;
  if ((rc = build_right_envs(ctx, v))) return rc;
  CK(cudaStreamSynchronize(ctx->st));
  ctx->rh[r].mps = true;
  return check_device_errors(ctx);
}

int tdvp_ps_step(tdvp_ctx* ctx, double dt_fs, int n_steps, int precision, int krylov_mode, double krylov_tol) {
  if (!ctx) return TDVP_ERR_INVALID_ARG;
  if (n_steps < 0 || !(krylov_tol >= 0) || !std::isfinite(dt_fs)) return fail(ctx, TDVP_ERR_INVALID_ARG, "ps_step: bad args");
  if (precision < TDVP_PREC_FP64 || precision > TDVP_PREC_LAST)
    return fail(ctx, TDVP_ERR_INVALID_ARG, "ps_step: unsupported precision");
  if (krylov_mode != TDVP_KRYLOV_ADAPTIVE && krylov_mode != TDVP_KRYLOV_LEARNED)
    return fail(ctx, TDVP_ERR_INVALID_ARG, "ps_step: unsupported krylov mode");
  if (krylov_mode == TDVP_KRYLOV_LEARNED && !ctx->mlp_ready)
    return fail(ctx, TDVP_ERR_STATE, "ps_step: the learned controller has no weights");
  ctx->krylov_mode = krylov_mode;
  if (!all_ready(ctx)) return fail(ctx, TDVP_ERR_STATE, "ps_step: every realisation needs build_mpo and init");
  CK(cudaSetDevice(ctx->dev));
  const Views v = all_views(ctx);
  const int N = ctx->N;
  const double tau = dt_fs * kPhasePerCmFs;
  int rc, nc = 0;
  const int P = precision;
  if (ctx->graph_on && !ctx->prof && n_steps > 0) {
    if ((rc = graph_steps(ctx, v, tau, krylov_tol, P, n_steps))) return rc;
  } else {
    for (int step = 0; step < n_steps; ++step) {
      if ((rc = enqueue_step(ctx, v, tau, krylov_tol, P, &nc))) return rc;
    }
  }
  ctx->stats.steps += n_steps;
  ctx->stats.site_updates += (long long)(2 * N - 1) * ctx->R * n_steps;
  if ((rc = check_device_errors(ctx))) return rc;
  if ((rc = collect_tri_counts(ctx))) return rc;
  if (ctx->prof && (rc = prof_collect(ctx))) return rc;
  if (nc || ctx->graph_nc) {
    ctx->graph_nc = 0;
    return fail(ctx, TDVP_ERR_KRYLOV_NOT_CONVERGED, "some Lanczos solve stopped at kmax above the tolerance");
  }
  return TDVP_OK;
}

int tdvp_observables(tdvp_ctx* ctx, int r, double* pops, double* energy, double* norm) {
  if (!ctx) return TDVP_ERR_INVALID_ARG;
  if (r < 0 || r >= ctx->R) return fail(ctx, TDVP_ERR_INVALID_ARG, "observables: bad r");
  if (!ctx->rh[r].mps) return fail(ctx, TDVP_ERR_STATE, "observables: not initialised");
  CK(cudaSetDevice(ctx->dev));
  const Views v = one_view(ctx, r);
  const int N = ctx->N, M = ctx->n_el;
  int rc;
  LAUNCH(launch_set_identity_bond2(v.wk, 1, 1, ctx->st));
  for (int i = 0; i < N; ++i) {
    const Dims m = maxdims(ctx, i, v);
    if ((rc = g_op(ctx, v, OP_TR1, i, m.Dl, ctx->d[i] * m.Dr, 1))) return rc;
    if (ctx->is_el[i]) LAUNCH(launch_obs_local(i, ctx->label[i], v.sd, v.wk, 1, N, ctx->st));
    if ((rc = g_op(ctx, v, OP_TR3, i, m.Dr, m.Dr, 1))) return rc;
  }
  LAUNCH(launch_obs_norm(N - 1, M, v.wk, 1, ctx->st));
  // energy: <C|H[0]|C>/<C|C> at the centre (site 0)
  LAUNCH(launch_reset_ks(v.wk, 1, ctx->st));
  if ((rc = matvec_site(ctx, v, 0, OP_HX1))) return rc;
  LAUNCH(launch_obs_energy(M + 1, v.sd, v.wk, 1, N, ctx->st));
  double* h = ctx->h_obs + (size_t)r * (M + 4);
  CK(cudaMemcpyAsync(h, ctx->h_work[r].obs, sizeof(double) * (M + 3), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  const double nn = h[M];
  if (pops) for (int m = 0; m < M; ++m) pops[m] = h[m] / nn;
  if (norm) *norm = std::sqrt(std::max(nn, 0.0));
  if (energy) *energy = h[M + 1] / h[M + 2];
  return check_device_errors(ctx);
}

int tdvp_chain_info(tdvp_ctx* ctx, int r, int* n_sites, int* phys_dims, int* bond_dims, int* mpo_dims) {
  if (!ctx || r < 0 || r >= ctx->R) return TDVP_ERR_INVALID_ARG;
  if (ctx->N == 0) return fail(ctx, TDVP_ERR_STATE, "chain_info: build_mpo first");
  if (n_sites) *n_sites = ctx->N;
  if (phys_dims) std::copy(ctx->d.begin(), ctx->d.end(), phys_dims);
  if (mpo_dims) std::copy(ctx->Wb.begin(), ctx->Wb.end(), mpo_dims);
  if (bond_dims) {
    if (!ctx->rh[r].mps) return fail(ctx, TDVP_ERR_STATE, "chain_info: not initialised");
    std::copy(ctx->rh[r].bd.begin(), ctx->rh[r].bd.end(), bond_dims);
  }
  return TDVP_OK;
}

int tdvp_get_site(tdvp_ctx* ctx, int r, int i, double* re_im) {
  if (!ctx || r < 0 || r >= ctx->R || !re_im) return TDVP_ERR_INVALID_ARG;
  if (!ctx->rh[r].mps || i < 0 || i >= ctx->N) return fail(ctx, TDVP_ERR_INVALID_ARG, "get_site: bad site");
  CK(cudaSetDevice(ctx->dev));
  const SiteDev& S = ctx->h_sites[(size_t)r * ctx->N + i];
  CK(cudaMemcpyAsync(re_im, S.A, sizeof(zc) * (size_t)S.Dl * S.d * S.Dr, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return TDVP_OK;
}

int tdvp_move_center(tdvp_ctx* ctx, int r, int site) {
  if (!ctx || r < 0 || r >= ctx->R) return TDVP_ERR_INVALID_ARG;
  if (!ctx->rh[r].mps || site < 0 || site >= ctx->N) return fail(ctx, TDVP_ERR_INVALID_ARG, "move_center: bad site");
  CK(cudaSetDevice(ctx->dev));
  const Views v = one_view(ctx, r);
  int rc;
  for (int i = 0; i < site; ++i) {
    if ((rc = gauge_qr(ctx, v, i, 0))) return rc;
    if ((rc = env_left(ctx, v, i))) return rc;
    const Dims m = maxdims(ctx, i + 1, v);
    PhaseScope ps(ctx, TDVP_PH_MATMUL_QR);
    if ((rc = g_op(ctx, v, OP_ABS_L, i, m.Dl, ctx->d[i + 1] * m.Dr, 1))) return rc;
    LAUNCH(launch_copy_vec(1, i + 1, v.sd, v.wk, 1, ctx->N, m.Dl * ctx->d[i + 1] * m.Dr, ctx->st));
  }
  CK(cudaStreamSynchronize(ctx->st));
  return check_device_errors(ctx);
}

int tdvp_center_to_zero(tdvp_ctx* ctx, int r) {
  if (!ctx || r < 0 || r >= ctx->R) return TDVP_ERR_INVALID_ARG;
  if (!ctx->rh[r].mps) return fail(ctx, TDVP_ERR_STATE, "center_to_zero: not initialised");
  CK(cudaSetDevice(ctx->dev));
  const Views v = one_view(ctx, r);
  int rc;
  for (int i = ctx->N - 1; i >= 1; --i) {
    if ((rc = gauge_qr(ctx, v, i, 1))) return rc;
    if ((rc = env_right(ctx, v, i))) return rc;
    const Dims m = maxdims(ctx, i - 1, v);
    if ((rc = g_op(ctx, v, OP_ABS_R, i, m.Dl * ctx->d[i - 1], m.Dr, 1))) return rc;
    LAUNCH(launch_copy_vec(1, i - 1, v.sd, v.wk, 1, ctx->N, m.Dl * ctx->d[i - 1] * m.Dr, ctx->st));
  }
  CK(cudaStreamSynchronize(ctx->st));
  return check_device_errors(ctx);
}

int tdvp_apply_heff(tdvp_ctx* ctx, int r, int i, int precision, const double* x, double* y) {
  if (!ctx || r < 0 || r >= ctx->R || !x || !y) return TDVP_ERR_INVALID_ARG;
  if (!ctx->rh[r].mps || i < 0 || i >= ctx->N) return fail(ctx, TDVP_ERR_INVALID_ARG, "apply_heff: bad site");
  if (precision < TDVP_PREC_FP64 || precision > TDVP_PREC_LAST) return fail(ctx, TDVP_ERR_INVALID_ARG, "apply_heff: precision");
  CK(cudaSetDevice(ctx->dev));
  const Views v = one_view(ctx, r);
  const SiteDev& S = ctx->h_sites[(size_t)r * ctx->N + i];
  const size_t n = (size_t)S.Dl * S.d * S.Dr;
  CK(cudaMemcpyAsync(ctx->h_work[r].x, x, n * sizeof(zc), cudaMemcpyHostToDevice, ctx->st));
  LAUNCH(launch_reset_ks(v.wk, 1, ctx->st));
  int rc;
  if (precision == TDVP_PREC_FP64) {
    if ((rc = matvec_site(ctx, v, i, OP_MV1))) return rc;
  } else {
    ctx->l_site = ctx->r_site = -1;
    if ((rc = prepare_tc_solve(ctx, v, 0, i, tc_mode(precision)))) return rc;
    if ((rc = matvec_site_tc(ctx, v, i, tc_mode(precision)))) return rc;
  }
  CK(cudaMemcpyAsync(y, ctx->h_work[r].w, n * sizeof(zc), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return check_device_errors(ctx);
}

int tdvp_apply_h0(tdvp_ctx* ctx, int r, int i, int precision, const double* x, double* y) {
  if (!ctx || r < 0 || r >= ctx->R || !x || !y) return TDVP_ERR_INVALID_ARG;
  if (!ctx->rh[r].mps || i < 0 || i >= ctx->N - 1) return fail(ctx, TDVP_ERR_INVALID_ARG, "apply_h0: bad bond");
  if (precision < TDVP_PREC_FP64 || precision > TDVP_PREC_LAST) return fail(ctx, TDVP_ERR_INVALID_ARG, "apply_h0: precision");
  CK(cudaSetDevice(ctx->dev));
  const Views v = one_view(ctx, r);
  const int Db = ctx->rh[r].bd[i + 1];
  const size_t n = (size_t)Db * Db;
  CK(cudaMemcpyAsync(ctx->h_work[r].x, x, n * sizeof(zc), cudaMemcpyHostToDevice, ctx->st));
  LAUNCH(launch_reset_ks(v.wk, 1, ctx->st));
  int rc;
  if (precision == TDVP_PREC_FP64) {
    if ((rc = matvec_bond(ctx, v, i))) return rc;
  } else {
    ctx->l_site = ctx->r_site = -1;
    if ((rc = prepare_tc_solve(ctx, v, 1, i, tc_mode(precision)))) return rc;
    if ((rc = matvec_bond_tc(ctx, v, i, tc_mode(precision)))) return rc;
  }
  CK(cudaMemcpyAsync(y, ctx->h_work[r].w, n * sizeof(zc), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return check_device_errors(ctx);
}

int tdvp_debug_qr(tdvp_ctx* ctx, int m, int n, const double* C, double* Q, double* Rout) {
  if (!ctx || !C || !Q || !Rout || n < 1 || m < n) return TDVP_ERR_INVALID_ARG;
  if (!ctx->rh[0].mps) return fail(ctx, TDVP_ERR_STATE, "debug_qr: realisation 0 must be initialised");
  CK(cudaSetDevice(ctx->dev));
  // the kernel works on rows: X = C^T (n x m)
  long long nmax = 1, Dmax = 1, mmax = 1;
  const auto& bd = ctx->rh[0].bd;
  for (int i = 0; i < ctx->N; ++i) {
    nmax = std::max(nmax, (long long)bd[i] * ctx->d[i] * bd[i + 1]);
    Dmax = std::max<long long>(Dmax, std::max(bd[i], bd[i + 1]));
    mmax = std::max<long long>(mmax, std::max<long long>((long long)bd[i] * ctx->d[i], (long long)ctx->d[i] * bd[i + 1]));
  }
  if ((long long)m * n > nmax || n > Dmax || m > mmax || n > 256)
    return fail(ctx, TDVP_ERR_INVALID_ARG, "debug_qr: matrix larger than the work buffers");
  std::vector<zc> X((size_t)n * m);
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < n; ++b) X[(size_t)b * m + a] = zmake(C[2 * ((size_t)a * n + b)], C[2 * ((size_t)a * n + b) + 1]);
  const Views v = one_view(ctx, 0);
  CK(cudaMemcpyAsync(ctx->h_work[0].scratch, X.data(), X.size() * sizeof(zc), cudaMemcpyHostToDevice, ctx->st));
  {
    const int rc = run_qr_timed(ctx, TDVP_CAT_OTHER, v, 2, 0, m, n, qr_mode(ctx, 1, m, n), ctx->rank_rtol, n, m);
    if (rc) return rc;
  }
  std::vector<zc> R((size_t)n * n);
  CK(cudaMemcpyAsync(X.data(), ctx->h_work[0].scratch, X.size() * sizeof(zc), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(R.data(), ctx->h_work[0].bond, R.size() * sizeof(zc), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < n; ++b) {
      Q[2 * ((size_t)a * n + b)] = X[(size_t)b * m + a].x;
      Q[2 * ((size_t)a * n + b) + 1] = X[(size_t)b * m + a].y;
    }
  std::memcpy(Rout, R.data(), R.size() * sizeof(zc));
  return check_device_errors(ctx);
}

int tdvp_debug_expm(tdvp_ctx* ctx, int r, int i, double z_re, double z_im, double tol, const double* vin,
                    double* out, int* k_out) {
  if (!ctx || r < 0 || r >= ctx->R || !vin || !out) return TDVP_ERR_INVALID_ARG;
  if (z_re != 0.0) return fail(ctx, TDVP_ERR_INVALID_ARG, "debug_expm: exponent must be purely imaginary");
  if (!ctx->rh[r].mps || i < 0 || i >= ctx->N) return fail(ctx, TDVP_ERR_INVALID_ARG, "debug_expm: bad site");
  CK(cudaSetDevice(ctx->dev));
  const Views v = one_view(ctx, r);
  const SiteDev& S = ctx->h_sites[(size_t)r * ctx->N + i];
  const size_t n = (size_t)S.Dl * S.d * S.Dr;
  CK(cudaMemcpyAsync(ctx->h_work[r].x, vin, n * sizeof(zc), cudaMemcpyHostToDevice, ctx->st));
  int nc = 0, rc;
  const int saved = ctx->khist[2 * i];
  if ((rc = expm(ctx, v, 0, i, 0, 3, z_im, tol, &nc))) return rc;
  if (k_out) *k_out = ctx->h_flags[r] & 0xffff;
  ctx->khist[2 * i] = saved;
  CK(cudaMemcpyAsync(out, ctx->h_work[r].w, n * sizeof(zc), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return TDVP_OK;
}

int tdvp_stats(tdvp_ctx* ctx, tdvp_stats_t* out) {
  if (!ctx || !out) return TDVP_ERR_INVALID_ARG;
  *out = ctx->stats;
  return TDVP_OK;
}

void tdvp_reset_stats(tdvp_ctx* ctx) {
  if (ctx) ctx->stats = tdvp_stats_t{};
}

int tdvp_controller_set_weights(tdvp_ctx* ctx, const float* w, int n) {
  if (!ctx || !w) return TDVP_ERR_INVALID_ARG;
  if (n != MLP_NPARAM) return fail(ctx, TDVP_ERR_INVALID_ARG, "controller: wrong number of weights");
  CK(cudaSetDevice(ctx->dev));
  if (!ctx->d_mlp) {
    CK(cudaMalloc(&ctx->d_mlp, sizeof(float) * MLP_NPARAM));
    CK(cudaMalloc(&ctx->d_mlp_m, sizeof(float) * MLP_NPARAM));
    CK(cudaMalloc(&ctx->d_mlp_v, sizeof(float) * MLP_NPARAM));
  }
  CK(cudaMemcpyAsync(ctx->d_mlp, w, sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemsetAsync(ctx->d_mlp_m, 0, sizeof(float) * MLP_NPARAM, ctx->st));
  CK(cudaMemsetAsync(ctx->d_mlp_v, 0, sizeof(float) * MLP_NPARAM, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  ctx->mlp_ready = 1;
  ctx->mlp_step = 0;
  return TDVP_OK;
}

int tdvp_controller_get_weights(tdvp_ctx* ctx, float* w, int n) {
  if (!ctx || !w) return TDVP_ERR_INVALID_ARG;
  if (n != MLP_NPARAM || !ctx->mlp_ready) return fail(ctx, TDVP_ERR_INVALID_ARG, "controller: no weights");
  CK(cudaMemcpyAsync(w, ctx->d_mlp, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return TDVP_OK;
}

int tdvp_controller_logging(tdvp_ctx* ctx, long long capacity) {
  if (!ctx || capacity < 0) return TDVP_ERR_INVALID_ARG;
  CK(cudaSetDevice(ctx->dev));
  if (capacity == 0) { ctx->logging = 0; return TDVP_OK; }
  if (capacity != ctx->log_cap) {
    cudaFree(ctx->d_log);
    ctx->d_log = nullptr;
    CK(cudaMalloc(&ctx->d_log, sizeof(float) * (MLP_NIN + 1) * capacity));
    if (!ctx->d_log_count) CK(cudaMalloc(&ctx->d_log_count, sizeof(unsigned)));
    ctx->log_cap = capacity;
  }
  CK(cudaMemsetAsync(ctx->d_log_count, 0, sizeof(unsigned), ctx->st));
  ctx->logging = 1;
  return TDVP_OK;
}

long long log_size(tdvp_ctx* ctx) {
  unsigned cnt = 0;
  if (!ctx->d_log_count) return 0;
  if (cudaMemcpyAsync(&cnt, ctx->d_log_count, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->st) != cudaSuccess ||
      cudaStreamSynchronize(ctx->st) != cudaSuccess)
    return -1;
  return std::min<long long>(cnt, ctx->log_cap);
}

int tdvp_controller_log(tdvp_ctx* ctx, float* out, long long max_rows, long long* rows) {
  if (!ctx || !rows) return TDVP_ERR_INVALID_ARG;
  CK(cudaSetDevice(ctx->dev));
  const long long n = log_size(ctx);
  if (n < 0) return fail(ctx, TDVP_ERR_CUDA, "controller: reading the log size failed");
  *rows = n;
  if (out && max_rows > 0 && n > 0) {
    CK(cudaMemcpyAsync(out, ctx->d_log, sizeof(float) * (MLP_NIN + 1) * std::min(n, max_rows), cudaMemcpyDeviceToHost,
                       ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
  }
  return TDVP_OK;
}

// loss and gradient of controller head `head` on B rows of `data` (device); `partial` holds
// mlp_partial_floats(B) floats; *loss (host, may be null) synchronises to read the loss
int controller_grad(tdvp_ctx* ctx, int head, const float* d_data, long long idx0, int B, float* partial, float* d_grad,
                    float* loss_acc, float* loss) {
  cudaError_t e = launch_mlp_grad(head, d_data, idx0, B, ctx->d_mlp, partial, d_grad, loss_acc, ctx->st);
  if (e == cudaSuccess && loss) {
    e = cudaMemcpyAsync(loss, d_grad + MLP_NPARAM, sizeof(float), cudaMemcpyDeviceToHost, ctx->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
  }
  if (e != cudaSuccess) return fail(ctx, TDVP_ERR_CUDA, std::string("controller gradient: ") + cudaGetErrorString(e));
  return TDVP_OK;
}

int tdvp_controller_loss_grad(tdvp_ctx* ctx, int head, const float* X, const float* t, int B, float* loss,
                              float* grad) {
  if (!ctx || !X || !t || B < 1 || !grad || !loss || (head != 0 && head != 1)) return TDVP_ERR_INVALID_ARG;
  if (!ctx->mlp_ready) return fail(ctx, TDVP_ERR_STATE, "controller: set weights first");
  CK(cudaSetDevice(ctx->dev));
  std::vector<float> rows((size_t)B * (MLP_NIN + 1));
  for (int b = 0; b < B; ++b) {
    for (int q = 0; q < MLP_NIN; ++q) rows[(size_t)b * (MLP_NIN + 1) + q] = X[(size_t)b * MLP_NIN + q];
    rows[(size_t)b * (MLP_NIN + 1) + MLP_NIN] = t[b];
  }
  float *d_rows = nullptr, *d_grad = nullptr, *d_part = nullptr;
  const cudaError_t e1 = cudaMalloc(&d_rows, sizeof(float) * rows.size());
  const cudaError_t e2 = cudaMalloc(&d_grad, sizeof(float) * (MLP_NPARAM + 1));
  const cudaError_t e3 = cudaMalloc(&d_part, sizeof(float) * mlp_partial_floats(B));
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
    cudaFree(d_rows);
    cudaFree(d_grad);
    cudaFree(d_part);
    return fail(ctx, TDVP_ERR_OOM, "controller: cudaMalloc of the gradient buffers failed");
  }
  int rc = TDVP_OK;
  if (cudaMemcpyAsync(d_rows, rows.data(), sizeof(float) * rows.size(), cudaMemcpyHostToDevice, ctx->st) != cudaSuccess)
    rc = fail(ctx, TDVP_ERR_CUDA, "controller: upload failed");
  if (!rc) rc = controller_grad(ctx, head, d_rows, 0, B, d_part, d_grad, nullptr, loss);
  if (!rc && (cudaMemcpyAsync(grad, d_grad, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToHost, ctx->st) != cudaSuccess ||
              cudaStreamSynchronize(ctx->st) != cudaSuccess))
    rc = fail(ctx, TDVP_ERR_CUDA, "controller: download failed");
  cudaFree(d_rows);
  cudaFree(d_grad);
  cudaFree(d_part);
  return rc;
}

// Two stages on the solve log, each `epochs` passes in mini-batches of `batch`: (1) trunk and the
// Krylov-dimension head by mean-squared error, (2) the acceptance head alone by the logistic loss
// (its labels depend on the stage-1 prediction).  Adam moments start from zero in each stage.  The
// mean loss of each stage's last epoch goes to final_loss[0], final_loss[1]; the host reads them
// once at the end.
int tdvp_controller_train(tdvp_ctx* ctx, int epochs, int batch, float lr, float* final_loss) {
  if (!ctx || epochs < 1 || batch < 1 || !(lr > 0)) return TDVP_ERR_INVALID_ARG;
  if (!ctx->mlp_ready) return fail(ctx, TDVP_ERR_STATE, "controller: set (initial) weights first");
  CK(cudaSetDevice(ctx->dev));
  const long long n = log_size(ctx);
  if (n < 1) return fail(ctx, TDVP_ERR_STATE, "controller: the solve log is empty");
  const int Bmax = (int)std::min<long long>(batch, n);
  float *d_grad = nullptr, *d_part = nullptr, *d_loss = nullptr;
  const cudaError_t e1 = cudaMalloc(&d_grad, sizeof(float) * (MLP_NPARAM + 1));
  const cudaError_t e2 = cudaMalloc(&d_part, sizeof(float) * mlp_partial_floats(Bmax));
  const cudaError_t e3 = cudaMalloc(&d_loss, sizeof(float) * 2);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
    cudaFree(d_grad);
    cudaFree(d_part);
    cudaFree(d_loss);
    return fail(ctx, TDVP_ERR_OOM, "controller: cudaMalloc of the training buffers failed");
  }
  int rc = TDVP_OK;
  long long nbatches = 0;
  for (int stage = 0; stage < 2 && !rc; ++stage) {
    const int p0 = stage == 0 ? 0 : MLP_NPARAM_K, p1 = stage == 0 ? MLP_NPARAM_K : MLP_NPARAM;
    if (cudaMemsetAsync(ctx->d_mlp_m, 0, sizeof(float) * MLP_NPARAM, ctx->st) != cudaSuccess ||
        cudaMemsetAsync(ctx->d_mlp_v, 0, sizeof(float) * MLP_NPARAM, ctx->st) != cudaSuccess) {
      rc = fail(ctx, TDVP_ERR_CUDA, "controller: clearing the Adam moments failed");
      break;
    }
    int t = 0;
    for (int ep = 0; ep < epochs && !rc; ++ep) {
      if (cudaMemsetAsync(d_loss + stage, 0, sizeof(float), ctx->st) != cudaSuccess) {
        rc = fail(ctx, TDVP_ERR_CUDA, "controller: loss reset failed");
        break;
      }
      nbatches = 0;
      for (long long i0 = 0; i0 < n && !rc; i0 += batch) {
        const int B = (int)std::min<long long>(batch, n - i0);
        rc = controller_grad(ctx, stage, ctx->d_log, i0, B, d_part, d_grad, d_loss + stage, nullptr);
        if (rc) break;
        ++t;
        if (launch_mlp_adam(ctx->d_mlp, d_grad, ctx->d_mlp_m, ctx->d_mlp_v, lr, t, p0, p1, ctx->st) != cudaSuccess)
          rc = fail(ctx, TDVP_ERR_CUDA, "controller: Adam update failed");
        ++nbatches;
      }
    }
    ctx->mlp_step += t;
  }
  float h[2] = {0.f, 0.f};
  if (!rc && (cudaMemcpyAsync(h, d_loss, sizeof(float) * 2, cudaMemcpyDeviceToHost, ctx->st) != cudaSuccess ||
              cudaStreamSynchronize(ctx->st) != cudaSuccess))
    rc = fail(ctx, TDVP_ERR_CUDA, "controller: reading the loss failed");
  cudaFree(d_grad);
  cudaFree(d_part);
  cudaFree(d_loss);
  if (final_loss) {
    final_loss[0] = h[0] / (float)std::max(1LL, nbatches);
    final_loss[1] = h[1] / (float)std::max(1LL, nbatches);
  }
  graph_reset(ctx);        // captured steps hold no copy of the weights, but keep the rule simple
  return rc;
}

int tdvp_autotune(tdvp_ctx* ctx) {
  if (!ctx) return TDVP_ERR_INVALID_ARG;
  graph_reset(ctx);
  if (!all_ready(ctx)) return fail(ctx, TDVP_ERR_STATE, "autotune: every realisation needs build_mpo and init");
  CK(cudaSetDevice(ctx->dev));
  const Views v = all_views(ctx);
  std::mt19937_64 rng(12044);
  std::normal_distribution<double> nd(0.0, 1.0);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // every QR launch of the sweep (one per run of consecutive realisations with equal shape), timed
  // in the realisations' QR scratch (the state is not touched) on a random full-rank and a random
  // rank-deficient matrix (rank n/8) of the run's shape: the sweep meets both, and the kernels'
  // row-by-row paths differ in cost
  for (int i = 0; i < ctx->N; ++i) {
    for (int dir : {0, 3}) {
      if ((dir == 0 && i == ctx->N - 1) || (dir == 3 && i == 0)) continue;
      for (const QrRun& run : qr_runs(ctx, v, i, dir == 0 ? 0 : 1)) {
        const int mm = run.m, nn = run.n;
        const auto key = std::make_tuple(run.R, mm, nn);
        if (ctx->qr_tuned.count(key) || nn > 256) continue;
        const Views sv = sub_view(ctx, v, run.r0, run.R);
        // M[kind]: nn x mm row-major; kind 0 full rank, kind 1 rank max(1, nn / 8)
        std::vector<zc> M[2];
        {
          const int rk = std::max(1, nn / 8);
          M[0].resize((size_t)nn * mm);
          for (auto& z : M[0]) z = zmake(nd(rng), nd(rng));
          std::vector<zc> P((size_t)nn * rk), Qm((size_t)rk * mm);
          for (auto& z : P) z = zmake(nd(rng), nd(rng));
          for (auto& z : Qm) z = zmake(nd(rng), nd(rng));
          M[1].assign((size_t)nn * mm, zmake(0, 0));
          for (int a = 0; a < nn; ++a)
            for (int c = 0; c < mm; ++c) {
              zc acc = zmake(0, 0);
              for (int t = 0; t < rk; ++t) acc = zfma(P[(size_t)a * rk + t], Qm[(size_t)t * mm + c], acc);
              M[1][(size_t)a * mm + c] = acc;
            }
        }
        // the cluster kernel reads the left-to-right shape through its transposed view
        std::vector<zc> MT[2];
        for (int kind = 0; kind < 2; ++kind) {
          MT[kind].resize(M[kind].size());
          for (int a = 0; a < nn; ++a)
            for (int c = 0; c < mm; ++c) MT[kind][(size_t)c * nn + a] = M[kind][(size_t)a * mm + c];
        }
        std::vector<int> cands;
        for (int B : {1, 2, 4, 8, 16, 24, 32, 48, 64, 80, 96, 128, 148})
          if (B <= mm && B <= ctx->qr_cap) cands.push_back(B);
        for (int C : {1, 2, 4, 8, 16})
          if (cqr_fits(ctx, C, mm, nn)) cands.push_back(-C);
        int best_mode = qr_mode(ctx, run.R, mm, nn);
        float best = 1e30f;
        for (int mode : cands) {
          const bool trans = mode < 0 && dir == 0;
          const int tdir = dir == 0 ? 4 : 3;
          float total = 0;
          for (int kind = 0; kind < 2; ++kind) {
            const std::vector<zc>& src = trans ? MT[kind] : M[kind];
            float tmin = 1e30f;
            for (int rep = 0; rep < 2; ++rep) {
              for (int q = 0; q < run.R; ++q)
                CK(cudaMemcpyAsync(ctx->h_work[v.r0 + run.r0 + q].scratch, src.data(), src.size() * sizeof(zc),
                                   cudaMemcpyHostToDevice, ctx->st));
              CK(cudaEventRecord(e0, ctx->st));
              const int rc = run_qr(ctx, sv, tdir, i, mm, nn, mode, 1e-13, 0, 0);
              if (rc) return rc;
              CK(cudaEventRecord(e1, ctx->st));
              CK(cudaEventSynchronize(e1));
              float ms = 0;
              CK(cudaEventElapsedTime(&ms, e0, e1));
              tmin = std::min(tmin, ms);
            }
            total += tmin;
          }
          if (total < best) { best = total; best_mode = mode; }
        }
        ctx->qr_tuned[key] = best_mode;
      }
    }
  }
  // the tensor-core GEMMs of the Lanczos matvecs: for every distinct (op, M, N, K) of the chain,
  // time each split-K cluster size on the work buffers (operand contents do not change the time;
  // the outputs are scratch: T1, the packed T of the bond matvec, w) in the TF32x3 mode, and keep
  // the fastest.  The solves are marked unfinished so that the stages do not skip themselves; the
  // next exponential's start resets that mark.
  if (ctx->h_work[0].tc_x) {
    for (int r = 0; r < ctx->R; ++r)
      CK(cudaMemsetAsync(&ctx->h_work[r].ks->done, 0, sizeof(int), ctx->st));
    for (int i = 0; i < ctx->N; ++i) {
      const Dims m = maxdims(ctx, i, v);
      const int d = ctx->d[i], Wl = ctx->Wb[i], Wr = ctx->Wb[i + 1];
      struct Shape { int op, M, N, K; };
      std::vector<Shape> shapes = {{TC_MV1, Wl * m.Dl, d * m.Dr, m.Dl}, {TC_MV3, m.Dl * d, m.Dr, Wr * m.Dr}};
      if (i < ctx->N - 1) {
        shapes.push_back({TC_Z1, Wr * m.Dr, m.Dr, m.Dr});
        shapes.push_back({TC_Z3, m.Dr, m.Dr, Wr * m.Dr});
      }
      for (const Shape& sh : shapes) {
        const auto key = std::make_tuple(sh.op, ctx->R, sh.M, sh.N, sh.K);
        if (ctx->tc_tuned.count(key)) continue;
        int best_S = 0;
        float best = 1e30f;
        for (int S : {1, 2, 4, 8}) {
          if (S > (sh.K + 31) / 32) break;
          float tmin = 1e30f;
          for (int rep = 0; rep < 3; ++rep) {
            CK(cudaEventRecord(e0, ctx->st));
            CK(launch_tc_gemm(sh.op, i, v.sd, v.wk, v.R, ctx->N, sh.M, sh.N, sh.K, TC_PM_SPLIT, ctx->st, S));
            CK(cudaEventRecord(e1, ctx->st));
            CK(cudaEventSynchronize(e1));
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            tmin = std::min(tmin, ms);
          }
          if (tmin < best) { best = tmin; best_S = S; }
        }
        ctx->tc_tuned[key] = best_S;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return check_device_errors(ctx);
}

int tdvp_set_option(tdvp_ctx* ctx, int option, double value) {
  if (!ctx) return TDVP_ERR_INVALID_ARG;
  graph_reset(ctx);
  switch (option) {
    case TDVP_OPT_RANK_RTOL:
      if (!(value > 0.0 && value < 1.0)) return fail(ctx, TDVP_ERR_INVALID_ARG, "rank rtol must be in (0, 1)");
      ctx->rank_rtol = value;
      return TDVP_OK;
    case TDVP_OPT_KRYLOV_CHECK_ALL:
      ctx->check_every = value != 0.0 ? 1 : 0;
      return TDVP_OK;
    case TDVP_OPT_GRAPH:
      ctx->graph_on = value != 0.0 ? 1 : 0;
      return TDVP_OK;
    case TDVP_OPT_PDL:
      g_tdvp_pdl = value != 0.0 ? 1 : 0;
      return TDVP_OK;
    case TDVP_OPT_FUSED_LANCZOS:
      graph_reset(ctx);
      ctx->fused_lz = value != 0.0 ? 1 : 0;
      return TDVP_OK;
    case TDVP_OPT_LANCZOS_CHUNKS: {
      const int c = (int)value;
      if ((double)c != value || c < 1 || c > TDVP_MAX_VEC_BLOCKS)
        return fail(ctx, TDVP_ERR_INVALID_ARG, "Lanczos chunks: an integer in [1, 148]");
      graph_reset(ctx);
      ctx->lz_chunks = c;
      return TDVP_OK;
    }
    case TDVP_OPT_ENV_FP64:
      graph_reset(ctx);
      ctx->env_fp64 = value != 0.0 ? 1 : 0;
      return TDVP_OK;
    case TDVP_OPT_STALL_TEST:
      if (!(value >= 0.0 && value <= 1.0)) return fail(ctx, TDVP_ERR_INVALID_ARG, "stall test: wait limit in [0, 1] s");
      graph_reset(ctx);
      ctx->stall_test = value;
      return TDVP_OK;
    case TDVP_OPT_QR_KERNEL: {
      const int c = (int)value;
      if ((double)c != value || !(c == -2 || c == -1 || c == 0 || c == 1 || c == 2 || c == 4 || c == 8 || c == 16))
        return fail(ctx, TDVP_ERR_INVALID_ARG, "QR kernel option must be -2, -1, 0, 1, 2, 4, 8 or 16");
      if (c > 0 && !ctx->cqr_ok[c]) return fail(ctx, TDVP_ERR_INVALID_ARG, "cluster size not launchable on this device");
      ctx->qr_force = c;
      return TDVP_OK;
    }
  }
  return fail(ctx, TDVP_ERR_INVALID_ARG, "unknown option");
}

int tdvp_set_profiling(tdvp_ctx* ctx, int on) {
  if (!ctx) return TDVP_ERR_INVALID_ARG;
  if (!on && ctx->prof) {
    int rc = prof_collect(ctx);
    if (rc) return rc;
  }
  ctx->prof = on ? 1 : 0;
  return TDVP_OK;
}

}  // extern "C"
