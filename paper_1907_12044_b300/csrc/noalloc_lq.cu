// tdvp_lq_noalloc: the right-to-left gauge shift X = L Q for callers that cannot allocate device
// memory.  Same arithmetic as row_qr_kernel (rows orthogonalised one after another by classical
// Gram-Schmidt with one re-orthogonalisation pass, rank-deficient rows completed from unit
// vectors), but every scratch buffer lives in one file-scope device array, so a call allocates
// nothing.  The caller provides X (input), Q and L (outputs) in device memory.
#include "tdvp_internal.cuh"
#include "../../include/tdvp.h"

#include <mutex>

namespace {

constexpr int NA_NMAX = 256;        // rows (bond dimension) accepted
constexpr int NA_MMAX = 16384;      // columns accepted
constexpr int NA_BMAX = 64;         // blocks per call
constexpr int NA_PS = NA_NMAX + 4;  // stride of one block's partial sums
constexpr int NT = 256;
constexpr int NW = NT / 32;
constexpr unsigned long long NA_WAIT_NS = 1000000000ull;   // a barrier wait gives up after 1 s

constexpr size_t NA_OFF_PART = 0;                                            // 3 x [BMAX][PS] complex
constexpr size_t NA_OFF_COLSQ = NA_OFF_PART + 3ull * NA_BMAX * NA_PS * sizeof(zc);   // [MMAX] double
constexpr size_t NA_OFF_HP = NA_OFF_COLSQ + NA_MMAX * sizeof(double);         // [NMAX] complex
constexpr size_t NA_OFF_WORDS = NA_OFF_HP + NA_NMAX * sizeof(zc);             // barrier count, generation, error
constexpr size_t NA_BYTES = NA_OFF_WORDS + 256;                              // 934,144 bytes

// Scratch shared by every call on a device; it stays resident until the process exits.
static __device__ __align__(256) unsigned char g_lq_scratch[NA_BYTES];

struct NaView {
  zc* part;
  double* colsq;
  zc* hp;
  unsigned* bar;   // [0] arrivals, [1] generation
  int* err;
};

__device__ NaView na_view(unsigned char* base) {
  NaView v;
  v.part = reinterpret_cast<zc*>(base + NA_OFF_PART);
  v.colsq = reinterpret_cast<double*>(base + NA_OFF_COLSQ);
  v.hp = reinterpret_cast<zc*>(base + NA_OFF_HP);
  v.bar = reinterpret_cast<unsigned*>(base + NA_OFF_WORDS);
  v.err = reinterpret_cast<int*>(base + NA_OFF_WORDS + 8);
  return v;
}

__device__ __forceinline__ unsigned long long na_gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier of the cooperative launch (one arrival word and one generation word).  Every wait
// is bounded by wall-clock time (NA_WAIT_NS, %globaltimer): past it the block records
// TDVP_ERR_DEVICE_TIMEOUT and returns false, and so does every block that sees the error word.
__device__ bool na_sync(const NaView& S, int nblocks) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = S.bar + 1;
    volatile int* err = S.err;
    int good = (*err == 0);
    if (good && nblocks > 1) {
      const unsigned g = *gen;
      __threadfence();
      const unsigned arrived = atomicAdd(S.bar, 1u) + 1u;
      if (arrived == (unsigned)nblocks) {
        atomicExch(S.bar, 0u);
        __threadfence();
        atomicAdd(S.bar + 1, 1u);
      } else {
        const unsigned long long t0 = na_gtimer();
        while (*gen == g) {
          if (*err != 0) { good = 0; break; }
          if (na_gtimer() - t0 > NA_WAIT_NS) { atomicExch(S.err, TDVP_ERR_DEVICE_TIMEOUT); good = 0; break; }
          __nanosleep(64);
        }
      }
      __threadfence();
    }
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

__device__ void na_dots(const zc* X, int m, int j, const zc* x, int c0, int c1, zc* out) {
  const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
  for (int t = wid; t < j; t += NW) {
    const zc* q = X + (long long)t * m;
    zc s = zmake(0, 0);
    for (int c = c0 + lane; c < c1; c += 32) s = zcfma(q[c], x[c], s);
    for (int o = 16; o > 0; o >>= 1) {
      s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
    }
    if (lane == 0) out[t] = s;
  }
}

__device__ void na_reduce(const zc* P, int B, int cnt, zc* h) {
  const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
  for (int t = wid; t < cnt; t += NW) {
    zc s = zmake(0, 0);
    for (int b = lane; b < B; b += 32) s = zadd(s, __ldcg(P + (long long)b * NA_PS + t));
    for (int o = 16; o > 0; o >>= 1) {
      s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
    }
    if (lane == 0) h[t] = s;
  }
  __syncthreads();
}

__device__ void na_update(const zc* X, int m, int j, zc* x, int c0, int c1, const zc* h, zc (*buf)[32]) {
  const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
  for (int cb = c0; cb < c1; cb += 32) {
    const int c = cb + lane;
    zc acc = zmake(0, 0);
    if (c < c1)
      for (int t = wid; t < j; t += NW) acc = zfma(h[t], X[(long long)t * m + c], acc);
    buf[wid][lane] = acc;
    __syncthreads();
    if (wid == 0 && c < c1) {
      zc s = buf[0][lane];
      for (int w = 1; w < NW; ++w) s = zadd(s, buf[w][lane]);
      x[c] = zsub(x[c], s);
    }
    __syncthreads();
  }
}

__device__ double na_norm2(const zc* x, int c0, int c1, double* red) {
  double s = 0;
  for (int c = c0 + threadIdx.x; c < c1; c += NT) s += zabs2(x[c]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __syncthreads();
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  double t = 0;
  for (int w = 0; w < NW; ++w) t += red[w];
  return t;
}

__device__ double na_scalar(const zc* P, int B, int slot) {
  const int lane = threadIdx.x % 32;
  double s = 0;
  for (int b = lane; b < B; b += 32) s += __ldcg(P + (long long)b * NA_PS + slot).x;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// X (n x m, in place -> Q) = L Q, L (n x n) lower triangular.  B blocks own column slabs.
__global__ void __launch_bounds__(NT)
lq_noalloc_kernel(zc* X, zc* L, int n, int m, int B, double rtol, unsigned char* scratch) {
  __shared__ zc h1[NA_NMAX];
  __shared__ zc h2[NA_NMAX];
  __shared__ zc buf[NW][32];
  __shared__ double red[NW];
  __shared__ int sel;
  const NaView S = na_view(scratch);
  const int b = blockIdx.x;
  const int c0 = (int)((long long)m * b / B), c1 = (int)((long long)m * (b + 1) / B);
  zc* P1 = S.part;
  zc* P2 = S.part + (long long)NA_BMAX * NA_PS;
  zc* P3 = S.part + 2LL * NA_BMAX * NA_PS;
  {
    double s = 0;
    const int cs = c1 - c0;
    for (long long e = threadIdx.x; e < (long long)n * cs; e += NT) {
      const int row = (int)(e / cs), c = c0 + (int)(e % cs);
      s += zabs2(X[(long long)row * m + c]);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0;
      for (int w = 0; w < NW; ++w) t += red[w];
      P3[(long long)b * NA_PS] = zmake(t, 0);
    }
    for (int c = c0 + threadIdx.x; c < c1; c += NT) S.colsq[c] = 0.0;
  }
  if (!na_sync(S, B)) return;
  const double thresh = rtol * sqrt(na_scalar(P3, B, 0));
  for (int j = 0; j < n; ++j) {
    zc* x = X + (long long)j * m;
    if (j > 0) {
      na_dots(X, m, j, x, c0, c1, P1 + (long long)b * NA_PS);
      if (!na_sync(S, B)) return;
      na_reduce(P1, B, j, h1);
      na_update(X, m, j, x, c0, c1, h1, buf);
    }
    na_dots(X, m, j, x, c0, c1, P2 + (long long)b * NA_PS);
    {
      const double s = na_norm2(x, c0, c1, red);
      if (threadIdx.x == 0) P2[(long long)b * NA_PS + n] = zmake(s, 0);
    }
    if (!na_sync(S, B)) return;
    na_reduce(P2, B, j, h2);
    const double s1 = na_scalar(P2, B, n);
    na_update(X, m, j, x, c0, c1, h2, buf);
    double hh = 0;
    {
      double v = 0;
      for (int t = threadIdx.x; t < j; t += NT) v += zabs2(h2[t]);
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      __syncthreads();
      if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = v;
      __syncthreads();
      for (int w = 0; w < NW; ++w) hh += red[w];
    }
    double nrm2 = s1 - hh;
    if (nrm2 <= 1e4 * thresh * thresh) {
      const double s = na_norm2(x, c0, c1, red);
      if (threadIdx.x == 0) P3[(long long)b * NA_PS] = zmake(s, 0);
      if (!na_sync(S, B)) return;
      nrm2 = na_scalar(P3, B, 0);
      if (!na_sync(S, B)) return;
    }
    const double nrm = sqrt(nrm2 > 0 ? nrm2 : 0.0);
    const bool full = nrm > thresh;
    if (b == 0) {
      for (int t = threadIdx.x; t < n; t += NT) {
        zc v = zmake(0, 0);
        if (t < j) v = zadd(j > 0 ? h1[t] : zmake(0, 0), h2[t]);
        else if (t == j) v = zmake(full ? nrm : 0.0, 0);
        L[(long long)j * n + t] = v;
      }
    }
    if (full) {
      const double inv = 1.0 / nrm;
      for (int c = c0 + threadIdx.x; c < c1; c += NT) {
        const zc v = zscale(x[c], inv);
        x[c] = v;
        S.colsq[c] += zabs2(v);
      }
      __syncthreads();
      continue;
    }
    // completion from the first unit vector at distance >= 1/2 from the rows so far
    {
      int first = 0x7fffffff, besti = 0x7fffffff;
      double bestv = -1.0;
      for (int c = c0 + threadIdx.x; c < c1; c += NT) {
        const double dist = 1.0 - S.colsq[c];
        if (dist >= 0.25 && c < first) first = c;
        if (dist > bestv || (dist == bestv && c < besti)) { bestv = dist; besti = c; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const int f2 = __shfl_xor_sync(0xffffffffu, first, o);
        const double v2 = __shfl_xor_sync(0xffffffffu, bestv, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, besti, o);
        first = min(first, f2);
        if (v2 > bestv || (v2 == bestv && i2 < besti)) { bestv = v2; besti = i2; }
      }
      __syncthreads();
      if (threadIdx.x % 32 == 0) {
        buf[threadIdx.x / 32][0] = zmake((double)first, bestv);
        buf[threadIdx.x / 32][1] = zmake((double)besti, 0);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double f = buf[0][0].x, bv = buf[0][0].y, bi = buf[0][1].x;
        for (int w = 1; w < NW; ++w) {
          f = fmin(f, buf[w][0].x);
          const double v2 = buf[w][0].y, i2 = buf[w][1].x;
          if (v2 > bv || (v2 == bv && i2 < bi)) { bv = v2; bi = i2; }
        }
        P3[(long long)b * NA_PS + 0] = zmake(f, 0);
        P3[(long long)b * NA_PS + 1] = zmake(bv, bi);
      }
    }
    if (!na_sync(S, B)) return;
    if (threadIdx.x == 0) {
      double f = 2147483647.0, bv = -2.0, bi = 2147483647.0;
      for (int bb = 0; bb < B; ++bb) {
        f = fmin(f, __ldcg(P3 + (long long)bb * NA_PS).x);
        const zc q = __ldcg(P3 + (long long)bb * NA_PS + 1);
        if (q.x > bv || (q.x == bv && q.y < bi)) { bv = q.x; bi = q.y; }
      }
      sel = (f < 2147483647.0) ? (int)f : (int)bi;
    }
    __syncthreads();
    const int p = sel;
    if (p >= c0 && p < c1)
      for (int t = threadIdx.x; t < j; t += NT) S.hp[t] = zconj(X[(long long)t * m + p]);
    if (!na_sync(S, B)) return;
    for (int t = threadIdx.x; t < j; t += NT) h1[t] = __ldcg(S.hp + t);
    __syncthreads();
    for (int c = c0 + threadIdx.x; c < c1; c += NT) x[c] = zmake(c == p ? 1.0 : 0.0, 0);
    __syncthreads();
    na_update(X, m, j, x, c0, c1, h1, buf);
    na_dots(X, m, j, x, c0, c1, P1 + (long long)b * NA_PS);
    if (!na_sync(S, B)) return;
    na_reduce(P1, B, j, h2);
    na_update(X, m, j, x, c0, c1, h2, buf);
    {
      const double s = na_norm2(x, c0, c1, red);
      if (threadIdx.x == 0) P2[(long long)b * NA_PS + n] = zmake(s, 0);
    }
    if (!na_sync(S, B)) return;
    const double en = sqrt(na_scalar(P2, B, n));
    const double inv = en > 0 ? 1.0 / en : 0.0;
    for (int c = c0 + threadIdx.x; c < c1; c += NT) {
      const zc v = zscale(x[c], inv);
      x[c] = v;
      S.colsq[c] += zabs2(v);
    }
    __syncthreads();
  }
}

// Device address of the scratch array and the co-resident block count, looked up once per device
// and again whenever the current context of that device is a different one (after a
// cudaDeviceReset the module is loaded anew and the array may sit elsewhere).  The context is
// identified by its driver-assigned unique id, read through the driver entry points the runtime
// exposes; none of these calls allocates device memory.
struct NaDevice {
  unsigned char* scratch = nullptr;
  int blocks = 0;
  unsigned long long ctx_id = 0;
};
std::mutex g_na_mu;
NaDevice g_na_dev[64];

typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);

// unique id of the calling thread's current context (0 if the driver cannot tell)
unsigned long long na_context_id() {
  static CtxGetCurrentFn get_cur = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
      get_cur = reinterpret_cast<CtxGetCurrentFn>(f1);
      get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    looked_up = true;
  }
  void* c = nullptr;
  unsigned long long id = 0;
  if (!get_cur || !get_id || get_cur(&c) != 0 || !c || get_id(c, &id) != 0) return 0;
  return id;
}

int na_setup(int dev, NaDevice* out) {
  std::lock_guard<std::mutex> lock(g_na_mu);
  NaDevice& d = g_na_dev[dev];
  const unsigned long long id = na_context_id();
  if (!d.scratch || id != d.ctx_id) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_lq_scratch) != cudaSuccess || !p) return TDVP_ERR_CUDA;
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lq_noalloc_kernel, NT, 0) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return TDVP_ERR_CUDA;
    d.blocks = per_sm * sms;
    d.scratch = static_cast<unsigned char*>(p);
    d.ctx_id = id;
  }
  *out = d;
  return TDVP_OK;
}

// true if the byte ranges [a, a + na) and [b, b + nb) share a byte
bool na_overlap(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + nb && y < x + na;
}

}  // namespace

extern "C" int tdvp_lq_noalloc(int n, int m, const double* X, double* Q, double* L, void* cuda_stream) {
  if (n < 1 || m < n || n > NA_NMAX || m > NA_MMAX || !X || !Q || !L) return TDVP_ERR_INVALID_ARG;
  const size_t xb = sizeof(zc) * (size_t)n * m, lb = sizeof(zc) * (size_t)n * n;
  if (na_overlap(X, xb, Q, xb) || na_overlap(X, xb, L, lb) || na_overlap(Q, xb, L, lb)) return TDVP_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return TDVP_ERR_CUDA;
  NaDevice nd;
  int rc = na_setup(dev, &nd);
  if (rc) return rc;
  if (cudaMemcpyAsync(Q, X, xb, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return TDVP_ERR_CUDA;
  // barrier words and the error word must start at zero; the rest is written before it is read
  if (cudaMemsetAsync(nd.scratch + NA_OFF_WORDS, 0, 256, st) != cudaSuccess) return TDVP_ERR_CUDA;
  int B = (m + 31) / 32;
  B = B < 1 ? 1 : (B > NA_BMAX ? NA_BMAX : B);
  if (B > nd.blocks) B = nd.blocks;
  zc* Xq = reinterpret_cast<zc*>(Q);
  zc* Lz = reinterpret_cast<zc*>(L);
  double rtol = 1e-13;
  unsigned char* scr = nd.scratch;
  void* args[] = {&Xq, &Lz, &n, &m, &B, &rtol, &scr};
  if (cudaLaunchCooperativeKernel((const void*)lq_noalloc_kernel, dim3(B), dim3(NT), args, 0, st) != cudaSuccess)
    return TDVP_ERR_CUDA;
  int err = 0;
  if (cudaMemcpyAsync(&err, nd.scratch + NA_OFF_WORDS + 8, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return TDVP_ERR_CUDA;
  return err ? TDVP_ERR_DEVICE_TIMEOUT : TDVP_OK;
}
