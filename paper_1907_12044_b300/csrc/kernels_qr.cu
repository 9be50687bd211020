// Gauge-shift decomposition of Eq. QR (and its mirror "RQ"/LQ) on the device, FP64.
//
// The matrix is handled as X (n rows x m columns, row-major, n <= m): X = Rc * Qr with Qr having
// orthonormal rows and Rc lower triangular.  For the left-to-right shift X is the transpose of
// the site tensor C[(l s), r], so Q = Qr^T and R = Rc^T; for the right-to-left shift X is
// C[l, (s r)] itself.  Rows are orthogonalised one after another by classical Gram-Schmidt with
// one re-orthogonalisation pass.  A row whose residual is <= rtol*||X||_F is treated as linearly
// dependent: its diagonal entry is 0 and the row is replaced by the first unit vector e_p whose
// distance to the span of the rows so far is >= 1/2 (1 - sum_t |Qr[t][p]|^2 >= 1/4), else by the
// one farthest from it, orthogonalised with the same two passes (the completion of a weakly
// correlated start that Sec. II.C calls for).
//
// One realisation is processed by B blocks, each owning a contiguous slab of columns; every
// access to X and Qr stays inside the slab, and only per-block partial sums cross blocks.  The
// blocks of a realisation meet at a group barrier (global counter + generation word) whose wait
// is bounded: after ~1 s it records TDVP_ERR_DEVICE_TIMEOUT in the realisation's error word and
// every block returns.  The kernel is launched cooperatively, so all blocks are co-resident.
#include "tdvp_internal.cuh"
#include <cooperative_groups.h>

namespace {

constexpr int QT = TDVP_QR_THREADS;       // 256 threads = 8 warps
constexpr int NW = QT / 32;
constexpr int QR_NMAX = 512;              // largest n (bond dimension) handled
constexpr long long SPIN_LIMIT = 1LL << 24;

struct QrJob {
  zc* X;
  zc* Rout;
  int n, m;
  int rtrans;    // 1: Rout[t*n + j] = Rc[j][t] (R = Rc^T); 0: Rout[j*n + t] = Rc[j][t]
};

__device__ QrJob qr_job(int dir, int site, const SiteDev* sdr, const WorkDev& W, int dn, int dm) {
  QrJob J;
  if (dir == 0) {
    const SiteDev& s = sdr[site];
    J.X = W.scratch; J.n = s.Dr; J.m = s.Dl * s.d; J.Rout = W.bond; J.rtrans = 1;
  } else if (dir == 1) {
    const SiteDev& s = sdr[site];
    J.X = s.A; J.n = s.Dl; J.m = s.d * s.Dr; J.Rout = W.bond; J.rtrans = 0;
  } else {
    J.X = W.scratch; J.n = dn; J.m = dm; J.Rout = W.bond; J.rtrans = 1;
  }
  return J;
}

// Bounded barrier over the B blocks of one realisation.  Returns false if this or an earlier
// wait gave up (the caller then returns).
__device__ bool group_sync(const WorkDev& W, int nblocks) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = W.bar + 1;
    volatile int* err = W.err;
    int good = (*err == 0);
    if (good && nblocks > 1) {
      const unsigned g = *gen;
      __threadfence();
      const unsigned arrived = atomicAdd(W.bar, 1u) + 1u;
      if (arrived == (unsigned)nblocks) {
        atomicExch(W.bar, 0u);
        __threadfence();
        atomicAdd(W.bar + 1, 1u);
      } else {
        long long spins = 0;
        while (*gen == g) {
          if (*err != 0) { good = 0; break; }
          if (++spins > SPIN_LIMIT) { atomicExch(W.err, -5); good = 0; break; }
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

__device__ __forceinline__ zc ldcg(const zc* p) { return __ldcg(p); }

// Partial dots p_t = sum_{c in slab} conj(Q_t[c]) x[c] for t < j: warp per t, lanes over columns.
__device__ void slab_dots(const zc* X, int m, int j, const zc* x, int c0, int c1, zc* Pout) {
  const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
  for (int t = wid; t < j; t += NW) {
    const zc* q = X + (long long)t * m;
    zc s = zmake(0, 0);
    for (int c = c0 + lane; c < c1; c += 32) s = zcfma(q[c], x[c], s);
    for (int o = 16; o > 0; o >>= 1) {
      s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
    }
    if (lane == 0) Pout[t] = s;
  }
}

// h_t = sum_b P[b][t] for t < cnt in block order (identical in every block).
__device__ void reduce_over_blocks(const zc* Pbase, int PS, int B, int cnt, zc* h) {
  const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
  for (int t = wid; t < cnt; t += NW) {
    zc s = zmake(0, 0);
    for (int b = lane; b < B; b += 32) s = zadd(s, ldcg(Pbase + (long long)b * PS + t));
    for (int o = 16; o > 0; o >>= 1) {
      s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
    }
    if (lane == 0) h[t] = s;
  }
  __syncthreads();
}

// x[c] -= sum_{t<j} h_t Q_t[c] over the slab: warp w sums t = w (mod 8), then a fixed-order merge.
__device__ void slab_update(const zc* X, int m, int j, zc* x, int c0, int c1, const zc* h, zc (*buf)[32]) {
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

__device__ double slab_norm2(const zc* x, int c0, int c1, double* red) {
  double s = 0;
  for (int c = c0 + threadIdx.x; c < c1; c += QT) s += zabs2(x[c]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
  __syncthreads();
  if (lane == 0) red[wid] = s;
  __syncthreads();
  double t = 0;
  for (int w = 0; w < NW; ++w) t += red[w];
  return t;
}

__device__ double sum_scalar_over_blocks(const zc* Pbase, int PS, int B, int slot) {
  // fixed order: lanes stride over blocks, then butterfly; every block gets the same value
  const int lane = threadIdx.x % 32;
  double s = 0;
  for (int b = lane; b < B; b += 32) s += ldcg(Pbase + (long long)b * PS + slot).x;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;   // valid in every lane of every warp
}

__global__ void __launch_bounds__(QT)
row_qr_kernel(int dir, int site, const SiteDev* __restrict__ sd, const WorkDev* __restrict__ wk, int N_sites,
              int B, double rtol, int dn, int dm) {
  __shared__ zc h1[QR_NMAX];
  __shared__ zc h2[QR_NMAX];
  __shared__ zc buf[NW][32];
  __shared__ double red[NW];
  __shared__ int sel[4];
  const int r = blockIdx.x / B, b = blockIdx.x % B;
  const SiteDev* sdr = sd + (long long)r * N_sites;
  const WorkDev& W = wk[r];
  const QrJob J = qr_job(dir, site, sdr, W, dn, dm);
  const int n = J.n, m = J.m;
  if (n <= 0 || n > QR_NMAX || n > m) {
    if (b == 0 && threadIdx.x == 0) atomicExch(W.err, -1);
    return;
  }
  const int c0 = (int)((long long)m * b / B), c1 = (int)((long long)m * (b + 1) / B);
  zc* X = J.X;
  const int PS = n + 4;
  zc* P1 = W.qpart;
  zc* P2 = W.qpart + (long long)B * PS;
  zc* P3 = W.qpart + 2LL * B * PS;
  double* colsq = W.colsq;

  // ||X||_F over the slab
  {
    double s = 0;
    const int cs = c1 - c0;
    for (long long e = threadIdx.x; e < (long long)n * cs; e += QT) {
      const int row = (int)(e / cs), c = c0 + (int)(e % cs);
      s += zabs2(X[(long long)row * m + c]);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0;
      for (int w = 0; w < NW; ++w) t += red[w];
      P3[(long long)b * PS] = zmake(t, 0);
    }
    for (int c = c0 + threadIdx.x; c < c1; c += QT) colsq[c] = 0.0;
  }
  if (!group_sync(W, B)) return;
  const double thresh = rtol * sqrt(sum_scalar_over_blocks(P3, PS, B, 0));

  for (int j = 0; j < n; ++j) {
    zc* x = X + (long long)j * m;
    // first pass
    if (j > 0) {
      slab_dots(X, m, j, x, c0, c1, P1 + (long long)b * PS);
      if (!group_sync(W, B)) return;
      reduce_over_blocks(P1, PS, B, j, h1);
      slab_update(X, m, j, x, c0, c1, h1, buf);
    }
    // second pass dots and the norm after the first pass
    slab_dots(X, m, j, x, c0, c1, P2 + (long long)b * PS);
    {
      const double s = slab_norm2(x, c0, c1, red);
      if (threadIdx.x == 0) P2[(long long)b * PS + n] = zmake(s, 0);
    }
    if (!group_sync(W, B)) return;
    reduce_over_blocks(P2, PS, B, j, h2);
    const double s1 = sum_scalar_over_blocks(P2, PS, B, n);
    slab_update(X, m, j, x, c0, c1, h2, buf);
    double hh = 0;
    {
      double v = 0;
      for (int t = threadIdx.x; t < j; t += QT) v += zabs2(h2[t]);
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      __syncthreads();
      if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = v;
      __syncthreads();
      for (int w = 0; w < NW; ++w) hh += red[w];
    }
    double nrm2 = s1 - hh;
    if (nrm2 <= 1e4 * thresh * thresh) {          // near the rank threshold: measure directly
      const double s = slab_norm2(x, c0, c1, red);
      if (threadIdx.x == 0) P3[(long long)b * PS] = zmake(s, 0);
      if (!group_sync(W, B)) return;
      nrm2 = sum_scalar_over_blocks(P3, PS, B, 0);
      if (!group_sync(W, B)) return;              // P3 is reused below
    }
    const double nrm = sqrt(nrm2 > 0 ? nrm2 : 0.0);
    const bool full = nrm > thresh;
    if (b == 0) {
      for (int t = threadIdx.x; t < n; t += QT) {
        zc v = zmake(0, 0);
        if (t < j) v = zadd(j > 0 ? h1[t] : zmake(0, 0), h2[t]);
        else if (t == j) v = zmake(full ? nrm : 0.0, 0);
        const long long o = J.rtrans ? (long long)t * n + j : (long long)j * n + t;
        J.Rout[o] = v;
      }
    }
    if (full) {
      const double inv = 1.0 / nrm;
      for (int c = c0 + threadIdx.x; c < c1; c += QT) {
        const zc v = zscale(x[c], inv);
        x[c] = v;
        colsq[c] += zabs2(v);
      }
      __syncthreads();
      continue;
    }
    // ---- completion by a unit vector e_p ----
    {
      int first = 0x7fffffff, besti = 0x7fffffff;
      double bestv = -1.0;
      for (int c = c0 + threadIdx.x; c < c1; c += QT) {
        const double dist = 1.0 - colsq[c];
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
      if (threadIdx.x % 32 == 0) { buf[threadIdx.x / 32][0] = zmake((double)first, bestv); buf[threadIdx.x / 32][1] = zmake((double)besti, 0); }
      __syncthreads();
      if (threadIdx.x == 0) {
        double f = buf[0][0].x, bv = buf[0][0].y, bi = buf[0][1].x;
        for (int w = 1; w < NW; ++w) {
          f = fmin(f, buf[w][0].x);
          const double v2 = buf[w][0].y, i2 = buf[w][1].x;
          if (v2 > bv || (v2 == bv && i2 < bi)) { bv = v2; bi = i2; }
        }
        P3[(long long)b * PS + 0] = zmake(f, 0);
        P3[(long long)b * PS + 1] = zmake(bv, bi);
      }
    }
    if (!group_sync(W, B)) return;
    if (threadIdx.x == 0) {
      double f = 2147483647.0, bv = -2.0, bi = 2147483647.0;
      for (int bb = 0; bb < B; ++bb) {
        f = fmin(f, ldcg(P3 + (long long)bb * PS).x);
        const zc q = ldcg(P3 + (long long)bb * PS + 1);
        if (q.x > bv || (q.x == bv && q.y < bi)) { bv = q.x; bi = q.y; }
      }
      sel[0] = (f < 2147483647.0) ? (int)f : (int)bi;
    }
    __syncthreads();
    const int p = sel[0];
    zc* hp = W.qhp;
    if (p >= c0 && p < c1)
      for (int t = threadIdx.x; t < j; t += QT) hp[t] = zconj(X[(long long)t * m + p]);
    if (!group_sync(W, B)) return;
    for (int t = threadIdx.x; t < j; t += QT) h1[t] = ldcg(hp + t);
    __syncthreads();
    for (int c = c0 + threadIdx.x; c < c1; c += QT) x[c] = zmake(c == p ? 1.0 : 0.0, 0);
    __syncthreads();
    slab_update(X, m, j, x, c0, c1, h1, buf);
    slab_dots(X, m, j, x, c0, c1, P1 + (long long)b * PS);
    if (!group_sync(W, B)) return;
    reduce_over_blocks(P1, PS, B, j, h2);
    slab_update(X, m, j, x, c0, c1, h2, buf);
    {
      const double s = slab_norm2(x, c0, c1, red);
      if (threadIdx.x == 0) P2[(long long)b * PS + n] = zmake(s, 0);
    }
    if (!group_sync(W, B)) return;
    const double en = sqrt(sum_scalar_over_blocks(P2, PS, B, n));
    const double inv = en > 0 ? 1.0 / en : 0.0;
    for (int c = c0 + threadIdx.x; c < c1; c += QT) {
      const zc v = zscale(x[c], inv);
      x[c] = v;
      colsq[c] += zabs2(v);
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_row_qr(int dir, int site, const SiteDev* sd, const WorkDev* wk, int R, int N_sites,
                          int blocks_per_r, double rtol, int dbg_n, int dbg_m, cudaStream_t st) {
  int B = blocks_per_r < 1 ? 1 : blocks_per_r;
  void* args[] = {&dir, &site, (void*)&sd, (void*)&wk, &N_sites, &B, &rtol, &dbg_n, &dbg_m};
  dim3 grid(R * B), block(QT);
  return cudaLaunchCooperativeKernel((const void*)row_qr_kernel, grid, block, args, 0, st);
}

int qr_max_coresident_blocks(int device) {
  int per_sm = 0, sms = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, row_qr_kernel, QT, 0);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  return per_sm * sms;
}
