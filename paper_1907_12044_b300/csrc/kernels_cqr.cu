// Gauge-shift decomposition of Eq. QR (and its mirror LQ) by one thread-block cluster per
// realisation, with the whole matrix resident in the cluster's shared memory.  FP64.
//
// The matrix is X (n rows x m columns, n <= m), X = Rc * Qr with Qr having orthonormal rows and
// Rc lower triangular; for the left-to-right shift X is the transpose of C[(l s), r] and is read
// and written through that transposed view (no separate transpose pass), for the right-to-left
// shift X is C[l, (s r)] itself.
//
// Definition followed (the CPU oracle's): rows in order, classical Gram-Schmidt with one
// re-orthogonalisation pass; both passes' coefficients go to Rc; a row whose residual after the
// two passes is <= rtol*||X||_F gets a zero diagonal entry and is replaced by the first unit
// vector e_p with 1 - sum_t |Qr[t][p]|^2 >= 1/4 (else the farthest one, first on ties),
// orthogonalised by the same two passes and normalised.
//
// Layout: CTA k of a cluster of C holds the column slab [m k / C, m (k+1) / C) of all n rows in
// shared memory, plus its per-column sums |Qr[t][c]|^2.  Every reduction over columns is a
// per-CTA partial in shared memory, a hardware cluster barrier, and a sum of the C partials read
// through distributed shared memory in the fixed order k = 0..C-1, which every CTA does for
// itself; all CTAs therefore hold bit-identical coefficients and take identical branches.
// A full-rank row costs two cluster barriers (first-pass dots; residual, second-pass dots and
// norm), a rank-deficient row one more (completion vector).  The residual norm after the second
// pass is ||x'||^2 - ||g||^2 with x' the first-pass residual and g the second-pass coefficients:
// exact in exact arithmetic, and with x' already small its rounding error is O(eps ||x'||^2).
//
// There is no wait in this kernel other than the hardware barriers, and every branch that
// encloses one depends only on values all CTAs of the cluster share, so every CTA reaches every
// barrier.
#include <cooperative_groups.h>

#include "tdvp_internal.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int CT = TDVP_QR_THREADS;   // 256 threads = 8 warps
constexpr int CNW = CT / 32;
constexpr int CQR_NMAX = 256;

struct CqrJob {
  zc* X;          // global matrix
  zc* Rout;
  int n, m;
  int trans;      // 1: X[t][c] lives at X[c*n + t]; 0: at X[t*m + c]
  int rtrans;     // 1: Rout[t*n + j] = Rc[j][t]; 0: Rout[j*n + t] = Rc[j][t]
};

__device__ CqrJob cqr_job(int dir, int site, const SiteDev* sdr, const WorkDev& W, int dn, int dm) {
  CqrJob J;
  J.Rout = W.bond;
  const SiteDev& s = sdr[site];
  switch (dir) {
    case 0:  J.X = s.A;       J.n = s.Dr; J.m = s.Dl * s.d; J.trans = 1; J.rtrans = 1; break;
    case 1:  J.X = s.A;       J.n = s.Dl; J.m = s.d * s.Dr; J.trans = 0; J.rtrans = 0; break;
    case 3:  J.X = W.scratch; J.n = s.Dl; J.m = s.d * s.Dr; J.trans = 0; J.rtrans = 0; break;
    case 4:  J.X = W.scratch; J.n = s.Dr; J.m = s.Dl * s.d; J.trans = 1; J.rtrans = 1; break;
    default: J.X = W.scratch; J.n = dn;   J.m = dm;         J.trans = 0; J.rtrans = 1; break;
  }
  return J;
}

__host__ __device__ inline int slab_ld(int m, int C) { return ((m + C - 1) / C) | 1; }

// shared-memory bytes for an n x m matrix on a cluster of C
__host__ __device__ inline long long cqr_bytes(int n, int m, int C) {
  const long long ld = slab_ld(m, C);
  return 16LL * (n * ld + 2LL * (n + 4) + 3LL * n) + 8LL * ld;
}

// Partial dot products out[t] = sum_{c in slab} conj(Xs[t][c]) x[c] for t < j.  Groups of tpe
// consecutive lanes share one t and split the columns; a fixed shuffle tree combines them.
__device__ void slab_dots(const zc* Xs, int ld, const zc* x, int cs, int j, zc* out) {
  if (j <= 0) return;
  int tpe = 1;
  while (tpe < 32 && tpe * 2 * j <= CT) tpe *= 2;
  const int groups = CT / tpe;
  const int sub = threadIdx.x % tpe;
  for (int t0 = 0; t0 < j; t0 += groups) {
    const int t = t0 + threadIdx.x / tpe;
    zc a0 = zmake(0, 0), a1 = a0;
    if (t < j) {
      const zc* q = Xs + (long long)t * ld;
      int c = sub;
      for (; c + tpe < cs; c += 2 * tpe) {
        a0 = zcfma(q[c], x[c], a0);
        a1 = zcfma(q[c + tpe], x[c + tpe], a1);
      }
      if (c < cs) a0 = zcfma(q[c], x[c], a0);
    }
    zc s = zadd(a0, a1);
    for (int o = tpe / 2; o > 0; o >>= 1) {
      s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
    }
    if (t < j && sub == 0) out[t] = s;
  }
}

// x[c] = base(c) - sum_{t<j} h[t] Xs[t][c] on the slab, then post(c, value).  base(c) is x[c]
// or, for a completion vector, the unit vector e_p.  Groups of tpe lanes split the t sum.
template <class Post>
__device__ void slab_update(zc* Xs, int ld, zc* x, int cs, int j, const zc* h, int unit_p, Post post) {
  int tpe = 1;
  while (tpe < 32 && tpe * 2 * cs <= CT && tpe * 2 <= j) tpe *= 2;
  const int groups = CT / tpe;
  const int sub = threadIdx.x % tpe;
  for (int c0 = 0; c0 < cs; c0 += groups) {
    const int c = c0 + threadIdx.x / tpe;
    zc a0 = zmake(0, 0), a1 = a0;
    if (c < cs) {
      int t = sub;
      for (; t + tpe < j; t += 2 * tpe) {
        a0 = zfma(h[t], Xs[(long long)t * ld + c], a0);
        a1 = zfma(h[t + tpe], Xs[(long long)(t + tpe) * ld + c], a1);
      }
      if (t < j) a0 = zfma(h[t], Xs[(long long)t * ld + c], a0);
    }
    zc s = zadd(a0, a1);
    for (int o = tpe / 2; o > 0; o >>= 1) {
      s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
    }
    if (c < cs && sub == 0) {
      const zc b = unit_p >= 0 ? zmake(c == unit_p ? 1.0 : 0.0, 0.0) : x[c];
      post(c, zsub(b, s));
    }
  }
}

// sum of slot `off` of the C partial buffers whose base addresses are rb[0..C-1], in the order
// q = 0..C-1; all C loads are issued before the first add
__device__ __forceinline__ zc gather_sum(zc* const* rb, int C, int off) {
  zc v[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = q < C ? rb[q][off] : zmake(0, 0);
  zc s = v[0];
#pragma unroll
  for (int q = 1; q < 16; ++q) if (q < C) s = zadd(s, v[q]);
  return s;
}

__device__ double cta_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = v;
  __syncthreads();
  double t = 0;
  for (int w = 0; w < CNW; ++w) t += red[w];
  return t;
}

__global__ void __launch_bounds__(CT)
cqr_kernel(int dir, int site, const SiteDev* __restrict__ sd, const WorkDev* __restrict__ wk, int N_sites,
           double rtol, int dn, int dm) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[CNW];
  __shared__ double sc[4];
  __shared__ zc cand[2 * CNW];
  __shared__ zc* rb[2][16];     // the partial buffers of every CTA of the cluster (both parities)
  __shared__ int sp;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int k = (int)cl.block_rank();
  const int r = blockIdx.x / C;
  const SiteDev* sdr = sd + (long long)r * N_sites;
  const WorkDev& W = wk[r];
  const CqrJob J = cqr_job(dir, site, sdr, W, dn, dm);
  const int n = J.n, m = J.m;
  // every CTA of the cluster sees the same job, so all return here together or none does
  if (n <= 0 || n > CQR_NMAX || n > m) {
    if (k == 0 && threadIdx.x == 0) atomicExch(W.err, -1);
    return;
  }
  const int ld = slab_ld(m, C);
  const int c0 = (int)((long long)m * k / C), c1 = (int)((long long)m * (k + 1) / C), cs = c1 - c0;
  const int PL = n + 4;
  zc* Xs = reinterpret_cast<zc*>(smem);         // [n][ld]
  zc* buf = Xs + (long long)n * ld;              // [2][PL] partials: dots, then norm and candidates
  zc* h1 = buf + 2 * PL;                         // first-pass coefficients
  zc* g = h1 + n;                                // second-pass coefficients
  zc* qp = g + n;                                // conj(Qr[t][p]) of a completion
  double* colsq = reinterpret_cast<double*>(qp + n);

  if (threadIdx.x < 2 * C) rb[threadIdx.x / C][threadIdx.x % C] = cl.map_shared_rank(buf + (threadIdx.x / C) * PL, threadIdx.x % C);

  // ---- load the slab, ||X||_F ----
  {
    double s = 0;
    const long long E = (long long)n * cs;
    for (long long e = threadIdx.x; e < E; e += CT) {
      int t, c;
      if (J.trans) { c = (int)(e / n); t = (int)(e % n); }     // consecutive threads: consecutive t
      else { t = (int)(e / cs); c = (int)(e % cs); }
      const zc v = J.trans ? J.X[(long long)(c0 + c) * n + t] : J.X[(long long)t * m + c0 + c];
      Xs[(long long)t * ld + c] = v;
      s += zabs2(v);
    }
    for (int c = threadIdx.x; c < cs; c += CT) colsq[c] = 0.0;
    s = cta_sum(s, red);
    if (threadIdx.x == 0) buf[n] = zmake(s, 0.0);
  }
  cl.sync();
  if (threadIdx.x == 0) sc[0] = rtol * sqrt(gather_sum(rb[0], C, n).x);
  __syncthreads();
  const double thresh = sc[0];
  int ph = 1;   // parity of the next partial buffer

  for (int j = 0; j < n; ++j) {
    zc* x = Xs + (long long)j * ld;
    // ---- (A) first-pass dots and completion candidates ----
    if (j > 0) {
      zc* P = buf + ph * PL;
      slab_dots(Xs, ld, x, cs, j, P);
      {
        int first = 0x7fffffff, besti = 0x7fffffff;
        double bestv = -1.0;
        for (int c = threadIdx.x; c < cs; c += CT) {
          const double dist = 1.0 - colsq[c];
          if (dist >= 0.25 && c0 + c < first) first = c0 + c;
          if (dist > bestv || (dist == bestv && c0 + c < besti)) { bestv = dist; besti = c0 + c; }
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
          cand[2 * (threadIdx.x / 32)] = zmake((double)first, bestv);
          cand[2 * (threadIdx.x / 32) + 1] = zmake((double)besti, 0.0);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          double f = cand[0].x, bv = cand[0].y, bi = cand[1].x;
          for (int w = 1; w < CNW; ++w) {
            f = fmin(f, cand[2 * w].x);
            const double v2 = cand[2 * w].y, i2 = cand[2 * w + 1].x;
            if (v2 > bv || (v2 == bv && i2 < bi)) { bv = v2; bi = i2; }
          }
          P[n + 1] = zmake(f, 0.0);
          P[n + 2] = zmake(bv, bi);
        }
      }
      cl.sync();
      if (threadIdx.x < j) {
        h1[threadIdx.x] = gather_sum(rb[ph], C, threadIdx.x);
      } else if (threadIdx.x == j) {
        zc f[16], b[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          f[q] = q < C ? rb[ph][q][n + 1] : zmake(2147483647.0, 0);
          b[q] = q < C ? rb[ph][q][n + 2] : zmake(-2.0, 2147483647.0);
        }
        double fm = 2147483647.0, bv = -2.0, bi = 2147483647.0;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          fm = fmin(fm, f[q].x);
          if (b[q].x > bv || (b[q].x == bv && b[q].y < bi)) { bv = b[q].x; bi = b[q].y; }
        }
        const int p = (fm < 2147483647.0) ? (int)fm : (bi < 2147483647.0 ? (int)bi : 0);
        sp = min(max(p, 0), m - 1);
      }
      ph ^= 1;
      __syncthreads();
    } else if (threadIdx.x == 0) {
      sp = 0;     // no rows yet: every unit vector is at distance 1, the first qualifies
    }
    // ---- (B) first-pass update, second-pass dots, residual norm ----
    {
      zc* P = buf + ph * PL;
      slab_update(Xs, ld, x, cs, j, h1, -1, [&](int c, zc v) { x[c] = v; });
      __syncthreads();
      slab_dots(Xs, ld, x, cs, j, P);
      double s = 0;
      for (int c = threadIdx.x; c < cs; c += CT) s += zabs2(x[c]);
      s = cta_sum(s, red);
      if (threadIdx.x == 0) P[n] = zmake(s, 0.0);
      cl.sync();
      if (threadIdx.x < j) g[threadIdx.x] = gather_sum(rb[ph], C, threadIdx.x);
      else if (threadIdx.x == j) sc[1] = gather_sum(rb[ph], C, n).x;
      ph ^= 1;
      __syncthreads();
    }
    double gg = 0;
    {
      double v = 0;
      for (int t = threadIdx.x; t < j; t += CT) v += zabs2(g[t]);
      gg = cta_sum(v, red);
    }
    const double en_x = sqrt(fmax(sc[1] - gg, 0.0));
    const bool full = en_x > thresh;
    // Rc row j: both passes' coefficients, diagonal = residual norm (0 when dropped)
    if (k == 0) {
      for (int t = threadIdx.x; t < n; t += CT) {
        zc v = zmake(0, 0);
        if (t < j) v = zadd(h1[t], g[t]);
        else if (t == j) v = zmake(full ? en_x : 0.0, 0.0);
        J.Rout[J.rtrans ? (long long)t * n + j : (long long)j * n + t] = v;
      }
    }
    double en = en_x;
    if (!full) {
      // ---- (C') completion: e_p - sum_t conj(Qr[t][p]) Qr[t], then its second pass ----
      const int p = sp;
      int owner = 0;
      while (owner + 1 < C && (int)((long long)m * (owner + 1) / C) <= p) ++owner;
      const int po = p - (int)((long long)m * owner / C);
      const zc* Xo = cl.map_shared_rank(Xs, owner);
      for (int t = threadIdx.x; t < j; t += CT) qp[t] = zconj(Xo[(long long)t * ld + po]);
      __syncthreads();
      const int unit = (p >= c0 && p < c1) ? p - c0 : cs;    // cs: the unit entry is elsewhere
      zc* P = buf + ph * PL;
      slab_update(Xs, ld, x, cs, j, qp, unit, [&](int c, zc v) { x[c] = v; });
      __syncthreads();
      slab_dots(Xs, ld, x, cs, j, P);
      double s = 0;
      for (int c = threadIdx.x; c < cs; c += CT) s += zabs2(x[c]);
      s = cta_sum(s, red);
      if (threadIdx.x == 0) P[n] = zmake(s, 0.0);
      cl.sync();
      if (threadIdx.x < j) g[threadIdx.x] = gather_sum(rb[ph], C, threadIdx.x);
      else if (threadIdx.x == j) sc[1] = gather_sum(rb[ph], C, n).x;
      ph ^= 1;
      __syncthreads();
      double v = 0;
      for (int t = threadIdx.x; t < j; t += CT) v += zabs2(g[t]);
      gg = cta_sum(v, red);
      en = sqrt(fmax(sc[1] - gg, 0.0));
    }
    // ---- (D) second-pass update and normalisation ----
    const double inv = en > 0 ? 1.0 / en : 0.0;
    slab_update(Xs, ld, x, cs, j, g, -1, [&](int c, zc v) {
      const zc q = zscale(v, inv);
      x[c] = q;
      colsq[c] += zabs2(q);
    });
    __syncthreads();
  }

  // ---- write the slab of Qr back ----
  {
    const long long E = (long long)n * cs;
    for (long long e = threadIdx.x; e < E; e += CT) {
      int t, c;
      if (J.trans) { c = (int)(e / n); t = (int)(e % n); }
      else { t = (int)(e / cs); c = (int)(e % cs); }
      const zc v = Xs[(long long)t * ld + c];
      if (J.trans) J.X[(long long)(c0 + c) * n + t] = v;
      else J.X[(long long)t * m + c0 + c] = v;
    }
  }
  cl.sync();    // no CTA leaves while another may still read its shared memory
}

}  // namespace

long long cqr_smem_bytes(int n, int m, int C) { return cqr_bytes(n, m, C); }

cudaError_t cqr_setup(int device) {
  (void)device;
  cudaError_t e = cudaFuncSetAttribute(cqr_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(cqr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TDVP_CQR_SMEM_MAX);
}

// number of clusters of C that can be resident at once with `smem` bytes each (0: not launchable)
int cqr_max_clusters(int C, long long smem) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(CT);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int nc = 0;
  if (cudaOccupancyMaxActiveClusters(&nc, (void*)cqr_kernel, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nc;
}

cudaError_t launch_cluster_qr(int dir, int site, const SiteDev* sd, const WorkDev* wk, int R, int N_sites, int C,
                              long long smem, double rtol, int dbg_n, int dbg_m, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(R * C);
  cfg.blockDim = dim3(CT);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, cqr_kernel, dir, site, sd, wk, N_sites, rtol, dbg_n, dbg_m);
}
