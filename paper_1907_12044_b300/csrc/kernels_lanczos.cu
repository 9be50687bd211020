// Lanczos exponential exp(i theta H) v of the TDVP-PS local steps (Sec. II.A.2, TDVP-PS: the
// Krylov subspace method, Lanczos for a Hermitian operator, dimension adaptive until the result
// converges).  FP64 throughout.
//
// Per iteration j the host enqueues: matvec (x -> w), then
//   dots     p_t = <V_t, w>                         (partial sums per chunk)
//   upd1     h1 = sum p; w -= V h1; p2_t = <V_t, w>  (first Gram-Schmidt pass)
//   upd2     h2 = sum p2; w -= V h2; |w|^2 partials  (re-orthogonalisation pass); the block
//            that finishes last (atomic count per realisation) then takes the tridiagonal step:
//            beta_j = |w|; alpha_j = Re(h1_j + h2_j); c = exp(i theta T_{j+1}) e_1 (Chebyshev);
//            stop when ||v|| beta_j |c_j| <= tol, or k = kcap, or beta_j = 0
//   next     V_{j+1} = x = w / beta_j
// Every kernel of an iteration returns at once when the solve of its realisation is done, so
// the host may enqueue more iterations than needed.  Reductions are two-level with a fixed
// order, so results are bit-reproducible run to run.
#include "tdvp_internal.cuh"
#include "tc_pack.cuh"
#include <cmath>

namespace {

constexpr int NT = TDVP_VEC_THREADS;
constexpr int PSTRIDE = TDVP_KMAX_HARD + 2;
constexpr int TRI_THREADS = NT;   // the tridiagonal step runs in a block of the vector kernel
constexpr int MAX_CHEB = 512;
constexpr int BESSEL_CAP = 2 * MAX_CHEB;   // Miller start m = N + 24 + x + 1 with N <= 497, x <= 400
constexpr double CHEB_XSUB = 400.0;        // largest x of one Chebyshev series (N(400) = 497 terms)
constexpr int CHEB_MAX_SUB = 64;           // substeps of one exponential at most (x <= 25600)

// Terms of the Jacobi-Anger series exp(i x T~) = sum_{n<=N} (2 - delta_n0) i^n J_n(x) T_n(T~) so
// that the dropped tail 2 sum_{n>N} |J_n(x)| stays below 1e-17: past n = x the Bessel functions
// fall off over the Airy transition width ~x^(1/3), so N = x + 12 x^(1/3) + 8 (checked against
// independently computed J_n for x from 1 to 480; a fixed margin N = x + 30 leaves 3e-11 at x = 50
// and 1e-4 at x = 480).
__device__ __forceinline__ int cheb_terms(double x) { return (int)ceil(x + 12.0 * cbrt(x)) + 8; }
constexpr int TRI_SH = 3 * TRI_THREADS + MAX_CHEB + 2 * (TRI_THREADS / 32) + 8 + 2 * BESSEL_CAP;

struct VecGeom {
  long long n;       // vector length
  int nblk;          // chunks used by this realisation
  long long c0, c1;  // chunk of this block
};

__device__ __forceinline__ long long vec_len(const SiteDev* sdr, int site, int kind) {
  const SiteDev& s = sdr[site];
  return kind == 0 ? (long long)s.Dl * s.d * s.Dr : (long long)s.Dr * s.Dr;
}

// chunking of a vector of n elements: ceil(n / 32) chunks, at most `cap` (<= 148); every kernel of
// one solve uses the same cap, so a block owns the same elements and partial-sum slots throughout
__device__ __forceinline__ VecGeom geom(long long n, int b, int cap) {
  VecGeom g;
  g.n = n;
  long long nb = (n + TDVP_VEC_CHUNK - 1) / TDVP_VEC_CHUNK;
  if (nb > cap) nb = cap;
  if (nb < 1) nb = 1;
  g.nblk = (int)nb;
  const long long ch = (n + nb - 1) / nb;
  g.c0 = (long long)b * ch;
  g.c1 = g.c0 + ch < n ? g.c0 + ch : n;
  return g;
}

__device__ __forceinline__ zc* P(const WorkDev& W, int tab, int b, int t) {
  return W.part + ((long long)tab * TDVP_MAX_VEC_BLOCKS + b) * PSTRIDE + t;
}

__device__ __forceinline__ zc* src_ptr(const WorkDev& W, const SiteDev* sdr, int site, int which) {
  if (which == 0) return W.x;
  if (which == 1) return sdr[site].A;
  if (which == 2) return W.bond;
  return W.w;
}

// Block-wide sum of a complex value; result valid in every thread.  `red` holds 2*(NT/32) doubles.
__device__ __forceinline__ zc block_zsum(zc v, double* red) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
  __syncthreads();
  if (lane == 0) { red[2 * wid] = v.x; red[2 * wid + 1] = v.y; }
  __syncthreads();
  zc s = zmake(0, 0);
  for (int i = 0; i < NT / 32; ++i) { s.x += red[2 * i]; s.y += red[2 * i + 1]; }
  return s;
}

// h[t] = sum_b P(tab, b, t) for t <= j, one warp per t in a fixed order (same in every block).
__device__ void reduce_partials(const WorkDev& W, int tab, int nblk, int j, zc* h) {
  const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
  for (int t = wid; t <= j; t += NT / 32) {
    zc s = zmake(0, 0);
    for (int b = lane; b < nblk; b += 32) s = zadd(s, __ldcg(P(W, tab, b, t)));
    for (int o = 16; o > 0; o >>= 1) {
      s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
    }
    if (lane == 0) h[t] = s;
  }
  __syncthreads();
}

// Sum over the 32 lanes of a warp of G complex values per lane, for all G at once: a butterfly in
// which each step halves the values a lane keeps and adds its partner's half.  After log2(G) steps
// lane l holds the warp total of value (l % G) partially reduced over groups of G lanes, which the
// remaining steps finish.  Returns the total of value (lane % G) (valid in every lane).
template <int G>
__device__ __forceinline__ zc warp_transpose_sum(zc (&v)[G]) {
  const int lane = threadIdx.x % 32;
#pragma unroll
  for (int half = G / 2; half >= 1; half >>= 1) {
    const bool upper = (lane & half) != 0;
#pragma unroll
    for (int q = 0; q < half; ++q) {
      // keep v[q + half] if upper else v[q]; send the other one to the partner lane
      const zc send = upper ? v[q] : v[q + half];
      zc got;
      got.x = __shfl_xor_sync(0xffffffffu, send.x, half);
      got.y = __shfl_xor_sync(0xffffffffu, send.y, half);
      const zc keep = upper ? v[q + half] : v[q];
      v[q] = zadd(keep, got);
    }
  }
  zc s = v[0];   // now lane holds partial of value (lane % G)
#pragma unroll
  for (int o = G; o < 32; o <<= 1) {
    s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
    s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
  }
  return s;
}

constexpr int DOT_G = 8;   // coefficients summed per pass over the chunk

// Partial dots p_t = sum_{e in chunk} conj(V_t[e]) w[e] for t <= j into table `tab`.  `wsum` is a
// shared buffer of (NT/32) * DOT_G complex values (16-byte aligned as a zc array).
__device__ void chunk_dots(const WorkDev& W, const VecGeom& g, int j, int tab, int b, zc* wsum) {
  constexpr int G = DOT_G;
  const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
  for (int t0 = 0; t0 <= j; t0 += G) {
    zc acc[G];
#pragma unroll
    for (int q = 0; q < G; ++q) acc[q] = zmake(0, 0);
    for (long long e = g.c0 + threadIdx.x; e < g.c1; e += NT) {
      const zc we = W.w[e];
#pragma unroll
      for (int q = 0; q < G; ++q)
        if (t0 + q <= j) acc[q] = zcfma(W.V[(t0 + q) * W.ldV + e], we, acc[q]);
    }
    const zc s = warp_transpose_sum<G>(acc);
    if (lane < G) wsum[wid * G + lane] = s;
    __syncthreads();
    if (threadIdx.x < G && t0 + (int)threadIdx.x <= j) {
      zc tot = zmake(0, 0);
      for (int w = 0; w < NT / 32; ++w) tot = zadd(tot, wsum[w * G + threadIdx.x]);
      *P(W, tab, b, t0 + threadIdx.x) = tot;
    }
    __syncthreads();
  }
}

// Element e of the Krylov vector of (site, kind) as the packed B operand of the next tensor-core
// matvec: site vectors x[a][(s b)] give row (s b), k = a; bond vectors D[l][r] give row r, k = l.
__device__ __forceinline__ void pack_krylov(const LzArgs& a, const SiteDev* sdr, const WorkDev& W, long long e,
                                            zc v) {
  const SiteDev& s = sdr[a.site];
  const int Nn = a.kind == 0 ? s.d * s.Dr : s.Dr;
  const int Kd = a.kind == 0 ? s.Dl : s.Dr;
  const int k = (int)(e / Nn), n = (int)(e % Nn);
  tcpack::pk_store(W.tc_x, tcpack::BN, (Kd + tcpack::BK - 1) / tcpack::BK, n, k, v.x, v.y, a.pack_pm);
}

__global__ void __launch_bounds__(NT) lz_start1(LzArgs a) {
  pdl_enter();
  __shared__ double red[2 * 8 * NT / 32];
  const int r = blockIdx.y, b = blockIdx.x;
  const SiteDev* sdr = a.sd + (long long)r * a.N_sites;
  const WorkDev& W = a.wk[r];
  const VecGeom g = geom(vec_len(sdr, a.site, a.kind), b, a.bcap);
  if (b >= g.nblk) return;
  const zc* src = src_ptr(W, sdr, a.site, a.src);
  zc acc = zmake(0, 0);
  for (long long e = g.c0 + threadIdx.x; e < g.c1; e += NT) acc.x += zabs2(src[e]);
  const zc s = block_zsum(acc, red);
  if (threadIdx.x == 0) *P(W, 2, b, 0) = s;
}

__global__ void __launch_bounds__(NT) lz_start2(LzArgs a) {
  pdl_enter();
  __shared__ zc h[1];
  const int r = blockIdx.y, b = blockIdx.x;
  const SiteDev* sdr = a.sd + (long long)r * a.N_sites;
  const WorkDev& W = a.wk[r];
  const VecGeom g = geom(vec_len(sdr, a.site, a.kind), b, a.bcap);
  if (b >= g.nblk) return;
  reduce_partials(W, 2, g.nblk, 0, h);
  const double nrm = sqrt(h[0].x);
  const double inv = nrm > 0 ? 1.0 / nrm : 0.0;
  const zc* src = src_ptr(W, sdr, a.site, a.src);
  for (long long e = g.c0 + threadIdx.x; e < g.c1; e += NT) {
    const zc v = zscale(src[e], inv);
    W.V[e] = v;
    W.x[e] = v;
    if (a.pack_pm >= 0) pack_krylov(a, sdr, W, e, v);
  }
  if (b == 0 && threadIdx.x == 0) {
    W.lzc[0] = 0u;          // last-block counter and barrier word of the fused iteration kernel
    W.lzc[1] = 0u;
    KState* ks = W.ks;
    ks->nrm = nrm;
    ks->k = 0;
    ks->n = (int)g.n;
    ks->kcap = (int)(g.n < a.kmax ? g.n : a.kmax);
    ks->notconv = 0;
    ks->err = 0;
    ks->jcur = 0;
    const bool bad = !isfinite(nrm);
    ks->status = bad ? -6 : 0;
    ks->done = (nrm == 0.0 || bad) ? 1 : 0;
    // a zero start vector is finished at k = 0 (the result is zero); a non-finite one is an error
    if (bad) {
      a.flags[r] = -1;
      if (a.devj) atomicExch(W.err, -7);
    } else if (nrm == 0.0) {
      a.flags[r] = TDVP_KFLAG_DONE;
    }
  }
}

__global__ void __launch_bounds__(NT) lz_dots(LzArgs a, int j) {
  pdl_enter();
  __shared__ zc wsum[DOT_G * NT / 32];
  const int r = blockIdx.y, b = blockIdx.x;
  const WorkDev& W = a.wk[r];
  if (W.ks->done) return;
  if (a.devj) j = W.ks->jcur;
  const SiteDev* sdr = a.sd + (long long)r * a.N_sites;
  const VecGeom g = geom(vec_len(sdr, a.site, a.kind), b, a.bcap);
  if (b >= g.nblk) return;
  chunk_dots(W, g, j, 0, b, wsum);
}

__device__ void tri_step(const LzArgs& a, int r, int j, double* sh, zc* c, double* al, double* be,
                         double* betaj_s);

// pass 1 (tab_in = 0, tab_out = 1) or pass 2 (tab_in = 1, norm partials into table 2; the last
// block to finish then takes the tridiagonal step)
__global__ void __launch_bounds__(NT) lz_upd(LzArgs a, int j, int pass) {
  pdl_enter();
  __shared__ double red[2 * NT / 32];
  __shared__ zc wsum[DOT_G * NT / 32];
  __shared__ zc h[TDVP_KMAX_HARD];
  const int r = blockIdx.y, b = blockIdx.x;
  const WorkDev& W = a.wk[r];
  if (W.ks->done) return;
  if (a.devj) j = W.ks->jcur;
  const SiteDev* sdr = a.sd + (long long)r * a.N_sites;
  const VecGeom g = geom(vec_len(sdr, a.site, a.kind), b, a.bcap);
  if (b >= g.nblk) return;
  reduce_partials(W, pass == 1 ? 0 : 1, g.nblk, j, h);
  double nn = 0;
  for (long long e = g.c0 + threadIdx.x; e < g.c1; e += NT) {
    zc we = W.w[e];
    for (int t = 0; t <= j; ++t) we = zfms(h[t], W.V[t * W.ldV + e], we);
    W.w[e] = we;
    nn += zabs2(we);
  }
  if (pass == 1) {
    __syncthreads();
    chunk_dots(W, g, j, 1, b, wsum);
    if (b == 0 && threadIdx.x == 0) W.ks->alpha[j] = h[j].x;
  } else {
    const zc s = block_zsum(zmake(nn, 0), red);
    if (threadIdx.x == 0) *P(W, 2, b, 0) = s;
    if (b == 0 && threadIdx.x == 0) W.ks->alpha[j] += h[j].x;
    // the last block of this realisation to finish takes the tridiagonal step
    __shared__ int last;
    __shared__ double sh[TRI_SH];
    __shared__ zc c[TRI_THREADS];
    __shared__ double al[TDVP_KMAX_HARD], be[TDVP_KMAX_HARD], betaj_s;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned old = atomicAdd(W.lzc, 1u);
      last = old == (unsigned)(g.nblk - 1);
      if (last) *W.lzc = 0u;     // every block of this realisation has arrived: reset for the next pass
    }
    __syncthreads();
    if (last) {
      __threadfence();
      tri_step(a, r, j, sh, c, al, be, &betaj_s);
    }
  }
}

// Bessel functions J_0..J_N at x >= 0 by Miller's downward recurrence J_{n-1} = (2n/x) J_n - J_{n+1},
// normalised with J_0 + 2 sum_{k>=1} J_{2k} = 1.  Single thread.
__device__ void bessel_j(double x, int N, double* J) {
  for (int n = 0; n <= N; ++n) J[n] = 0.0;
  if (x < 1e-14) { J[0] = 1.0; return; }
  int m = N + 24 + (int)x;
  m += (m & 1);
  double jp1 = 0.0, jn = 1e-200, S = 2.0 * jn;   // m even: contributes 2 J_m
  for (int n = m; n >= 1; --n) {
    const double jm1 = (2.0 * n / x) * jn - jp1;
    jp1 = jn;
    jn = jm1;
    const int idx = n - 1;
    if (idx <= N) J[idx] = jn;
    if ((idx & 1) == 0) S += (idx == 0 ? 1.0 : 2.0) * jn;
    if (fabs(jn) > 1e150) {
      jn *= 1e-150; jp1 *= 1e-150; S *= 1e-150;
      for (int q = idx; q <= N; ++q) J[q] *= 1e-150;
    }
  }
  const double inv = 1.0 / S;
  for (int n = 0; n <= N; ++n) J[n] *= inv;
}


// The same values by every thread of the block: the recurrence factors 2n/x are computed in
// parallel, thread 0 runs the recurrence (one fused multiply-add per step, the overflow guard every
// 8 steps), and the normalisation sum and scaling are block reductions.  Needs m = N + 25 + x + 1
// <= BESSEL_CAP; `cf`, `raw`: BESSEL_CAP doubles each, `red`: one double per warp.
__device__ void bessel_block(double x, int N, double* J, double* cf, double* raw, double* red) {
  const int t = threadIdx.x;
  int m = N + 24 + (int)x;
  m += (m & 1);
  const double ix = 1.0 / x;
  for (int n = t + 1; n <= m; n += blockDim.x) cf[n] = (2.0 * n) * ix;
  __syncthreads();
  if (t == 0) {
    double jp1 = 0.0, jn = 1e-200;
    raw[m] = jn;
    for (int n = m; n >= 1; --n) {
      const double jm1 = fma(cf[n], jn, -jp1);
      jp1 = jn;
      jn = jm1;
      raw[n - 1] = jn;
      if ((n & 7) == 0 && fabs(jn) > 1e140) {
        jn *= 1e-150; jp1 *= 1e-150;
        for (int q2 = n - 1; q2 <= m; ++q2) raw[q2] *= 1e-150;
      }
    }
  }
  __syncthreads();
  // S = raw_0 + 2 sum_{k >= 1} raw_{2k}
  double s = 0.0;
  for (int n = 2 * (t + 1); n <= m; n += 2 * blockDim.x) s += raw[n];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (t % 32 == 0) red[t / 32] = s;
  __syncthreads();
  double S = 0.0;
  for (int w = 0; w < (int)blockDim.x / 32; ++w) S += red[w];
  S = raw[0] + 2.0 * S;
  const double inv = 1.0 / S;
  for (int n = t; n <= N; n += blockDim.x) J[n] = raw[n] * inv;
  __syncthreads();
}

// c = exp(i theta T) e_1 for T = tridiag(beta[0..k-2], alpha[0..k-1]) by a Chebyshev expansion on
// the Gershgorin interval [lo, hi]: exp(i x T~) = sum_n (2 - delta_n0) i^n J_n(x) T_n(T~)
// (Jacobi-Anger), T~ = (T - c0)/h, x = theta h.  The vectors T_n(T~) e_1 are real.
// Thread t (< k) owns component t.  Returns false when |x| needs more than CHEB_MAX_SUB substeps.
__device__ bool tridiag_expi(const double* alpha, const double* beta, int k, double theta, zc* out,
                             double* sh /* >= TRI_SH doubles */) {
  const int t = threadIdx.x;
  double* vcur = sh;                       // [TRI_THREADS]
  double* J = sh + TRI_THREADS;            // [MAX_CHEB]
  double* red = J + MAX_CHEB;              // [2 per warp]
  double* bnd = red + 2 * (TRI_THREADS / 32);   // lo, hi
  // Gershgorin bounds
  double lo = 1e300, hi = -1e300;
  double at = 0, bl = 0, br = 0;
  if (t < k) {
    at = alpha[t];
    bl = t > 0 ? beta[t - 1] : 0.0;
    br = t < k - 1 ? beta[t] : 0.0;
    const double rad = fabs(bl) + fabs(br);
    lo = at - rad;
    hi = at + rad;
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if (t % 32 == 0) { red[2 * (t / 32)] = lo; red[2 * (t / 32) + 1] = hi; }
  __syncthreads();
  if (t == 0) {
    double l = red[0], h2 = red[1];
    for (int w = 1; w < TRI_THREADS / 32; ++w) { l = fmin(l, red[2 * w]); h2 = fmax(h2, red[2 * w + 1]); }
    bnd[0] = l; bnd[1] = h2;
  }
  __syncthreads();
  const double c0 = 0.5 * (bnd[0] + bnd[1]);
  const double h = 0.5 * (bnd[1] - bnd[0]);
  double sr, cr;
  sincos(theta * c0, &sr, &cr);
  const zc ph = zmake(cr, sr);                  // exp(i theta c0)
  const double x = theta * h;
  if (h <= 0.0 || fabs(x) < 1e-14) {           // T is a multiple of the identity
    if (t < k) out[t] = t == 0 ? ph : zmake(0, 0);
    __syncthreads();
    return true;
  }
  // exp(i x T~) = (exp(i (x/s) T~))^s: s = 1 unless one series would need more than MAX_CHEB terms
  const int nsub = (int)ceil(fabs(x) / CHEB_XSUB);
  if (nsub > CHEB_MAX_SUB) return false;
  const int s = nsub < 1 ? 1 : nsub;
  const double ax = fabs(x) / s;
  const int N = cheb_terms(ax);
  double* cfb = bnd + 8;
  {
    double* raw = cfb + BESSEL_CAP;
    const int mneed = N + 24 + (int)ax + 2;
    if (mneed + 1 <= BESSEL_CAP) {
      bessel_block(ax, N, J, cfb, raw, red);
    } else {
      if (t == 0) bessel_j(ax, N, J);
      __syncthreads();
    }
  }
  const double sgn = x >= 0 ? 1.0 : -1.0;      // J_n(-a) = (-1)^n J_n(a)
  const double ih = 1.0 / h;
  int Nlast = N;
  while (Nlast > 2 && fabs(J[Nlast]) < 1e-18 && fabs(J[Nlast - 1]) < 1e-18) --Nlast;
  if (s > 1) {
    // s substeps on a complex vector u (u = e_1, then the previous substep's result): the same
    // three-term recurrence on the real and imaginary parts, coefficients i^n (2 - delta) J_n
    double* vr = vcur;
    double* vi = cfb;                         // Bessel scratch, free again (>= TRI_THREADS doubles)
    double ur = (t == 0) ? 1.0 : 0.0, ui = 0.0;
    for (int q = 0; q < s; ++q) {
      vr[t] = ur; vi[t] = ui;
      __syncthreads();
      double pr = ur, pi = ui, cr = 0.0, ci = 0.0;
      if (t < k) {
        const double lr = t > 0 ? vr[t - 1] : 0.0, rr = t < k - 1 ? vr[t + 1] : 0.0;
        const double li = t > 0 ? vi[t - 1] : 0.0, ri = t < k - 1 ? vi[t + 1] : 0.0;
        cr = ((at - c0) * pr + bl * lr + br * rr) * ih;
        ci = ((at - c0) * pi + bl * li + br * ri) * ih;
      }
      const double cf1 = 2.0 * J[1] * sgn;
      double ar = J[0] * pr - cf1 * ci, ai = J[0] * pi + cf1 * cr;
      __syncthreads();
      vr[t] = cr; vi[t] = ci;
      __syncthreads();
      for (int n = 1; n < Nlast; ++n) {
        double nr = 0.0, ni = 0.0;
        if (t < k) {
          const double lr = t > 0 ? vr[t - 1] : 0.0, rr = t < k - 1 ? vr[t + 1] : 0.0;
          const double li = t > 0 ? vi[t - 1] : 0.0, ri = t < k - 1 ? vi[t + 1] : 0.0;
          nr = 2.0 * ((at - c0) * cr + bl * lr + br * rr) * ih - pr;
          ni = 2.0 * ((at - c0) * ci + bl * li + br * ri) * ih - pi;
        }
        const int m = n + 1;
        double cf = 2.0 * J[m];
        if (sgn < 0 && (m & 1)) cf = -cf;
        switch (m & 3) {                      // i^m (nr + i ni)
          case 0: ar += cf * nr; ai += cf * ni; break;
          case 1: ar -= cf * ni; ai += cf * nr; break;
          case 2: ar -= cf * nr; ai -= cf * ni; break;
          default: ar += cf * ni; ai -= cf * nr; break;
        }
        pr = cr; pi = ci; cr = nr; ci = ni;
        __syncthreads();
        vr[t] = nr; vi[t] = ni;
        __syncthreads();
      }
      ur = t < k ? ar : 0.0;
      ui = t < k ? ai : 0.0;
      __syncthreads();
    }
    if (t < k) out[t] = zmul(ph, zmake(ur, ui));
    __syncthreads();
    return true;
  }
  if (k <= 32) {
    // one warp: component t in lane t, neighbours by shuffles, no block barriers in the loop;
    // T_{n+1} e_1 = 2 T~ T_n e_1 - T_{n-1} e_1 with T~ = (T - c0)/h
    if (t < 32) {
      const bool act = t < k;
      const double A = act ? 2.0 * (at - c0) * ih : 0.0;
      const double BL = (act && t > 0) ? 2.0 * bl * ih : 0.0;
      const double BR = (act && t < k - 1) ? 2.0 * br * ih : 0.0;
      double vp = (t == 0) ? 1.0 : 0.0;
      double vc;
      {
        const double left = __shfl_up_sync(0xffffffffu, vp, 1), right = __shfl_down_sync(0xffffffffu, vp, 1);
        vc = 0.5 * fma(A, vp, fma(BL, left, BR * right));
      }
      zc acc = zmake(J[0] * vp, 2.0 * J[1] * sgn * vc);
      for (int n = 1; n < Nlast; ++n) {
        const double left = __shfl_up_sync(0xffffffffu, vc, 1), right = __shfl_down_sync(0xffffffffu, vc, 1);
        const double vn = fma(A, vc, fma(BL, left, fma(BR, right, -vp)));
        const int m = n + 1;
        double cf = 2.0 * J[m];
        if (sgn < 0 && (m & 1)) cf = -cf;
        switch (m & 3) {
          case 0: acc.x = fma(cf, vn, acc.x); break;
          case 1: acc.y = fma(cf, vn, acc.y); break;
          case 2: acc.x = fma(-cf, vn, acc.x); break;
          default: acc.y = fma(-cf, vn, acc.y); break;
        }
        vp = vc;
        vc = vn;
      }
      if (act) out[t] = zmul(ph, acc);
    }
    __syncthreads();
    return true;
  }
  // coefficient of T_n: (2 - delta) i^n J_n(x); i^n cycles 1, i, -1, -i
  double vprev = (t == 0) ? 1.0 : 0.0;          // T_0 e_1
  vcur[t] = vprev;
  __syncthreads();
  double v1 = 0;
  if (t < k) {
    const double left = t > 0 ? vcur[t - 1] : 0.0, right = t < k - 1 ? vcur[t + 1] : 0.0;
    v1 = ((at - c0) * vprev + bl * left + br * right) * ih;   // T_1 e_1
  }
  zc acc = zmake(J[0] * vprev, 0.0);
  {
    const double cf = 2.0 * J[1] * sgn;         // i^1 * sgn
    acc.y += cf * v1;
  }
  __syncthreads();
  vcur[t] = v1;
  double vc = v1;
  __syncthreads();
  for (int n = 1; n < Nlast; ++n) {
    double vn = 0;
    if (t < k) {
      const double left = t > 0 ? vcur[t - 1] : 0.0, right = t < k - 1 ? vcur[t + 1] : 0.0;
      vn = 2.0 * ((at - c0) * vc + bl * left + br * right) * ih - vprev;
    }
    const int m = n + 1;
    double cf = 2.0 * J[m];
    if (sgn < 0 && (m & 1)) cf = -cf;
    switch (m & 3) {
      case 0: acc.x += cf * vn; break;
      case 1: acc.y += cf * vn; break;
      case 2: acc.x -= cf * vn; break;
      default: acc.y -= cf * vn; break;
    }
    vprev = vc;
    vc = vn;
    __syncthreads();
    vcur[t] = vn;
    __syncthreads();
  }
  if (t < k) out[t] = zmul(ph, acc);
  __syncthreads();
  return true;
}

// The tridiagonal step of iteration j of realisation r: beta_j from the norm partials, controller
// features and prediction at j = 0, then (from the first tested k on) exp(i theta T_k) e_1 and the
// a-posteriori test.  Run by the last block of the second orthogonalisation pass to finish; every
// value the other blocks wrote in that kernel is read through L2.  `al`, `be`: KMAX doubles each.
__device__ void tri_step(const LzArgs& a, int r, int j, double* sh, zc* c, double* al, double* be,
                         double* betaj_s) {
  int* flags = a.flags;
  const WorkDev& W = a.wk[r];
  KState* ks = W.ks;
  const SiteDev* sdr = a.sd + (long long)r * a.N_sites;
  const VecGeom g = geom(vec_len(sdr, a.site, a.kind), 0, a.bcap);
  if (threadIdx.x < 32) {
    double s = 0;
    for (int b = threadIdx.x; b < g.nblk; b += 32) s += __ldcg(&P(W, 2, b, 0)->x);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *betaj_s = sqrt(s);
  }
  for (int t = threadIdx.x; t <= j; t += blockDim.x) {
    al[t] = __ldcg(&ks->alpha[t]);
    if (t < j) be[t] = __ldcg(&ks->beta[t]);
  }
  __syncthreads();
  const double beta = *betaj_s;
  const int k = j + 1;
  if (!isfinite(beta) || !isfinite(al[j])) {

    if (threadIdx.x == 0) {
      ks->status = -6; ks->done = 1; ks->k = 0; flags[r] = -1;
      if (a.devj) atomicExch(W.err, -7);
    }
    return;
  }
  const bool last = (k >= ks->kcap) || beta == 0.0;
  if (j == 0) {
    // controller features, known after the first Lanczos step
    if (threadIdx.x == 0) {
      const double th = fabs(a.theta), a0 = al[0];
      const double hn = sqrt(a0 * a0 + beta * beta);
      ks->feat[0] = (float)log10(1.0 + th * hn);
      ks->feat[1] = (float)a.kind;
      ks->feat[2] = (float)W.kprev[2 * a.site + a.kind] / 32.f;
      ks->feat[3] = (float)a.site / (float)(a.N_sites > 1 ? a.N_sites - 1 : 1);
      ks->feat[4] = (float)(log2((double)g.n) / 20.0);
      ks->feat[5] = (float)(log10(th + 1e-30) / 4.0);
      ks->feat[6] = (float)(-log10(a.tol + 1e-300) / 12.0);
      ks->feat[7] = (float)log10(1.0 + th * fabs(a0));
      ks->kpred = 0;
    }
    __syncthreads();
    if (a.mlp) {
      float za;
      const float y = mlp_infer(ks->feat, a.mlp, reinterpret_cast<float*>(sh), &za);
      if (threadIdx.x == 0) {
        // the dimension the controller predicts.  An iteration past the converged dimension costs
        // a whole matvec, a failed test only a tridiagonal exponential, so when the acceptance
        // head predicts that the test at kp passes (the solve may have converged earlier) the
        // first test is made one dimension before kp
        int kp = (int)fminf(fmaxf(floorf(y), 1.f), 126.f);
        if (za >= 0.f && kp > 1) kp -= 1;
        ks->kpred = kp;
      }
      __syncthreads();
    }
  }
  // a.jcheck = 0: from the previous Krylov dimension of this (site, kind) minus 2 (device-driven
  // loops; the host-driven loop passes the same rule evaluated on the host)
  const int jcheck = a.mlp ? max(1, ks->kpred)
                           : (a.jcheck > 0 ? a.jcheck : max(1, W.kprev[2 * a.site + a.kind] - 2));
  if (k < jcheck && !last) {
    if (threadIdx.x == 0) { ks->beta[j] = beta; ks->inv_beta = 1.0 / beta; }
    return;
  }
  if (threadIdx.x == 0) (*W.tri_count)++;
  const bool ok = tridiag_expi(al, be, k, a.theta, c, sh);
  if (!ok) {
    if (threadIdx.x == 0) {
      ks->status = -1; ks->done = 1; ks->k = 0; flags[r] = -1;
      if (a.devj) atomicExch(W.err, -7);
    }
    return;
  }
  const double err = ks->nrm * beta * sqrt(zabs2(c[k - 1]));
  const bool conv = err <= a.tol;
  if (conv || last) {
    if (threadIdx.x < k) ks->coef[threadIdx.x] = zscale(c[threadIdx.x], ks->nrm);
    if (threadIdx.x == 0) {
      ks->err = err;
      ks->k = k;
      ks->notconv = (!conv && beta > 0.0) ? 1 : 0;
      ks->done = 1;
      flags[r] = k | (ks->notconv << 16) | TDVP_KFLAG_DONE;
      W.kprev[2 * a.site + a.kind] = k;
      if (a.devj) {
        ks->dim_sum += k;
        ks->dim_max = max(ks->dim_max, k);
        ks->solves += 1;
        ks->nc_count += ks->notconv;
      }
      if (a.log) {
        const unsigned slot = atomicAdd(a.log_count, 1u);
        if ((long long)slot < a.log_cap) {
          for (int q = 0; q < MLP_NIN; ++q) a.log[(long long)slot * (MLP_NIN + 1) + q] = ks->feat[q];
          a.log[(long long)slot * (MLP_NIN + 1) + MLP_NIN] = (float)k;
        }
      }
    }
  } else if (threadIdx.x == 0) {
    ks->err = err;
    ks->beta[j] = beta;
    ks->inv_beta = 1.0 / beta;
  }
}

__global__ void __launch_bounds__(NT) lz_next(LzArgs a, int j) {
  pdl_enter();
  const int r = blockIdx.y, b = blockIdx.x;
  const WorkDev& W = a.wk[r];
  if (W.ks->done) return;
  if (a.devj) j = W.ks->jcur;
  const SiteDev* sdr = a.sd + (long long)r * a.N_sites;
  const VecGeom g = geom(vec_len(sdr, a.site, a.kind), b, a.bcap);
  if (b >= g.nblk) return;
  const double ib = W.ks->inv_beta;
  zc* Vn = W.V + (j + 1) * W.ldV;
  for (long long e = g.c0 + threadIdx.x; e < g.c1; e += NT) {
    const zc v = zscale(W.w[e], ib);
    Vn[e] = v;
    W.x[e] = v;
    if (a.pack_pm >= 0) pack_krylov(a, sdr, W, e, v);
  }
}

__device__ __forceinline__ unsigned long long lz_gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded barrier over the nblocks blocks of one realisation on the word W.lzc[1], whose low 31
// bits are zero between barriers: block 0 adds 2^31 - (nblocks - 1), every other block 1, so the
// top bit flips exactly when the last block arrives; a block waits until the top bit differs from
// the value it read at its arrival.  Gives up after wait_ns of wall-clock time (1 s unless a test
// shortens it; error word -5, TDVP_ERR_DEVICE_TIMEOUT) or when another block has given up; returns
// false then.
__device__ bool lz_group_sync(const WorkDev& W, int nblocks, int b, unsigned long long wait_ns) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile int* err = W.err;
    int good = (*err == 0);
    if (good && nblocks > 1) {
      const unsigned inc = (b == 0) ? (0x80000000u - (unsigned)(nblocks - 1)) : 1u;
      volatile unsigned* word = W.lzc + 1;
      __threadfence();
      const unsigned old = atomicAdd(W.lzc + 1, inc);
      const unsigned long long t0 = lz_gtimer();
      while (((old ^ *word) & 0x80000000u) == 0u) {
        if (*err != 0) { good = 0; break; }
        if (lz_gtimer() - t0 > wait_ns) { atomicExch(W.err, -5); good = 0; break; }
      }
      __threadfence();
    }
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// One Lanczos iteration j in one launch (the grid is cooperative, so the blocks of a realisation
// are co-resident and can wait for each other):
//   1. partial dots p_t = <V_t, w>, t <= j                                   | group barrier
//   2. h1 = sum p; w -= V h1; alpha_j = Re h1_j; partial dots of the second pass | group barrier
//   3. h2 = sum; w -= V h2; alpha_j += Re h2_j; |w|^2 partials; the block that finishes last
//      takes the tridiagonal step (beta_j, exp(i theta T) e_1, convergence)  | group barrier
//   4. unless the solve is done: V_{j+1} = x = w / beta_j (and its packed tensor-core operand)
// The arithmetic and its order are those of lz_dots, lz_upd (both passes) and lz_next.
__global__ void __launch_bounds__(NT) lz_iter(LzArgs a, int j) {
  __shared__ double red[2 * NT / 32];
  __shared__ zc wsum[DOT_G * NT / 32];
  __shared__ zc h[TDVP_KMAX_HARD];
  __shared__ int last;
  __shared__ double sh[TRI_SH];
  __shared__ zc c[TRI_THREADS];
  __shared__ double al[TDVP_KMAX_HARD], be[TDVP_KMAX_HARD], betaj_s;
  pdl_wait();
  const int r = blockIdx.y, b = blockIdx.x;
  const WorkDev& W = a.wk[r];
  if (W.ks->done) return;
  if (a.devj) j = W.ks->jcur;
  const SiteDev* sdr = a.sd + (long long)r * a.N_sites;
  const VecGeom g = geom(vec_len(sdr, a.site, a.kind), b, a.bcap);
  if (b >= g.nblk) return;
  chunk_dots(W, g, j, 0, b, wsum);
  // failure-path test: the first barrier counts one block more than the launch has, a participant
  // that never arrives, so every block's bounded wait runs out
  if (!lz_group_sync(W, a.stall ? g.nblk + 1 : g.nblk, b, a.wait_ns)) return;
  // first Gram-Schmidt pass
  reduce_partials(W, 0, g.nblk, j, h);
  for (long long e = g.c0 + threadIdx.x; e < g.c1; e += NT) {
    zc we = W.w[e];
    for (int t = 0; t <= j; ++t) we = zfms(h[t], W.V[t * W.ldV + e], we);
    W.w[e] = we;
  }
  __syncthreads();
  chunk_dots(W, g, j, 1, b, wsum);
  if (b == 0 && threadIdx.x == 0) W.ks->alpha[j] = h[j].x;
  if (!lz_group_sync(W, g.nblk, b, a.wait_ns)) return;
  // second pass and the norm partials
  reduce_partials(W, 1, g.nblk, j, h);
  double nn = 0;
  for (long long e = g.c0 + threadIdx.x; e < g.c1; e += NT) {
    zc we = W.w[e];
    for (int t = 0; t <= j; ++t) we = zfms(h[t], W.V[t * W.ldV + e], we);
    W.w[e] = we;
    nn += zabs2(we);
  }
  const zc s = block_zsum(zmake(nn, 0), red);
  if (threadIdx.x == 0) *P(W, 2, b, 0) = s;
  if (b == 0 && threadIdx.x == 0) W.ks->alpha[j] += h[j].x;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned old = atomicAdd(W.lzc, 1u);
    last = old == (unsigned)(g.nblk - 1);
    if (last) W.lzc[0] = 0u;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    tri_step(a, r, j, sh, c, al, be, &betaj_s);
  }
  if (!lz_group_sync(W, g.nblk, b, a.wait_ns)) return;
  // next Krylov vector (values of the tridiagonal step read through L2)
  KState* ks = W.ks;
  if (__ldcg(&ks->done)) return;
  const double ib = __ldcg(&ks->inv_beta);
  zc* Vn = W.V + (j + 1) * W.ldV;
  for (long long e = g.c0 + threadIdx.x; e < g.c1; e += NT) {
    const zc v = zscale(W.w[e], ib);
    Vn[e] = v;
    W.x[e] = v;
    if (a.pack_pm >= 0) pack_krylov(a, sdr, W, e, v);
  }
}

__global__ void __launch_bounds__(NT) lz_combine(LzArgs a) {
  pdl_enter();
  __shared__ zc cf[TDVP_KMAX_HARD];
  const int r = blockIdx.y, b = blockIdx.x;
  const WorkDev& W = a.wk[r];
  const SiteDev* sdr = a.sd + (long long)r * a.N_sites;
  const VecGeom g = geom(vec_len(sdr, a.site, a.kind), b, a.bcap);
  if (b >= g.nblk) return;
  const int k = W.ks->k;
  for (int t = threadIdx.x; t < k; t += NT) cf[t] = W.ks->coef[t];
  __syncthreads();
  zc* dst = src_ptr(W, sdr, a.site, a.dst);
  for (long long e = g.c0 + threadIdx.x; e < g.c1; e += NT) {
    zc acc = zmake(0, 0);
    for (int t = 0; t < k; ++t) acc = zfma(cf[t], W.V[t * W.ldV + e], acc);
    dst[e] = acc;
  }
}

// Loop control of a device-driven solve (one warp).  The body's kernels have all finished when
// this runs (graph dependency), so every unfinished solve's iteration index can advance.
__global__ void lz_loop_ctl(LzArgs a, int which) {
  pdl_enter();
  int active = 0;
  for (int r = threadIdx.x; r < a.R; r += 32) {
    KState* ks = a.wk[r].ks;
    if (!ks->done) {
      if (which == 1) ks->jcur += 1;
      if (ks->jcur >= a.kmax) {
        // cannot happen while the tridiagonal kernel stops every solve at its cap; it bounds the
        // device loop even so
        ks->done = 1;
        atomicCAS(a.wk[r].err, 0, -7);    // an earlier error (e.g. a timed-out wait) stays reported
      } else {
        active = 1;
      }
    }
  }
  active = __any_sync(0xffffffffu, active);
  if (threadIdx.x == 0) {
    if (which == 1 && a.loop_iters) a.loop_iters[a.loop_id] += 1u;
    cudaGraphSetConditional(a.cond, active ? 1u : 0u);
  }
}

}  // namespace

cudaError_t launch_lz_loop_ctl(const LzArgs& a, int which, cudaStream_t st) {
  { const cudaError_t e_ = launch_pdl(lz_loop_ctl, 1, 32, 0, st, a, which); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

cudaError_t launch_lz_start(const LzArgs& a, cudaStream_t st) {
  dim3 grid(a.nblk, a.R);
  { const cudaError_t e_ = launch_pdl(lz_start1, grid, NT, 0, st, a); if (e_ != cudaSuccess) return e_; }
  { const cudaError_t e_ = launch_pdl(lz_start2, grid, NT, 0, st, a); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

cudaError_t launch_lz_iter_pre(const LzArgs& a, int j, cudaStream_t st) {
  dim3 grid(a.nblk, a.R);
  { const cudaError_t e_ = launch_pdl(lz_dots, grid, NT, 0, st, a, j); if (e_ != cudaSuccess) return e_; }
  { const cudaError_t e_ = launch_pdl(lz_upd, grid, NT, 0, st, a, j, 1); if (e_ != cudaSuccess) return e_; }
  { const cudaError_t e_ = launch_pdl(lz_upd, grid, NT, 0, st, a, j, 2); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

cudaError_t launch_lz_iter_post(const LzArgs& a, int j, cudaStream_t st) {
  dim3 grid(a.nblk, a.R);
  { const cudaError_t e_ = launch_pdl(lz_next, grid, NT, 0, st, a, j); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

cudaError_t launch_lz_iter(const LzArgs& a, int j, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.gridDim = dim3(a.nblk, a.R);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, lz_iter, a, j);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// co-resident blocks of lz_iter on the whole device (0 if the query fails)
int lz_iter_capacity(int device) {
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lz_iter, NT, 0) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
  return per_sm * sms;
}

cudaError_t launch_lz_combine(const LzArgs& a, cudaStream_t st) {
  dim3 grid(a.nblk, a.R);
  { const cudaError_t e_ = launch_pdl(lz_combine, grid, NT, 0, st, a); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}
