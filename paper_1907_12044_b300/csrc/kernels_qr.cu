// Gauge-shift decomposition of Eq. QR (and its mirror "RQ"/LQ) on the device, FP64.
//
// The matrix is handled as X (n rows x m columns, row-major, n <= m): X = Rc * Qr with Qr having
// orthonormal rows and Rc lower triangular.  For the left-to-right shift X is the transpose of
// the site tensor C[(l s), r], so Q = Qr^T and R = Rc^T; for the right-to-left shift X is
// C[l, (s r)] itself.
//
// Definition followed (the same as the CPU oracle's): rows are orthogonalised in order by
// classical Gram-Schmidt with one re-orthogonalisation pass; a row whose residual is
// <= rtol*||X||_F is linearly dependent, gets a zero diagonal entry, and is replaced by the first
// unit vector e_p at distance >= 1/2 from the rows so far (1 - sum_t |Qr[t][p]|^2 >= 1/4), else
// the farthest one, orthogonalised with the same two passes.
//
// Blocked evaluation: rows are taken in panels of PB = 8.  A panel is projected twice against all
// earlier rows (block classical Gram-Schmidt), then orthonormalised inside the panel by two
// Cholesky-QR passes on its PB x PB Gram matrix.  In exact arithmetic this gives the same Q and
// R as the row-by-row process.  When the first Gram matrix shows a row whose squared residual is
// below 1e-10 of its squared norm (where Cholesky-QR loses accuracy) or below 100 rtol^2
// ||X||_F^2 (near the rank decision), the panel is redone row by row with the exact rule.  Above
// both bounds the pivot's rounding error, O(n eps) of the row's squared norm, is below 1e-4 of the
// pivot itself, so the pivot cannot be on the other side of rtol^2 ||X||_F^2 from the exact
// residual.
//
// One realisation is processed by B co-resident blocks (cooperative launch).  Dot products over
// whole rows are spread over all warps of all blocks; updates are done by the block that owns a
// slab of columns.  Phases are separated by a group barrier whose wait is bounded: after ~1 s it
// records TDVP_ERR_DEVICE_TIMEOUT in the realisation's error word and every block returns.
#include "tdvp_internal.cuh"

namespace {

constexpr int QT = TDVP_QR_THREADS;       // 256 threads = 8 warps
constexpr int NW = QT / 32;
constexpr int QR_NMAX = 256;              // largest n (bond dimension) handled
constexpr int PB = 8;                     // panel height
constexpr unsigned long long WAIT_NS = 1000000000ull;   // a barrier wait gives up after 1 s

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

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
  } else if (dir == 3) {          // right-to-left shape on the scratch buffer (autotuning)
    const SiteDev& s = sdr[site];
    J.X = W.scratch; J.n = s.Dl; J.m = s.d * s.Dr; J.Rout = W.bond; J.rtrans = 0;
  } else {
    J.X = W.scratch; J.n = dn; J.m = dm; J.Rout = W.bond; J.rtrans = 1;
  }
  return J;
}

// Bounded barrier over the B blocks of one realisation.  One atomic per block on one word: every
// block adds 1 except block 0, which adds 2^31 - (B-1), so the word's top bit flips exactly once
// per barrier; a block waits until the top bit differs from the value it read at its arrival.
// The wait gives up after 1 s (TDVP_ERR_DEVICE_TIMEOUT).  Returns false if this or an earlier
// wait gave up.
__device__ bool group_sync(const WorkDev& W, int nblocks) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile int* err = W.err;
    int good = (*err == 0);
    if (good && nblocks > 1) {
      const unsigned inc = (blockIdx.x % nblocks == 0) ? (0x80000000u - (unsigned)(nblocks - 1)) : 1u;
      volatile unsigned* word = W.bar;
      __threadfence();
      const unsigned old = atomicAdd(W.bar, inc);
      const unsigned long long t0 = gtimer();
      while (((old ^ *word) & 0x80000000u) == 0u) {
        if (*err != 0) { good = 0; break; }
        if (gtimer() - t0 > WAIT_NS) { atomicExch(W.err, -5); good = 0; break; }
      }
      __threadfence();
    }
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// sum_c conj(b[c]) a[c] over the whole row by one warp (rows may be written by other blocks).
// Four independent accumulators keep eight L2 loads per lane in flight.
__device__ __forceinline__ zc warp_dot(const zc* a, const zc* b, int m) {
  const int lane = threadIdx.x % 32;
  zc s0 = zmake(0, 0), s1 = s0, s2 = s0, s3 = s0;
  int c = lane;
  for (; c + 96 < m; c += 128) {
    const zc b0 = __ldcg(b + c), a0 = __ldcg(a + c);
    const zc b1 = __ldcg(b + c + 32), a1 = __ldcg(a + c + 32);
    const zc b2 = __ldcg(b + c + 64), a2 = __ldcg(a + c + 64);
    const zc b3 = __ldcg(b + c + 96), a3 = __ldcg(a + c + 96);
    s0 = zcfma(b0, a0, s0);
    s1 = zcfma(b1, a1, s1);
    s2 = zcfma(b2, a2, s2);
    s3 = zcfma(b3, a3, s3);
  }
  for (; c < m; c += 32) s0 = zcfma(__ldcg(b + c), __ldcg(a + c), s0);
  zc s = zadd(zadd(s0, s1), zadd(s2, s3));
  for (int o = 16; o > 0; o >>= 1) {
    s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
    s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
  }
  return s;
}

// Row dot products sum_c conj(X_t[c]) x[c] for t < j into out[t].  With fewer products than
// blocks each block takes whole products with all its warps splitting the row (one L2 round
// trip per lane, shared-memory combine); otherwise one warp per product.
__device__ void row_dots(const zc* X, int m, const zc* x, int j, zc* out, int b, int B, int gw, int nwarps, zc* sbuf) {
  const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
  if (j <= B) {
    for (int t = b; t < j; t += B) {
      const zc* q = X + (long long)t * m;
      zc s = zmake(0, 0);
      for (int c = threadIdx.x; c < m; c += QT) s = zcfma(__ldcg(q + c), __ldcg(x + c), s);
      for (int o = 16; o > 0; o >>= 1) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
      }
      __syncthreads();
      if (lane == 0) sbuf[wid] = s;
      __syncthreads();
      if (threadIdx.x == 0) {
        zc tot = sbuf[0];
        for (int w = 1; w < NW; ++w) tot = zadd(tot, sbuf[w]);
        out[t] = tot;
      }
    }
  } else {
    for (int t = gw; t < j; t += nwarps) {
      const zc s = warp_dot(x, X + (long long)t * m, m);
      if (lane == 0) out[t] = s;
    }
  }
}

// X[row0 + r][c] -= sum_{t<T} Hs[r*ldh + t] * X[t][c] for r < nb and c in the slab [c0, c1).
// Several threads share an element and split the t sum; their partial sums are combined by a
// fixed shuffle tree, so results do not depend on scheduling.
__device__ void slab_update(zc* X, int m, int row0, int nb, int T, const zc* Hs, int ldh, int c0, int c1) {
  const int cs = c1 - c0;
  const int E = nb * cs;
  if (E <= 0 || T <= 0) return;
  int tpe = 1;
  while (tpe * 2 <= 32 && tpe * 2 * E <= QT && tpe * 2 <= T) tpe *= 2;
  const int total = E * tpe;
  for (int base = 0; base < total; base += QT) {
    const int idx = base + threadIdx.x;
    const bool active = idx < total;
    const int e = idx / tpe, sub = idx % tpe;
    zc acc = zmake(0, 0);
    int r = 0, c = 0;
    if (active) {
      r = e / cs;
      c = c0 + e % cs;
      zc a1 = zmake(0, 0), a2 = a1, a3 = a1;
      int t = sub;
      for (; t + 3 * tpe < T; t += 4 * tpe) {
        const zc x0 = X[(long long)t * m + c], x1 = X[(long long)(t + tpe) * m + c];
        const zc x2 = X[(long long)(t + 2 * tpe) * m + c], x3 = X[(long long)(t + 3 * tpe) * m + c];
        acc = zfma(Hs[r * ldh + t], x0, acc);
        a1 = zfma(Hs[r * ldh + t + tpe], x1, a1);
        a2 = zfma(Hs[r * ldh + t + 2 * tpe], x2, a2);
        a3 = zfma(Hs[r * ldh + t + 3 * tpe], x3, a3);
      }
      for (; t < T; t += tpe) acc = zfma(Hs[r * ldh + t], X[(long long)t * m + c], acc);
      acc = zadd(zadd(acc, a1), zadd(a2, a3));
    }
    for (int o = tpe / 2; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (active && sub == 0) {
      zc* p = X + (long long)(row0 + r) * m + c;
      *p = zsub(*p, acc);
    }
  }
  __syncthreads();
}

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = v;
  __syncthreads();
  double t = 0;
  for (int w = 0; w < NW; ++w) t += red[w];
  return t;
}

// 1/sqrt(s) for s in [2^-100, 2^100]: the FP32 estimate refined by two Newton steps
// y <- y (3 - s y^2) / 2 (each squares the relative error), about 8 FP64 instructions instead of an
// FP64 square root and division, which matter on a serial chain where every FP64 instruction of a
// lone warp costs tens of cycles
__device__ __forceinline__ double rsqrt_nr(double s) {
  double y = (double)rsqrtf((float)s);
  y = y * fma(-0.5 * s * y, y, 1.5);
  y = y * fma(-0.5 * s * y, y, 1.5);
  return y;
}

// fixed-order sum of one double per block (every block gets the same value)
__device__ double sum_over_blocks(const zc* P, int B) {
  const int lane = threadIdx.x % 32;
  double s = 0;
  for (int b = lane; b < B; b += 32) s += __ldcg(P + b).x;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

struct Scratch {
  zc* H1;     // [PB][n]  first-pass coefficients of the panel rows
  zc* H2;     // [PB][n]  second-pass coefficients
  zc* G;      // [PB][PB] Gram matrix
  zc* hv;     // [2n]     coefficients of the row-by-row path
  zc* Pn;     // [2B]     per-block scalars
  zc* Pc;     // [2B]     per-block completion candidates
};

// ---- rank-deficient tail ----
// Taken after a dropped row j.  With Q_t (t < J0 = j+1) final, rows J0..n-1 are projected twice
// onto them (block Gram-Schmidt); a row whose residual is <= max(thresh/2, thresh - 1e-8 ||X||_F)
// is dropped under the exact rule as well, since the exact process tests it against a superset
// of these Q_t (residuals only shrink) and the two computed residuals differ by rounding only:
// each is within ~2 n m eps ||x|| of its exact value (n dot products of length m, two passes),
// together < 2e-9 ||x|| <= 1e-8 ||X||_F for n <= 256, m <= 16384.  The completions are then built one per group barrier:
// rows are kept unnormalised with their squared norms (so no row another block reads is
// rewritten) and every block picks the next unit vector itself, scanning forward from the
// previous one.  A completion is e_p minus its projection with the exact
// first-pass coefficients conj(Q_t[p]); being at distance >= 1/2 from the span (or the farthest
// unit vector), one pass leaves it orthogonal to O(eps).  Finally rows are normalised and the
// R coefficients of the dropped rows against the completions are taken from the backed-up rows.
// Only the prefix of rows that are certainly dropped is finished this way (a later row may
// be kept); the rows after it are restored and return to the row path.  Returns the number of
// rows finished (0: none, rows restored), -1 when a group barrier gave up.

constexpr int TAIL_KB = 8;   // completions per group barrier in the tail

__device__ int qr_tail(const QrJob& J, const WorkDev& W, const Scratch& S, int J0, int j0, int pend, int b, int B,
                       int gw, int nwarps, int c0, int c1, double thresh, double fro, zc* Hs, double* red,
                       double* ens, int* flag) {
  __shared__ zc Gb[TAIL_KB][TAIL_KB], Lb[TAIL_KB][TAIL_KB], Li[TAIL_KB][TAIL_KB];
  __shared__ double Ldi[TAIL_KB];                       // 1 / L_kk
  __shared__ zc Yb[QT];
  __shared__ int tflag[TAIL_KB + 1];
  const int n = J.n, m = J.m, Tn = n - J0, lane = threadIdx.x % 32;
  zc* X = J.X;
  zc* BK = W.qtail;                                     // [n][m] backup of rows J0..n-1
  zc* HT1 = BK + (long long)n * m;                      // [n][n]
  zc* HT2 = HT1 + (long long)n * n;                     // [n][n]
  double* TPN = reinterpret_cast<double*>(HT2 + (long long)n * n);   // [n][B] residual norms
  for (long long e = threadIdx.x; e < (long long)Tn * (c1 - c0); e += QT) {
    const int j = J0 + (int)(e / (c1 - c0)), c = c0 + (int)(e % (c1 - c0));
    BK[(long long)j * m + c] = X[(long long)j * m + c];
  }
  // two projection passes of rows J0..n-1 onto rows 0..J0-1
  for (int pass = 0; pass < 2; ++pass) {
    zc* HT = pass ? HT2 : HT1;
    for (int e = gw; e < Tn * J0; e += nwarps) {
      const int a = e / J0, t = e % J0;
      const zc s = warp_dot(X + (long long)(J0 + a) * m, X + (long long)t * m, m);
      if (lane == 0) HT[(long long)a * n + t] = s;
    }
    if (!group_sync(W, B)) return -1;
    // all tail rows in one slab pass when their coefficients fit in Hs, else in chunks
    const int chunk = J0 > 0 ? max(1, min(Tn, (PB * QR_NMAX) / J0)) : Tn;
    for (int a0 = 0; a0 < Tn; a0 += chunk) {
      const int nb = min(chunk, Tn - a0);
      if (a0 > 0) __syncthreads();
      for (int e = threadIdx.x; e < nb * J0; e += QT) Hs[e] = __ldcg(HT + (long long)(a0 + e / J0) * n + e % J0);
      __syncthreads();
      slab_update(X, m, J0 + a0, nb, J0, Hs, J0, c0, c1);
    }
    if (pass == 1) {
      // squared residual norms over this block's columns, one warp per row
      for (int a = threadIdx.x / 32; a < Tn; a += NW) {
        double s = 0;
        for (int c = c0 + lane; c < c1; c += 32) s += zabs2(X[(long long)(J0 + a) * m + c]);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) TPN[(long long)a * B + b] = s;
      }
    }
    if (!group_sync(W, B)) return -1;
  }
  // rows certainly dropped: the prefix of rows whose residual is <= thresh/2 (the same sums in
  // the same order in every block); later rows go back to the exact row path
  int Tc;
  {
    __shared__ int first_bad;
    if (threadIdx.x == 0) first_bad = Tn;
    __syncthreads();
    // certain-drop bound (squared), the same in every block: fro = ||X||_F
    const double lim = fmax(0.5 * thresh, thresh - 1e-8 * fro), lim2 = lim * lim;
    for (int a = threadIdx.x / 32; a < Tn; a += NW) {
      double s = 0;
      for (int bb = lane; bb < B; bb += 32) s += __ldcg(TPN + (long long)a * B + bb);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0 && !(s <= lim2)) atomicMin(&first_bad, a);
    }
    __syncthreads();
    Tc = first_bad;
    __syncthreads();
    if (Tc == 0) {
      for (long long e = threadIdx.x; e < (long long)Tn * (c1 - c0); e += QT) {
        const int j = J0 + (int)(e / (c1 - c0)), c = c0 + (int)(e % (c1 - c0));
        X[(long long)j * m + c] = BK[(long long)j * m + c];
      }
      return group_sync(W, B) ? 0 : -1;
    }
  }
  // completions, one group barrier each.  The first qualifying column only moves forward: a
  // column at distance < 1/2 stays so (the sums only grow) and a completed column drops to
  // distance 0, so the scan resumes after the previous choice, one warp per candidate column.
  // A warp loads its column of every earlier row in one round of loads, together with the
  // previous row's norm partials: the same values give the column's distance and, scaled, the
  // projection coefficients conj(Q_t[p]) if it is chosen.  Only when no column ahead qualifies
  // are all columns searched for the farthest one.
  const int wid = threadIdx.x / 32;
  int pnext = 0;
  int a = 0;
  bool prev_single = false;   // the previous row is a single completion whose norm is pending
  while (true) {
    const int j = J0 + a;
    // 1 / squared norm of a pending single completion (row j - 1), from its norm partials
    double einv_prev = 0.0;
    if (prev_single) {
      const double en2 = sum_over_blocks(S.Pn + ((a - 1) & 1) * B, B);
      einv_prev = en2 > 0.0 ? 1.0 / en2 : 0.0;
      if (threadIdx.x == 0) { ens[a - 1] = en2; ens[QR_NMAX + a - 1] = einv_prev; }
    }
    if (a >= Tc) break;
    // coefficient scale of row t: 1 for rows < J0 and batch completions (normalised),
    // 1/|x_t|^2 for single completions (stored unnormalised)
    auto scale = [&](int t) -> double {
      return t < J0 ? 1.0 : ((prev_single && t == j - 1) ? einv_prev : ens[QR_NMAX + t - J0]);
    };
    // squared norm of stored row t (1 for normalised rows)
    auto rnorm2 = [&](int t) -> double {
      return t < J0 ? 1.0 : ((prev_single && t == j - 1) ? 1.0 / einv_prev : ens[t - J0]);
    };
    const int ldc = j;
    int KB = min(TAIL_KB, Tc - a);
    if ((NW + KB) * ldc > PB * QR_NMAX) KB = max(1, (PB * QR_NMAX) / ldc - NW);
    if ((NW + KB) * ldc > PB * QR_NMAX) KB = 0;
    zc* cv = Hs;                    // [NW][ldc] this round's candidate columns, as coefficients
    zc* bslot = Hs + NW * ldc;      // [KB][ldc] accepted candidates, in column order
    // scan forward for up to max(KB, 1) qualifying columns
    const int want = max(KB, 1);
    int nf = 0, fw0 = -1;
    for (int c0s = pnext; c0s < m && nf < want; c0s += NW) {
      const int c = c0s + wid;
      int ok = 0;
      if (c < m) {
        double s = 0;
        for (int t = lane; t < j; t += 32) {
          const zc v = __ldcg(X + (long long)t * m + c);
          const double sc = scale(t);
          cv[wid * ldc + t] = zscale(zconj(v), sc);
          if (t >= J0) s += zabs2(v) * sc;
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        ok = (1.0 - (__ldcg(W.colsq + c) + s)) >= 0.25;
      }
      if (lane == 0) flag[2 + wid] = ok ? c : 0x7fffffff;
      __syncthreads();
      // accept qualifying columns of this round in order (the same decisions in every thread)
      int take[NW];
      int nt = 0;
      for (int w = 0; w < NW; ++w)
        if (flag[2 + w] != 0x7fffffff && nf + nt < want) take[nt++] = w;
      if (KB > 0) {
        for (int q2 = 0; q2 < nt; ++q2) {
          for (int t = threadIdx.x; t < j; t += QT) bslot[(nf + q2) * ldc + t] = cv[take[q2] * ldc + t];
          if (threadIdx.x == 0) tflag[nf + q2] = flag[2 + take[q2]];
        }
      } else if (nt > 0 && nf == 0) {
        fw0 = take[0];
        if (threadIdx.x == 0) tflag[0] = flag[2 + take[0]];
      }
      nf += nt;
      __syncthreads();
    }
    if (nf == 0) {
      // no column ahead at distance >= 1/2: the farthest column (first on ties), single
      int besti = 0x7fffffff;
      double bestv = -2.0;
      for (int c = wid; c < m; c += NW) {
        double s = 0;
        for (int t = J0 + lane; t < j; t += 32) s += zabs2(__ldcg(X + (long long)t * m + c)) * scale(t);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const double dv = 1.0 - (__ldcg(W.colsq + c) + s);
        if (dv > bestv || (dv == bestv && c < besti)) { bestv = dv; besti = c; }
      }
      if (lane == 0) { red[wid] = bestv; flag[2 + wid] = besti; }
      __syncthreads();
      if (threadIdx.x == 0) {
        double bv = red[0];
        int bi = flag[2];
        for (int w = 1; w < NW; ++w)
          if (red[w] > bv || (red[w] == bv && flag[2 + w] < bi)) { bv = red[w]; bi = flag[2 + w]; }
        tflag[0] = min(max(bi < 0x7fffffff ? bi : 0, 0), m - 1);
      }
      __syncthreads();
      for (int t = threadIdx.x; t < j; t += QT) cv[t] = zscale(zconj(__ldcg(X + (long long)t * m + tflag[0])), scale(t));
      fw0 = 0;
      nf = 1;
      __syncthreads();
    }
    int K = 0;
    if (nf >= 2 && KB >= 2) {
      // Gram matrix of the projected unit vectors y_k = e_{p_k} - sum_t conj(Q_t[p_k]) Q_t:
      // G_kl = delta_kl - sum_t conj(Q_t[p_k]) Q_t[p_l]; with the stored coefficients
      // cv_k[t] = conj(Q_t[p_k]) / |x_t| this is delta_kl - sum_t cv_k[t] conj(cv_l[t]) |x_t|^2
      const int Kc = nf;
      for (int e2 = wid; e2 < Kc * (Kc + 1) / 2; e2 += NW) {
        int kk = 0;
        while ((kk + 1) * (kk + 2) / 2 <= e2) ++kk;
        const int ll = e2 - kk * (kk + 1) / 2;
        zc s2 = zmake(0, 0);
        for (int t = lane; t < j; t += 32) {
          const zc u = bslot[kk * ldc + t], v = bslot[ll * ldc + t];
          s2 = zadd(s2, zscale(zmul(u, zconj(v)), rnorm2(t)));
        }
        for (int o = 16; o > 0; o >>= 1) {
          s2.x += __shfl_xor_sync(0xffffffffu, s2.x, o);
          s2.y += __shfl_xor_sync(0xffffffffu, s2.y, o);
        }
        if (lane == 0) Gb[kk][ll] = zmake((kk == ll ? 1.0 : 0.0) - s2.x, -s2.y);
      }
      __syncthreads();
      // Cholesky G = L L^H in warp 0; pivot k is the distance of p_k after the batch's earlier
      // completions, so the batch stops at the first pivot below 1/4 (the exact rule would skip
      // that column there)
      if (threadIdx.x < 32) {
        int kgood = Kc;
        for (int jj = 0; jj < Kc; ++jj) {
          const double sp = Gb[jj][jj].x;
          if (!(sp >= 0.25)) { kgood = jj; break; }
          const double inv = rsqrt_nr(sp), d = sp * inv;   // sp in [1/4, 1]
          if (lane == 0) Ldi[jj] = inv;
          for (int i = lane; i < Kc; i += 32)
            Lb[i][jj] = (i < jj) ? zmake(0, 0) : (i == jj ? zmake(d, 0) : zscale(Gb[i][jj], inv));
          __syncwarp();
          const int Tt = Kc - jj - 1;
          for (int e2 = lane; e2 < Tt * Tt; e2 += 32) {
            const int i = jj + 1 + e2 / Tt, k2 = jj + 1 + e2 % Tt;
            if (k2 <= i) Gb[i][k2] = zfms(Lb[i][jj], zconj(Lb[k2][jj]), Gb[i][k2]);
          }
          __syncwarp();
        }
        if (lane == 0) tflag[TAIL_KB] = kgood;
      }
      __syncthreads();
      K = tflag[TAIL_KB];
    }
    if (K >= 2) {
      // Li = L^{-1} (lower triangular), one warp per column
      for (int cc = wid; cc < K; cc += NW) {
        if (lane == 0) Li[cc][cc] = zmake(Ldi[cc], 0.0);
        for (int i = 0; i < cc; ++i) if (lane == 0) Li[i][cc] = zmake(0, 0);
        __syncwarp();
        for (int i = cc + 1; i < K; ++i) {
          zc s2 = zmake(0, 0);
          for (int k2 = cc + lane; k2 < i; k2 += 32) s2 = zfma(Lb[i][k2], Li[k2][cc], s2);
          for (int o = 16; o > 0; o >>= 1) {
            s2.x += __shfl_xor_sync(0xffffffffu, s2.x, o);
            s2.y += __shfl_xor_sync(0xffffffffu, s2.y, o);
          }
          if (lane == 0) Li[i][cc] = zscale(s2, -Ldi[i]);
          __syncwarp();
        }
      }
      // y_k on this block's columns into rows j..j+K-1, then rows <- Li y (column by column)
      for (long long e2 = threadIdx.x; e2 < (long long)K * (c1 - c0); e2 += QT) {
        const int k2 = (int)(e2 / (c1 - c0)), c = c0 + (int)(e2 % (c1 - c0));
        X[(long long)(j + k2) * m + c] = zmake(c == tflag[k2] ? 1.0 : 0.0, 0.0);
      }
      __syncthreads();
      slab_update(X, m, j, K, j, bslot, ldc, c0, c1);
      const int ccols = max(1, QT / K);
      for (int cb = c0; cb < c1; cb += ccols) {
        const int nc = min(ccols, c1 - cb);
        for (int e2 = threadIdx.x; e2 < K * nc; e2 += QT) Yb[e2] = X[(long long)(j + e2 / nc) * m + cb + e2 % nc];
        __syncthreads();
        for (int e2 = threadIdx.x; e2 < K * nc; e2 += QT) {
          const int k2 = e2 / nc, cl = e2 % nc;
          zc v = zmake(0, 0);
          for (int k3 = 0; k3 <= k2; ++k3) v = zfma(Li[k2][k3], Yb[k3 * nc + cl], v);
          X[(long long)(j + k2) * m + cb + cl] = v;
        }
        __syncthreads();
      }
      if (threadIdx.x == 0)
        for (int k2 = 0; k2 < K; ++k2) { ens[a + k2] = 1.0; ens[QR_NMAX + a + k2] = 1.0; }
      pnext = tflag[K - 1] + 1;
      a += K;
      prev_single = false;
      __syncthreads();
      if (!group_sync(W, B)) return -1;
      continue;
    }
    // single completion: x_j = e_p - sum_t conj(Q_t[p]) Q_t, norm over the blocks at the barrier
    const int p = tflag[0];
    const zc* hc = (KB > 0 && fw0 < 0) ? bslot : cv + (fw0 > 0 ? fw0 : 0) * ldc;
    pnext = p + 1;
    zc* x = X + (long long)j * m;
    for (int c = c0 + threadIdx.x; c < c1; c += QT) x[c] = zmake(c == p ? 1.0 : 0.0, 0.0);
    __syncthreads();
    slab_update(X, m, j, 1, j, hc, ldc, c0, c1);
    {
      double s = 0;
      for (int c = c0 + threadIdx.x; c < c1; c += QT) s += zabs2(x[c]);
      s = block_sum(s, red);
      if (threadIdx.x == 0) S.Pn[(a & 1) * B + b] = zmake(s, 0.0);
    }
    if (!group_sync(W, B)) return -1;
    a += 1;
    prev_single = true;
  }
  __syncthreads();
  // normalise the completions on the slab, add them to the column sums the row path uses, and
  // put the rows after them back as they were.  The reciprocal norms are computed once per row
  // (into the second half of ens, whose single-completion scales are no longer needed).
  for (int a = threadIdx.x; a < Tc; a += QT) ens[QR_NMAX + a] = ens[a] > 0.0 ? 1.0 / sqrt(ens[a]) : 0.0;
  __syncthreads();
  for (long long e = threadIdx.x; e < (long long)Tc * (c1 - c0); e += QT) {
    const int a = (int)(e / (c1 - c0)), c = c0 + (int)(e % (c1 - c0));
    zc* x = X + (long long)(J0 + a) * m;
    x[c] = zscale(x[c], ens[QR_NMAX + a]);
  }
  __syncthreads();
  for (int c = c0 + threadIdx.x; c < c1; c += QT) {
    double s = W.colsq[c];
    for (int a = 0; a < Tc; ++a) s += zabs2(X[(long long)(J0 + a) * m + c]);
    W.colsq[c] = s;
  }
  for (long long e = threadIdx.x; e < (long long)(Tn - Tc) * (c1 - c0); e += QT) {
    const int j = J0 + Tc + (int)(e / (c1 - c0)), c = c0 + (int)(e % (c1 - c0));
    X[(long long)j * m + c] = BK[(long long)j * m + c];
  }
  if (!group_sync(W, B)) return -1;
  // R rows of the dropped rows: against rows < J0 the two projection passes (plus the panel's
  // passes for rows the panel had already projected), against the completions the dot products
  // of the backed-up rows, zero on and above the diagonal
  for (int e = gw; e < Tc * Tn; e += nwarps) {
    const int a = e / Tn, a2 = e % Tn;
    const int j = J0 + a, t = J0 + a2;
    zc v = zmake(0, 0);
    if (a2 < a) v = warp_dot(BK + (long long)j * m, X + (long long)t * m, m);
    if (lane == 0) J.Rout[J.rtrans ? (long long)t * n + j : (long long)j * n + t] = v;
  }
  if (b == 0) {
    for (int e = threadIdx.x; e < Tc * J0; e += QT) {
      const int a = e / J0, t = e % J0, j = J0 + a;
      zc v = zadd(__ldcg(HT1 + (long long)a * n + t), __ldcg(HT2 + (long long)a * n + t));
      if (j < pend && t < j0) {
        const int rr = j - j0;
        v = zadd(v, zadd(__ldcg(S.H1 + rr * n + t), __ldcg(S.H2 + rr * n + t)));
      }
      J.Rout[J.rtrans ? (long long)t * n + j : (long long)j * n + t] = v;
    }
  }
  // when the row path continues, the next panel rewrites the panel coefficients (S.H1, S.H2)
  // and the next tail the row backup, which block 0 and the dot products above still read
  if (Tc < Tn && !group_sync(W, B)) return -1;
  return Tc;
}

__global__ void __launch_bounds__(QT)
bqr_kernel(int dir, int site, const SiteDev* __restrict__ sd, const WorkDev* __restrict__ wk, int N_sites, int B,
           double rtol, int dn, int dm) {
  pdl_wait();
  __shared__ zc Hs[PB * QR_NMAX];
  __shared__ zc L1[PB][PB];
  __shared__ zc L2[PB][PB];
  __shared__ zc Gs[PB][PB];
  __shared__ double Gd[PB];
  __shared__ double Ldi[PB];            // 1 / L_kk of the current Cholesky factor
  __shared__ zc sdot[NW];
  __shared__ double red[NW];
  __shared__ int flag[2 + 2 * NW];
  __shared__ double ens[2 * QR_NMAX];   // tail rows: squared norms, then their reciprocals
  int tail_tries = 0;
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
  const int lane = threadIdx.x % 32, gw = b * NW + threadIdx.x / 32, nwarps = B * NW;
  zc* X = J.X;
  Scratch S;
  S.H1 = W.qpart;
  S.H2 = S.H1 + PB * n;
  S.G = S.H2 + PB * n;
  S.hv = S.G + PB * PB;
  S.Pn = S.hv + 2 * n;
  S.Pc = S.Pn + 2 * B;
  double* colsq = W.colsq;

  // ||X||_F and the rank threshold
  {
    double s = 0;
    const int cs = c1 - c0;
    for (long long e = threadIdx.x; e < (long long)n * cs; e += QT) {
      const int row = (int)(e / cs), c = c0 + (int)(e % cs);
      s += zabs2(X[(long long)row * m + c]);
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) S.Pn[b] = zmake(s, 0);
    for (int c = c0 + threadIdx.x; c < c1; c += QT) colsq[c] = 0.0;
  }
  if (!group_sync(W, B)) return;
  const double fro2 = sum_over_blocks(S.Pn, B);
  const double thresh = rtol * sqrt(fro2);

  int jnext = n;
  for (int j0 = 0; j0 < n; j0 = jnext) {
    const int nb = min(PB, n - j0);
    jnext = j0 + nb;
    // ---- two block Gram-Schmidt passes against rows 0..j0-1 ----
    for (int pass = 0; pass < 2 && j0 > 0; ++pass) {
      zc* Hb = pass ? S.H2 : S.H1;
      for (int e = gw; e < nb * j0; e += nwarps) {
        const int rr = e / j0, t = e % j0;
        const zc s = warp_dot(X + (long long)(j0 + rr) * m, X + (long long)t * m, m);
        if (lane == 0) Hb[rr * n + t] = s;
      }
      if (!group_sync(W, B)) return;
      for (int e = threadIdx.x; e < nb * j0; e += QT) Hs[(e / j0) * j0 + e % j0] = __ldcg(Hb + (e / j0) * n + e % j0);
      __syncthreads();
      slab_update(X, m, j0, nb, j0, Hs, j0, c0, c1);
      if (!group_sync(W, B)) return;
    }
    // ---- two Cholesky-QR passes inside the panel ----
    bool fallback = false;
    for (int it = 0; it < 2; ++it) {
      for (int e = gw; e < nb * (nb + 1) / 2; e += nwarps) {
        int rr = 0;
        while ((rr + 1) * (rr + 2) / 2 <= e) ++rr;
        const int ss = e - rr * (rr + 1) / 2;
        const zc s = warp_dot(X + (long long)(j0 + rr) * m, X + (long long)(j0 + ss) * m, m);   // sum x_r conj(x_s)
        if (lane == 0) S.G[rr * PB + ss] = s;
      }
      if (!group_sync(W, B)) return;
      zc (*Lc)[PB] = it ? L2 : L1;
      // Gram matrix into shared memory with one parallel load, then a right-looking Cholesky in
      // warp 0 with one lane per entry of the trailing triangle (no serial global loads).
      for (int e = threadIdx.x; e < nb * nb; e += QT) {
        const int i = e / nb, k = e % nb;
        Gs[i][k] = (k <= i) ? __ldcg(S.G + i * PB + k) : zmake(0, 0);
        if (i == k) Gd[i] = Gs[i][k].x;
      }
      __syncthreads();
      if (threadIdx.x < 32) {
        int bad = 0;
        for (int jj = 0; jj < nb; ++jj) {
          const double s = Gs[jj][jj].x;            // Schur complement pivot
          if (!(s > 0.0) || (it == 0 && (s <= 1e-10 * Gd[jj] || s <= 100.0 * thresh * thresh))) { bad = it + 1; break; }
          const double inv = (s > 1e-30 && s < 1e30) ? rsqrt_nr(s) : 1.0 / sqrt(s), d = s * inv;
          if (lane == 0) Ldi[jj] = inv;
          for (int i = lane; i < nb; i += 32)
            Lc[i][jj] = (i < jj) ? zmake(0, 0) : (i == jj ? zmake(d, 0) : zscale(Gs[i][jj], inv));
          __syncwarp();
          const int T = nb - jj - 1;
          for (int e = lane; e < T * T; e += 32) {
            const int i = jj + 1 + e / T, k = jj + 1 + e % T;
            if (k <= i) Gs[i][k] = zfms(Lc[i][jj], zconj(Lc[k][jj]), Gs[i][k]);
          }
          __syncwarp();
        }
        if (lane == 0) flag[0] = bad;
      }
      __syncthreads();
      if (flag[0] == 2) {              // the rows are already orthonormal to ~1e-6 here
        if (b == 0 && threadIdx.x == 0) atomicExch(W.err, -6);
        return;
      }
      if (flag[0]) { fallback = true; break; }
      // x_panel <- Lc^{-1} x_panel on the slab columns
      for (int c = c0 + threadIdx.x; c < c1; c += QT) {
        zc y[PB];
        for (int rr = 0; rr < nb; ++rr) {
          zc v = X[(long long)(j0 + rr) * m + c];
          for (int k = 0; k < rr; ++k) v = zfms(Lc[rr][k], y[k], v);
          y[rr] = zscale(v, Ldi[rr]);
        }
        for (int rr = 0; rr < nb; ++rr) X[(long long)(j0 + rr) * m + c] = y[rr];
      }
      if (it == 1 && b == 0) {
        // the panel's rows of R, before the barrier that ends the panel: past it the other
        // blocks start the next panel's first-pass dots, which overwrite S.H1
        for (int e = threadIdx.x; e < nb * n; e += QT) {
          const int rr = e / n, t = e % n, j = j0 + rr;
          zc v = zmake(0, 0);
          if (t < j0) {
            v = zadd(__ldcg(S.H1 + rr * n + t), __ldcg(S.H2 + rr * n + t));
          } else if (t <= j) {
            const int s2 = t - j0;                       // (L1 L2)[rr][s2]
            for (int k = s2; k <= rr; ++k) v = zfma(L1[rr][k], L2[k][s2], v);
          }
          J.Rout[J.rtrans ? (long long)t * n + j : (long long)j * n + t] = v;
        }
      }
      if (!group_sync(W, B)) return;
    }
    if (!fallback) {
      for (int c = c0 + threadIdx.x; c < c1; c += QT) {
        double s = colsq[c];
        for (int rr = 0; rr < nb; ++rr) s += zabs2(X[(long long)(j0 + rr) * m + c]);
        colsq[c] = s;
      }
      __syncthreads();
      continue;
    }
    // ---- exact row-by-row path for this panel ----
    // Per row: (A) first-pass dots; (B) update, residual norm and completion candidates;
    // full rows: (C) second-pass dots, (D) update and normalise; rank-deficient rows:
    // (C') completion vector e_p - sum_t conj(Q_t[p]) Q_t and its norm, (D') normalise.
    // The rank decision is taken on the residual after the first pass (the second pass
    // changes it by O(eps ||x||), far below the threshold), and a completion vector is at
    // distance >= 1/2 from the span, so one projection pass leaves it orthogonal to O(eps).
    for (int j = j0; j < j0 + nb; ++j) {
      const int rr = j - j0;
      zc* x = X + (long long)j * m;
      // (A)
      row_dots(X, m, x, j, S.hv, b, B, gw, nwarps, sdot);
      if (!group_sync(W, B)) return;
      // (B)
      for (int t = threadIdx.x; t < j; t += QT) Hs[t] = __ldcg(S.hv + t);
      __syncthreads();
      slab_update(X, m, j, 1, j, Hs, j, c0, c1);
      {
        double s = 0;
        int first = 0x7fffffff, besti = 0x7fffffff;
        double bestv = -1.0;
        for (int c = c0 + threadIdx.x; c < c1; c += QT) {
          s += zabs2(x[c]);
          const double dist = 1.0 - colsq[c];
          if (dist >= 0.25 && c < first) first = c;
          if (dist > bestv || (dist == bestv && c < besti)) { bestv = dist; besti = c; }
        }
        s = block_sum(s, red);
        for (int o = 16; o > 0; o >>= 1) {
          const int f2 = __shfl_xor_sync(0xffffffffu, first, o);
          const double v2 = __shfl_xor_sync(0xffffffffu, bestv, o);
          const int i2 = __shfl_xor_sync(0xffffffffu, besti, o);
          first = min(first, f2);
          if (v2 > bestv || (v2 == bestv && i2 < besti)) { bestv = v2; besti = i2; }
        }
        __syncthreads();
        if (lane == 0) { Hs[PB * QR_NMAX - 2 * NW + 2 * (threadIdx.x / 32)] = zmake((double)first, bestv);
                         Hs[PB * QR_NMAX - 2 * NW + 2 * (threadIdx.x / 32) + 1] = zmake((double)besti, 0); }
        __syncthreads();
        if (threadIdx.x == 0) {
          const zc* cw = Hs + PB * QR_NMAX - 2 * NW;
          double f = cw[0].x, bv = cw[0].y, bi = cw[1].x;
          for (int w = 1; w < NW; ++w) {
            f = fmin(f, cw[2 * w].x);
            const double v2 = cw[2 * w].y, i2 = cw[2 * w + 1].x;
            if (v2 > bv || (v2 == bv && i2 < bi)) { bv = v2; bi = i2; }
          }
          S.Pn[b] = zmake(s, 0);
          S.Pc[2 * b] = zmake(f, 0);
          S.Pc[2 * b + 1] = zmake(bv, bi);
        }
      }
      if (!group_sync(W, B)) return;
      const double s1 = sum_over_blocks(S.Pn, B);
      const bool full = s1 > thresh * thresh;
      double en;
      if (full) {
        // (C)
        row_dots(X, m, x, j, S.hv + n, b, B, gw, nwarps, sdot);
        if (!group_sync(W, B)) return;
        // (D)
        for (int t = threadIdx.x; t < j; t += QT) Hs[t] = __ldcg(S.hv + n + t);
        __syncthreads();
        slab_update(X, m, j, 1, j, Hs, j, c0, c1);
        double hh = 0;
        {
          double v = 0;
          for (int t = threadIdx.x; t < j; t += QT) v += zabs2(Hs[t]);
          hh = block_sum(v, red);
        }
        en = sqrt(fmax(s1 - hh, 0.0));
      } else {
        // (C') completion from the first unit vector at distance >= 1/2 (else the farthest)
        if (threadIdx.x < 32) {
          double f = 2147483647.0, bv = -2.0, bi = 2147483647.0;
          for (int bb = lane; bb < B; bb += 32) {
            f = fmin(f, __ldcg(S.Pc + 2 * bb).x);
            const zc q = __ldcg(S.Pc + 2 * bb + 1);
            if (q.x > bv || (q.x == bv && q.y < bi)) { bv = q.x; bi = q.y; }
          }
          for (int o = 16; o > 0; o >>= 1) {
            const double f2 = __shfl_xor_sync(0xffffffffu, f, o);
            const double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
            const double i2 = __shfl_xor_sync(0xffffffffu, bi, o);
            f = fmin(f, f2);
            if (v2 > bv || (v2 == bv && i2 < bi)) { bv = v2; bi = i2; }
          }
          if (lane == 0) flag[1] = (f < 2147483647.0) ? (int)f : (int)bi;
        }
        __syncthreads();
        const int p = flag[1];
        for (int t = threadIdx.x; t < j; t += QT) Hs[t] = zconj(__ldcg(X + (long long)t * m + p));
        for (int c = c0 + threadIdx.x; c < c1; c += QT) x[c] = zmake(c == p ? 1.0 : 0.0, 0);
        __syncthreads();
        slab_update(X, m, j, 1, j, Hs, j, c0, c1);
        {
          double s = 0;
          for (int c = c0 + threadIdx.x; c < c1; c += QT) s += zabs2(x[c]);
          s = block_sum(s, red);
          if (threadIdx.x == 0) S.Pn[B + b] = zmake(s, 0);
        }
        if (!group_sync(W, B)) return;
        en = sqrt(sum_over_blocks(S.Pn + B, B));
      }
      if (b == 0) {
        for (int t = threadIdx.x; t < n; t += QT) {
          zc v = zmake(0, 0);
          if (t < j) {
            v = __ldcg(S.hv + t);
            if (full) v = zadd(v, __ldcg(S.hv + n + t));
            if (t < j0) v = zadd(v, zadd(__ldcg(S.H1 + rr * n + t), __ldcg(S.H2 + rr * n + t)));
          } else if (t == j) {
            v = zmake(full ? en : 0.0, 0);
          }
          J.Rout[J.rtrans ? (long long)t * n + j : (long long)j * n + t] = v;
        }
      }
      const double inv = en > 0 ? 1.0 / en : 0.0;
      for (int c = c0 + threadIdx.x; c < c1; c += QT) {
        const zc v = zscale(x[c], inv);
        x[c] = v;
        colsq[c] += zabs2(v);
      }
      if (!group_sync(W, B)) return;
      // after a dropped row, try to finish every later row as a completion in one go
      if (!full && tail_tries < 8 && n - (j + 1) >= 2) {
        ++tail_tries;
        const int done = qr_tail(J, W, S, j + 1, j0, j0 + nb, b, B, gw, nwarps, c0, c1, thresh, sqrt(fro2), Hs, red,
                                 ens, flag);
        if (done < 0) return;
        if (j + 1 + done >= n) return;
        if (done > 0) {
          j += done;                       // rows up to j are final
          if (j + 1 >= j0 + nb) { jnext = j + 1; break; }
        }
      }
    }
  }
}

}  // namespace

cudaError_t launch_row_qr(int dir, int site, const SiteDev* sd, const WorkDev* wk, int R, int N_sites,
                          int blocks_per_r, double rtol, int dbg_n, int dbg_m, cudaStream_t st) {
  int B = blocks_per_r < 1 ? 1 : blocks_per_r;
  // co-resident blocks (the group barrier waits on every block of a realisation); launched with
  // the cooperative attribute so that the launch can also be captured into a CUDA graph
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.gridDim = dim3(R * B);
  cfg.blockDim = dim3(QT);
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, bqr_kernel, dir, site, sd, wk, N_sites, B, rtol, dbg_n, dbg_m);
}

int qr_max_coresident_blocks(int device) {
  int per_sm = 0, sms = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bqr_kernel, QT, 0);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  return per_sm * sms;
}
