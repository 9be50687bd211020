// FP64 contraction kernels of the TDVP-PS sweep: the three stages of H[i] C (Eq. tdvp2_C with
// H[i] of Eq. tdvp1_H), the left/right environment updates (Eq. tdvp1_h1i, tdvp1_hiN with
// Eq. tdvp1_h), the zero-site H0 D of Eq. tdvp2_D, the absorption C_{i+1} = D_i R_{i+1}, and the
// transfer pass used for populations.  Every launch is batched over realisations; the GEMM
// operands of each batch entry are derived on the device from the site tables.
#include "tdvp_internal.cuh"

namespace {

constexpr int TM = 32, TN = 32, TK = 16;   // complex tile: 32 x 32 outputs, K slab 16
constexpr int GEMM_THREADS = 256;          // 16 x 16 threads, 2 x 2 outputs each

// Number of independent GEMMs of an operation at site i of one realisation.
__device__ __forceinline__ int op_batch(int op, const SiteDev& s) {
  switch (op) {
    case OP_MV1: case OP_EL1: case OP_HX1: return s.Wl;
    case OP_EL3: case OP_ER1: return s.Wr;
    case OP_ER3: return s.Wl;
    case OP_Z1: return s.Wr;          // bond between i and i+1 carries W_r(i) channels
    default: return 1;
  }
}

__device__ bool make_desc(int op, int site, int b, const SiteDev* sdr, const WorkDev& wk, GemmDesc& g) {
  const SiteDev& s = sdr[site];
  const int Dl = s.Dl, d = s.d, Dr = s.Dr;
  const long long nsite = (long long)Dl * d * Dr;
  g.nz = 1; g.sAz = 0; g.sBz = 0; g.opA = 0; g.opB = 0; g.skip = nullptr; g.ws = nullptr;
  switch (op) {
    case OP_MV1: case OP_EL1: case OP_HX1: {
      // T1[b] (Dl x d*Dr) = L_b (Dl x Dl) * X (Dl x d*Dr)
      g.A = s.Lenv + (long long)b * Dl * Dl; g.lda = Dl;
      g.B = (op == OP_MV1) ? wk.x : s.A; g.ldb = d * Dr;
      g.C = wk.T1 + b * nsite; g.ldc = d * Dr;
      g.M = Dl; g.N = d * Dr; g.K = Dl;
      if (op == OP_MV1) g.skip = &wk.ks->done;
      return true;
    }
    case OP_MV3: {
      // w (Dl*d x Dr) = sum_w' T2[w'] (Dl*d x Dr) * R_w'^T
      g.A = wk.T2; g.lda = Dr; g.sAz = nsite;
      g.B = s.Renv; g.ldb = Dr; g.sBz = (long long)Dr * Dr; g.opB = 1;
      g.C = wk.w; g.ldc = Dr;
      g.M = Dl * d; g.N = Dr; g.K = Dr; g.nz = s.Wr;
      g.skip = &wk.ks->done;
      g.ws = wk.T1;
      return true;
    }
    case OP_EL3: {
      // Lenv(i+1)_b (Dr x Dr) = A^H (Dr x Dl*d) * T2[b] (Dl*d x Dr)
      g.A = s.A; g.lda = Dr; g.opA = 2;
      g.B = wk.T2 + b * nsite; g.ldb = Dr;
      g.C = sdr[site + 1].Lenv + (long long)b * Dr * Dr; g.ldc = Dr;
      g.M = Dr; g.N = Dr; g.K = Dl * d;
      g.ws = wk.T1;
      return true;
    }
    case OP_ER1: {
      // T1[b] (Dl*d x Dr) = A (Dl*d x Dr) * R_b^T
      g.A = s.A; g.lda = Dr;
      g.B = s.Renv + (long long)b * Dr * Dr; g.ldb = Dr; g.opB = 1;
      g.C = wk.T1 + b * nsite; g.ldc = Dr;
      g.M = Dl * d; g.N = Dr; g.K = Dr;
      return true;
    }
    case OP_ER3: {
      // Renv(i-1)_b (Dl x Dl) = conj(A) (Dl x d*Dr) * T2[b]^T, T2[b] viewed Dl x d*Dr
      g.A = s.A; g.lda = d * Dr; g.opA = 3;
      g.B = wk.T2 + b * nsite; g.ldb = d * Dr; g.opB = 1;
      g.C = sdr[site - 1].Renv + (long long)b * Dl * Dl; g.ldc = Dl;
      g.M = Dl; g.N = Dl; g.K = d * Dr;
      g.ws = wk.T1;
      return true;
    }
    case OP_Z1: {
      // bond (site, site+1): T1[b] (Db x Db) = Lb_b * x, Lb = Lenv(site+1)
      const int Db = Dr;
      g.A = sdr[site + 1].Lenv + (long long)b * Db * Db; g.lda = Db;
      g.B = wk.x; g.ldb = Db;
      g.C = wk.T1 + (long long)b * Db * Db; g.ldc = Db;
      g.M = Db; g.N = Db; g.K = Db;
      g.skip = &wk.ks->done;
      g.ws = wk.T2;
      return true;
    }
    case OP_Z3: {
      const int Db = Dr;
      g.A = wk.T1; g.lda = Db; g.sAz = (long long)Db * Db;
      g.B = s.Renv; g.ldb = Db; g.sBz = (long long)Db * Db; g.opB = 1;
      g.C = wk.w; g.ldc = Db;
      g.M = Db; g.N = Db; g.K = Db; g.nz = s.Wr;
      g.skip = &wk.ks->done;
      g.ws = wk.T2;
      return true;
    }
    case OP_ABS_L: {
      // x (Db x d'*Dr') = bond (Db x Db) * A_{site+1} (Db x d'*Dr')
      const SiteDev& t = sdr[site + 1];
      g.A = wk.bond; g.lda = t.Dl;
      g.B = t.A; g.ldb = t.d * t.Dr;
      g.C = wk.x; g.ldc = t.d * t.Dr;
      g.M = t.Dl; g.N = t.d * t.Dr; g.K = t.Dl;
      return true;
    }
    case OP_ABS_R: {
      // x (Dl'*d' x Db) = A_{site-1} (Dl'*d' x Db) * bond (Db x Db)
      const SiteDev& t = sdr[site - 1];
      g.A = t.A; g.lda = t.Dr;
      g.B = wk.bond; g.ldb = t.Dr;
      g.C = wk.x; g.ldc = t.Dr;
      g.M = t.Dl * t.d; g.N = t.Dr; g.K = t.Dr;
      return true;
    }
    case OP_TR1: {
      // T1 (Dl x d*Dr) = E (Dl x Dl) * A
      g.A = (site % 2 == 0) ? wk.bond2 : wk.bond; g.lda = Dl;
      g.B = s.A; g.ldb = d * Dr;
      g.C = wk.T1; g.ldc = d * Dr;
      g.M = Dl; g.N = d * Dr; g.K = Dl;
      return true;
    }
    case OP_TR3: {
      // E' (Dr x Dr) = A^H T1
      g.A = s.A; g.lda = Dr; g.opA = 2;
      g.B = wk.T1; g.ldb = Dr;
      g.C = (site % 2 == 0) ? wk.bond : wk.bond2; g.ldc = Dr;
      g.M = Dr; g.N = Dr; g.K = Dl * d;
      g.ws = wk.T2;
      return true;
    }
  }
  return false;
}

__device__ __forceinline__ zc load_op(const zc* P, int ld, int op, int row, int col) {
  // element (row, col) of op(P)
  switch (op) {
    case 0: return P[(long long)row * ld + col];
    case 1: return P[(long long)col * ld + row];
    case 2: return zconj(P[(long long)col * ld + row]);
    default: return zconj(P[(long long)row * ld + col]);
  }
}

// grid.z = (realisation, batch entry, K split).  With nsplit > 1 the flattened inner index
// (z, k-tile) is cut into nsplit contiguous ranges; each block writes its partial tile to the
// workspace and zgemm_reduce_kernel adds the partials in split order (deterministic).
__global__ void __launch_bounds__(GEMM_THREADS)
zgemm_kernel(int op, int site, const SiteDev* __restrict__ sd, const WorkDev* __restrict__ wk, int N_sites,
             int nbatch, int nsplit) {
  pdl_wait();
  __shared__ GemmDesc g;
  __shared__ int live;
  __shared__ zc As[TK][TM + 1];
  __shared__ zc Bs[TK][TN + 1];
  const int split = blockIdx.z % nsplit;
  const int zb = blockIdx.z / nsplit;
  const int r = zb / nbatch;
  const int b = zb % nbatch;
  if (threadIdx.x == 0) {
    const SiteDev* sdr = sd + (long long)r * N_sites;
    live = 0;
    if (b < op_batch(op, sdr[site]) && make_desc(op, site, b, sdr, wk[r], g)) {
      const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
      live = (m0 < g.M && n0 < g.N && !(g.skip && *g.skip)) ? 1 : 0;
      if (nsplit > 1 && !g.ws) live = 0;
    }
  }
  __syncthreads();
  if (!live) return;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  zc acc00 = zmake(0, 0), acc01 = acc00, acc10 = acc00, acc11 = acc00;
  const int M = g.M, N = g.N, K = g.K;
  const bool a_kfast = (g.opA == 0 || g.opA == 3);
  const bool b_nfast = (g.opB == 0 || g.opB == 3);
  const int nkt = (K + TK - 1) / TK;
  const int ktot = g.nz * nkt;
  const int kt0 = (int)((long long)ktot * split / nsplit), kt1 = (int)((long long)ktot * (split + 1) / nsplit);
  for (int kt = kt0; kt < kt1; ++kt) {
    const int z = kt / nkt, k0 = (kt % nkt) * TK;
    const zc* Az = g.A + z * g.sAz;
    const zc* Bz = g.B + z * g.sBz;
    // stage op(A)[m0:m0+TM, k0:k0+TK] and op(B)[k0:k0+TK, n0:n0+TN]
    for (int e = threadIdx.x; e < TM * TK; e += GEMM_THREADS) {
      int mm, kk;
      if (a_kfast) { mm = e / TK; kk = e % TK; } else { mm = e % TM; kk = e / TM; }
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < K) ? load_op(Az, g.lda, g.opA, gm, gk) : zmake(0, 0);
    }
    for (int e = threadIdx.x; e < TK * TN; e += GEMM_THREADS) {
      int kk, nn;
      if (b_nfast) { kk = e / TN; nn = e % TN; } else { kk = e % TK; nn = e / TK; }
      const int gk = k0 + kk, gn = n0 + nn;
      Bs[kk][nn] = (gk < K && gn < N) ? load_op(Bz, g.ldb, g.opB, gk, gn) : zmake(0, 0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      const zc a0 = As[kk][ty], a1 = As[kk][ty + 16];
      const zc b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
      acc00 = zfma(a0, b0, acc00);
      acc01 = zfma(a0, b1, acc01);
      acc10 = zfma(a1, b0, acc10);
      acc11 = zfma(a1, b1, acc11);
    }
    __syncthreads();
  }
  zc* C = g.C;
  long long ldc = g.ldc;
  if (nsplit > 1) {   // partial tile into the workspace, dense M x N per (batch entry, split)
    C = g.ws + ((long long)b * nsplit + split) * M * N;
    ldc = N;
  }
  const int r0 = m0 + ty, r1 = m0 + ty + 16, c0 = n0 + tx, c1 = n0 + tx + 16;
  if (r0 < M && c0 < N) C[(long long)r0 * ldc + c0] = acc00;
  if (r0 < M && c1 < N) C[(long long)r0 * ldc + c1] = acc01;
  if (r1 < M && c0 < N) C[(long long)r1 * ldc + c0] = acc10;
  if (r1 < M && c1 < N) C[(long long)r1 * ldc + c1] = acc11;
}

__global__ void __launch_bounds__(256)
zgemm_reduce_kernel(int op, int site, const SiteDev* __restrict__ sd, const WorkDev* __restrict__ wk, int N_sites,
                    int nbatch, int nsplit) {
  pdl_wait();
  __shared__ GemmDesc g;
  __shared__ int live;
  const int r = blockIdx.y / nbatch, b = blockIdx.y % nbatch;
  if (threadIdx.x == 0) {
    const SiteDev* sdr = sd + (long long)r * N_sites;
    live = (b < op_batch(op, sdr[site]) && make_desc(op, site, b, sdr, wk[r], g) && g.ws && !(g.skip && *g.skip));
  }
  __syncthreads();
  if (!live) return;
  const long long MN = (long long)g.M * g.N;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= MN) return;
  const zc* P = g.ws + (long long)b * nsplit * MN + e;
  zc s = P[0];
  for (int q = 1; q < nsplit; ++q) s = zadd(s, P[q * MN]);
  g.C[(e / g.N) * g.ldc + e % g.N] = s;
}

// Middle stage: out[co][x][so][y] = sum_e val * in[ci][x][si][y] (the sparse MPO of Eq. mpo).
__global__ void __launch_bounds__(256)
wapply_kernel(int dir, int site, int lanczos, const SiteDev* __restrict__ sd, const WorkDev* __restrict__ wk,
              int N_sites) {
  pdl_wait();
  const int r = blockIdx.z;
  const SiteDev& s = sd[(long long)r * N_sites + site];
  const WorkDev& W = wk[r];
  if (lanczos && W.ks->done) return;
  const int X = s.Dl, Y = s.Dr, d = s.d;
  const int n_out = dir == 0 ? s.Wr : s.Wl;
  const int row = blockIdx.y;
  if (row >= n_out * d) return;
  const int xy = blockIdx.x * blockDim.x + threadIdx.x;
  if (xy >= X * Y) return;
  const int x = xy / Y, y = xy % Y;
  const WCsr& c = dir == 0 ? s.fw : s.bw;
  const int co = row / d, so = row % d;
  zc acc = zmake(0, 0);
  for (int e = c.ptr[row]; e < c.ptr[row + 1]; ++e) {
    const zc v = W.T1[(((long long)c.ci[e] * X + x) * d + c.si[e]) * Y + y];
    acc.x = fma(c.val[e], v.x, acc.x);
    acc.y = fma(c.val[e], v.y, acc.y);
  }
  W.T2[(((long long)co * X + x) * d + so) * Y + y] = acc;
}

// Site tensor (Dl*d x Dr) <-> scratch (Dr x Dl*d), realisation r = blockIdx.z.
__global__ void transpose_site_kernel(int to_scratch, int site, const SiteDev* __restrict__ sd,
                                      const WorkDev* __restrict__ wk, int N_sites) {
  pdl_wait();
  __shared__ zc tile[32][33];
  const int r = blockIdx.z;
  const SiteDev& s = sd[(long long)r * N_sites + site];
  const int rows = s.Dl * s.d, cols = s.Dr;          // the site tensor viewed as rows x cols
  zc* A = s.A;
  zc* S = wk[r].scratch;
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;   // 32 x 8 threads
  if (to_scratch) {
    if (by >= rows || bx >= cols) return;
    for (int j = ty; j < 32; j += 8) {
      const int rr = by + j, cc = bx + tx;
      if (rr < rows && cc < cols) tile[j][tx] = A[(long long)rr * cols + cc];
    }
    __syncthreads();
    for (int j = ty; j < 32; j += 8) {
      const int cc = bx + j, rr = by + tx;      // scratch[cc][rr]
      if (rr < rows && cc < cols) S[(long long)cc * rows + rr] = tile[tx][j];
    }
  } else {
    // scratch is cols x rows; blockIdx.y runs over scratch rows (= A cols)
    if (by >= cols || bx >= rows) return;
    for (int j = ty; j < 32; j += 8) {
      const int rr = by + j, cc = bx + tx;      // scratch[rr][cc]
      if (rr < cols && cc < rows) tile[j][tx] = S[(long long)rr * rows + cc];
    }
    __syncthreads();
    for (int j = ty; j < 32; j += 8) {
      const int cc = bx + j, rr = by + tx;      // A[cc][rr] = scratch[rr][cc]
      if (rr < cols && cc < rows) A[(long long)cc * cols + rr] = tile[tx][j];
    }
  }
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x / 32); ++i) s += red[i];
  return s;   // valid in thread 0
}

__global__ void set_identity_kernel(const WorkDev* __restrict__ wk, int n) {
  pdl_wait();
  const int r = blockIdx.x;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x)
    wk[r].bond2[e] = zmake((e / n) == (e % n) ? 1.0 : 0.0, 0.0);
}

// <n> at an electronic site: sum_{l', r} conj(A[l'][1][r]) T1[l'][1][r], T1 = E A.
__global__ void obs_local_kernel(int site, int slot, const SiteDev* __restrict__ sd,
                                 const WorkDev* __restrict__ wk, int N_sites) {
  pdl_wait();
  __shared__ double red[32];
  const int r = blockIdx.x;
  const SiteDev& s = sd[(long long)r * N_sites + site];
  const WorkDev& W = wk[r];
  double acc = 0;
  for (int e = threadIdx.x; e < s.Dl * s.Dr; e += blockDim.x) {
    const int l = e / s.Dr, rr = e % s.Dr;
    const long long off = ((long long)l * s.d + 1) * s.Dr + rr;
    const zc a = s.A[off], t = W.T1[off];
    acc += a.x * t.x + a.y * t.y;
  }
  const double tot = block_sum(acc, red);
  if (threadIdx.x == 0) W.obs[slot] = tot;
}

__global__ void obs_norm_kernel(int site, int slot, const WorkDev* __restrict__ wk) {
  pdl_wait();
  const int r = blockIdx.x;
  const WorkDev& W = wk[r];
  if (threadIdx.x == 0) W.obs[slot] = ((site % 2 == 0) ? W.bond : W.bond2)[0].x;
}

// <C|w> with C the site-0 tensor (w = H[0] C): energy numerator.
__global__ void obs_energy_kernel(int slot, const SiteDev* __restrict__ sd, const WorkDev* __restrict__ wk,
                                  int N_sites) {
  pdl_wait();
  __shared__ double red[32];
  const int r = blockIdx.x;
  const SiteDev& s = sd[(long long)r * N_sites + 0];
  const WorkDev& W = wk[r];
  const int n = s.Dl * s.d * s.Dr;
  double acc = 0, nn = 0;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const zc a = s.A[e], t = W.w[e];
    acc += a.x * t.x + a.y * t.y;
    nn += a.x * a.x + a.y * a.y;
  }
  const double tot = block_sum(acc, red);
  __syncthreads();
  const double tn = block_sum(nn, red);
  if (threadIdx.x == 0) { W.obs[slot] = tot; W.obs[slot + 1] = tn; }
}

// what 0: x <- A[site]; what 1: A[site] <- x; what 2: A[site] <- w
__global__ void copy_vec_kernel(int what, int site, const SiteDev* __restrict__ sd, const WorkDev* __restrict__ wk,
                                int N_sites) {
  pdl_wait();
  const int r = blockIdx.y;
  const SiteDev& s = sd[(long long)r * N_sites + site];
  const long long n = (long long)s.Dl * s.d * s.Dr;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  if (what == 0) wk[r].x[e] = s.A[e];
  else if (what == 1) s.A[e] = wk[r].x[e];
  else s.A[e] = wk[r].w[e];
}

__global__ void reset_ks_kernel(const WorkDev* __restrict__ wk) {
  pdl_wait();
  if (threadIdx.x == 0) { wk[blockIdx.x].ks->done = 0; wk[blockIdx.x].ks->status = 0; }
}

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace

cudaError_t launch_gemm(int op, int site, const SiteDev* sd, const WorkDev* wk, int R, int N_sites, int maxM,
                        int maxN, int nbatch, int nsplit, cudaStream_t st) {
  if (maxM <= 0 || maxN <= 0 || nbatch <= 0) return cudaSuccess;
  if (nsplit < 1) nsplit = 1;
  dim3 grid(cdiv(maxN, TN), cdiv(maxM, TM), R * nbatch * nsplit);
  { const cudaError_t e_ = launch_pdl(zgemm_kernel, grid, GEMM_THREADS, 0, st, op, site, sd, wk, N_sites, nbatch, nsplit); if (e_ != cudaSuccess) return e_; }
  if (nsplit > 1) {
    dim3 g2(cdiv((long long)maxM * maxN, 256), R * nbatch);
    { const cudaError_t e_ = launch_pdl(zgemm_reduce_kernel, g2, 256, 0, st, op, site, sd, wk, N_sites, nbatch, nsplit); if (e_ != cudaSuccess) return e_; }
  }
  return cudaGetLastError();
}

cudaError_t launch_wapply(int dir, int site, int lanczos, const SiteDev* sd, const WorkDev* wk, int R,
                          int N_sites, int max_xy, int n_rows, cudaStream_t st) {
  dim3 grid(cdiv(max_xy, 256), n_rows, R);
  { const cudaError_t e_ = launch_pdl(wapply_kernel, grid, 256, 0, st, dir, site, lanczos, sd, wk, N_sites); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

cudaError_t launch_transpose_site(int to_scratch, int site, const SiteDev* sd, const WorkDev* wk, int R,
                                  int N_sites, int maxRows, int maxCols, cudaStream_t st) {
  dim3 grid = to_scratch ? dim3(cdiv(maxCols, 32), cdiv(maxRows, 32), R) : dim3(cdiv(maxRows, 32), cdiv(maxCols, 32), R);
  { const cudaError_t e_ = launch_pdl(transpose_site_kernel, grid, 256, 0, st, to_scratch, site, sd, wk, N_sites); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

cudaError_t launch_set_identity_bond2(const WorkDev* wk, int R, int n, cudaStream_t st) {
  { const cudaError_t e_ = launch_pdl(set_identity_kernel, R, 128, 0, st, wk, n); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

cudaError_t launch_obs_local(int site, int slot, const SiteDev* sd, const WorkDev* wk, int R, int N_sites,
                             cudaStream_t st) {
  { const cudaError_t e_ = launch_pdl(obs_local_kernel, R, 256, 0, st, site, slot, sd, wk, N_sites); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

cudaError_t launch_obs_norm(int site, int slot, const WorkDev* wk, int R, cudaStream_t st) {
  { const cudaError_t e_ = launch_pdl(obs_norm_kernel, R, 32, 0, st, site, slot, wk); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

cudaError_t launch_obs_energy(int slot, const SiteDev* sd, const WorkDev* wk, int R, int N_sites, cudaStream_t st) {
  { const cudaError_t e_ = launch_pdl(obs_energy_kernel, R, 256, 0, st, slot, sd, wk, N_sites); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

cudaError_t launch_copy_vec(int what, int site, const SiteDev* sd, const WorkDev* wk, int R, int N_sites, int maxn,
                            cudaStream_t st) {
  dim3 grid(cdiv(maxn, 256), R);
  { const cudaError_t e_ = launch_pdl(copy_vec_kernel, grid, 256, 0, st, what, site, sd, wk, N_sites); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

cudaError_t launch_reset_ks(const WorkDev* wk, int R, cudaStream_t st) {
  { const cudaError_t e_ = launch_pdl(reset_ks_kernel, R, 32, 0, st, wk); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}
