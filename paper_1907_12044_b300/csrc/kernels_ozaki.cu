// FP64 complex GEMM emulated on the BF16 tensor cores by the Ozaki splitting.
//
// The FP64 parts of the method (the FP64 arm's contractions, the absorption C_{i+1} = D_i R_{i+1})
// run on B300's FP64 pipe, which is far slower than its tensor cores.  This entry point computes
// C = A B (A: m x k, B: k x n, C: m x n; complex FP64, row-major, interleaved re/im) from exact
// BF16 pieces of the operands (Ozaki, Ogita, Oishi, Rump 2012, error-free splitting; here on BF16
// rather than integer tensor cores, whose rate on B300 is far below the BF16 rate):
//
//   complex -> real:  [Cr; Ci] = [[Ar, -Ai], [Ai, Ar]] [Br; Bi], a (2m x 2k) by (2k x n) product;
//   splitting:        row R of the embedded A is scaled by 2^-eR (eR: the exponent that puts the
//                     row's largest magnitude below 1) and cut into s slices of 7 bits,
//                     x = sum_{i<s} q_i 2^(-7(i+1)) + rest, q_i = trunc(2^7 * remainder), |q_i| <= 127,
//                     |rest| < 2^(-7s); column c of the embedded B likewise (fc, p_j).  Every q and
//                     p is an integer of at most 7 bits: exact in BF16;
//   products:         C[R][c] ~= 2^(eR + fc) sum_{g<s} 2^(-7(g+2)) G_g[R][c],
//                     G_g = sum_{i+j=g} Q_i P_j (the pairs with i + j >= s are below the emulated
//                     precision and left out: s(s+1)/2 BF16 products per K tile);
//   exactness:        |q p| <= 127^2 < 2^14, and over a window of 128 K values and at most 8 slice
//                     pairs 8 * 128 * 127^2 = 16.5 M < 2^24, so the FP32 tensor-memory accumulation
//                     of G_g over one window is exact whatever its rounding;
//   accumulation:     after each window the epilogue warps read the s accumulators (tcgen05.ld) and
//                     add 2^(-7(g+2)) G_g into a float-float (hi + lo, two FP32) sum per element
//                     with an error-free two-sum; only these additions round (~2^-48 relative), so
//                     no FP64 instruction runs in the main loop.
//
// Error per element: |C - A B| <= 2k (s + 3) 2^(-7s) 2^(eR + fc) + ~2^-47 k 2^(eR + fc).
// s = 8 gives ~1e-14 relative to k max|A_R| max|B_c|; fewer slices trade accuracy for speed.
//
// Kernel: one CTA per 128 x 64 output tile of the embedded product, 160 threads; warp 4 lane 0
// issues 1-D bulk copies (two-stage ring, one contiguous block of s slice planes per operand and
// K tile) and the MMAs (kind::f16, BF16 in, FP32 in tensor memory, accumulator g at columns
// 64g..64g+63); warps 0-3 own one tensor-memory lane (one output row) each.  Every wait is
// bounded (1 s); on timeout the kernel records -5 in the workspace's error word, drains its copies
// and MMAs with bounded waits, frees its tensor memory and returns.
#include "tdvp_internal.cuh"
#include "tc_ptx.cuh"
#include "tdvp.h"
#include <cuda_bf16.h>
#include <climits>
#include <cstdint>

namespace {

constexpr int OZ_BM = 128, OZ_BN = 64, OZ_BK = 32;
constexpr int OZ_SMAX = 8;
constexpr int OZ_A_PLANE = OZ_BM * OZ_BK * 2;        // 8 KB: one BF16 slice of a 128 x 32 A tile
constexpr int OZ_B_PLANE = OZ_BN * OZ_BK * 2;        // 4 KB: one BF16 slice of a 64 x 32 B tile
constexpr int OZ_STAGES = 2;
constexpr int OZ_KW = 4;                             // K tiles per exact accumulation window
constexpr int OZ_EPI = 128;
constexpr int OZ_THREADS = OZ_EPI + 32;
constexpr int OZ_PART_LD = OZ_BN + 1;                // staging row stride in doubles
constexpr uint32_t OZ_TMEM_COLS = 512;

__host__ __device__ constexpr int oz_cdiv(long long a, int b) { return (int)((a + b - 1) / b); }

// byte offset of (row, kk) inside one BF16 K-major no-swizzle tile of 32 columns: core matrices of
// 8 rows x 16 bytes, adjacent in K 128 bytes apart, 8-row groups 512 bytes apart
__device__ __forceinline__ int oz_off(int row, int kk) {
  return (row >> 3) * 512 + (kk >> 3) * 128 + (row & 7) * 16 + (kk & 7) * 2;
}

// instruction descriptor: D = F32, A = B = BF16 (kind::f16), K-major, M = 128, N = 64
__device__ __forceinline__ uint32_t oz_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_BN >> 3) << 17) | ((uint32_t)(OZ_BM >> 4) << 24);
}

// exponent e with |v| < 2^e (frexp), INT_MIN for 0
__device__ __forceinline__ int oz_exp(double v) {
  if (v == 0.0) return INT_MIN;
  int e;
  frexp(v, &e);
  return e;
}

// row exponents of the embedded A (shared by rows r and r + m): one warp per complex row
__global__ void oz_row_exp_kernel(int m, int k, const zc* __restrict__ A, int* __restrict__ eA) {
  const int r = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x % 32;
  if (r >= m) return;
  double mx = 0.0;
  for (int c = lane; c < k; c += 32) {
    const zc v = A[(long long)r * k + c];
    mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) eA[r] = oz_exp(mx);
}

// column exponents of the embedded B (columns of B over both parts): eB starts at INT_MIN; each
// thread takes one column over a chunk of 64 rows
__global__ void oz_col_exp_kernel(int k, int n, const zc* __restrict__ B, int* __restrict__ fB) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x, r0 = blockIdx.y * 64;
  if (c >= n) return;
  double mx = 0.0;
  const int r1 = min(k, r0 + 64);
  for (int r = r0; r < r1; ++r) {
    const zc v = B[(long long)r * n + c];
    mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
  }
  if (mx > 0.0) atomicMax(&fB[c], oz_exp(mx));
}

// the s slices of x in [-1, 1): q_i = trunc(2^7 * remainder), written as BF16 (exact)
__device__ __forceinline__ void oz_slices(double x, int s, unsigned char* base, long long plane, int off) {
  for (int i = 0; i < s; ++i) {
    x *= 128.0;
    const double q = trunc(x);
    x -= q;
    *reinterpret_cast<__nv_bfloat16*>(base + i * plane + off) = __float2bfloat16_rn((float)q);
  }
}

// embedded A [(2m) x (2k)] -> slices, tile (mt, kt) block at ((mt * nkt + kt) * s) * 8 KB
__global__ void oz_pack_a_kernel(int m, int k, int s, const zc* __restrict__ A, const int* __restrict__ eA,
                                 unsigned char* __restrict__ P) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long K2 = 2LL * k;
  if (e >= 2LL * m * K2) return;
  const int R = (int)(e / K2), Kc = (int)(e % K2);
  const int r = R < m ? R : R - m, c = Kc < k ? Kc : Kc - k;
  const zc v = A[(long long)r * k + c];
  double x;
  if (R < m) x = Kc < k ? v.x : -v.y;     // [Ar, -Ai]
  else x = Kc < k ? v.y : v.x;            // [Ai,  Ar]
  const int er = eA[r];
  if (er == INT_MIN) return;              // zero row: the zeroed slices stand
  x = ldexp(x, -er);
  const int nkt = oz_cdiv(K2, OZ_BK), mt = R / OZ_BM, kt = Kc / OZ_BK;
  unsigned char* base = P + ((long long)mt * nkt + kt) * s * OZ_A_PLANE;
  oz_slices(x, s, base, OZ_A_PLANE, oz_off(R % OZ_BM, Kc % OZ_BK));
}

// embedded B [(2k) x n] as the B operand (rows = output columns, K-major), tile (nt, kt) block at
// ((nt * nkt + kt) * s) * 4 KB
__global__ void oz_pack_b_kernel(int k, int n, int s, const zc* __restrict__ B, const int* __restrict__ fB,
                                 unsigned char* __restrict__ P) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2LL * k * n) return;
  const int Kc = (int)(e / n), c = (int)(e % n);
  const zc v = B[(long long)(Kc < k ? Kc : Kc - k) * n + c];
  const int fc = fB[c];
  if (fc == INT_MIN) return;
  const double x = ldexp(Kc < k ? v.x : v.y, -fc);
  const int nkt = oz_cdiv(2LL * k, OZ_BK), nt = c / OZ_BN, kt = Kc / OZ_BK;
  unsigned char* base = P + ((long long)nt * nkt + kt) * s * OZ_B_PLANE;
  oz_slices(x, s, base, OZ_B_PLANE, oz_off(c % OZ_BN, Kc % OZ_BK));
}

// error-free sum of (hi, lo) and an exact FP32 value a (Knuth's two-sum; no contraction)
__device__ __forceinline__ void oz_add(float& hi, float& lo, float a) {
  const float s = __fadd_rn(hi, a);
  const float bp = __fadd_rn(s, -hi);
  const float err = __fadd_rn(__fadd_rn(hi, -__fadd_rn(s, -bp)), __fadd_rn(a, -bp));
  hi = s;
  lo = __fadd_rn(lo, err);
}

__global__ void __launch_bounds__(OZ_THREADS, 1)
oz_gemm_kernel(int m, int n, int k, int s, const unsigned char* __restrict__ PA, const unsigned char* __restrict__ PB,
               const int* __restrict__ eA, const int* __restrict__ fB, zc* __restrict__ C, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t full_bar[OZ_STAGES];
  __shared__ uint64_t done_bar[OZ_STAGES];
  __shared__ uint64_t acc_full, acc_free, drain_bar;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag, drain_fail;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int nt = blockIdx.x, mt = blockIdx.y;
  const int M2 = 2 * m, nkt = oz_cdiv(2LL * k, OZ_BK), nwin = oz_cdiv(nkt, OZ_KW);
  const uint32_t stage_a = (uint32_t)s * OZ_A_PLANE, stage_b = (uint32_t)s * OZ_B_PLANE;
  const uint32_t stage_bytes = stage_a + stage_b;
  if (threadIdx.x == 0) {
    abort_flag = 0;
    drain_fail = 0;
    for (int q = 0; q < OZ_STAGES; ++q) { mbar_init(&full_bar[q], 1); mbar_init(&done_bar[q], 1); }
    mbar_init(&acc_full, 1);
    mbar_init(&acc_free, OZ_EPI);
    mbar_init(&drain_bar, 1);
    mbar_fence_init();
  }
  if (warp == 0) tmem_alloc(&tmem_base, OZ_TMEM_COLS);
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = tmem_base;
  float hi[OZ_BN], lo[OZ_BN];
#pragma unroll
  for (int q = 0; q < OZ_BN; ++q) { hi[q] = 0.f; lo[q] = 0.f; }
  if (warp == OZ_EPI / 32) {
    if (lane == 0) {
      auto issue = [&](int kt) {
        const int st = kt % OZ_STAGES;
        unsigned char* sp = smem + st * stage_bytes;
        mbar_expect_tx(&full_bar[st], stage_bytes);
        bulk_load(sp, PA + ((long long)mt * nkt + kt) * stage_a, stage_a, &full_bar[st]);
        bulk_load(sp + stage_a, PB + ((long long)nt * nkt + kt) * stage_b, stage_b, &full_bar[st]);
      };
      const uint32_t idesc = oz_idesc();
      int issued = 0;
      for (; issued < OZ_STAGES && issued < nkt; ++issued) issue(issued);
      for (int kt = 0; kt < nkt && !abort_flag; ++kt) {
        const int st = kt % OZ_STAGES, w = kt / OZ_KW, kin = kt % OZ_KW;
        const uint32_t par = (uint32_t)((kt / OZ_STAGES) & 1);
        if (!mbar_wait(&full_bar[st], par)) { abort_flag = 1; break; }
        // the accumulators are free once the epilogue has read window w - 1
        if (kin == 0 && w > 0 && !mbar_wait_or(&acc_free, (uint32_t)((w - 1) & 1), &drain_fail)) {
          abort_flag = 1;
          break;
        }
        tc_after();
        const uint32_t abase = su32(smem + st * stage_bytes), bbase = abase + stage_a;
        for (int i = 0; i < s; ++i) {
          for (int j = 0; j + i < s; ++j) {
            const uint32_t d = tmem + (uint32_t)(i + j) * OZ_BN;
#pragma unroll
            for (int ks = 0; ks < OZ_BK / 16; ++ks) {
              // one instruction covers 16 BF16 of K per row (two core matrices, 256 bytes)
              const uint64_t da = sdesc(abase + i * OZ_A_PLANE + ks * 256, 512);
              const uint64_t db = sdesc(bbase + j * OZ_B_PLANE + ks * 256, 512);
              mma_bf16(d, da, db, idesc, (kin > 0 || ks > 0 || i > 0) ? 1u : 0u);
            }
          }
        }
        mma_commit(&done_bar[st]);
        if (kin == OZ_KW - 1 || kt == nkt - 1) mma_commit(&acc_full);
        if (issued < nkt) {
          if (!mbar_wait(&done_bar[st], par)) { abort_flag = 1; break; }
          issue(issued);
          ++issued;
        }
      }
      if (abort_flag) {
        for (int q = 0; q < OZ_STAGES; ++q) {
          int last = -1;
          for (int kt = 0; kt < issued; ++kt) if (kt % OZ_STAGES == q) last = kt;
          if (last >= 0) mbar_wait(&full_bar[q], (uint32_t)((last / OZ_STAGES) & 1));
        }
        mma_commit(&drain_bar);
        mbar_wait(&drain_bar, 0);
        atomicExch(err, -5);
      }
    }
    __syncwarp();
  } else {
    // warp w reads tensor-memory lanes 32w..32w+31: thread = row of the tile
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
    bool ok = true;
    for (int w = 0; w < nwin; ++w) {
      const bool got = mbar_wait_or(&acc_full, (uint32_t)(w & 1), &abort_flag);
      if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
      tc_after();
      for (int g = 0; g < s; ++g) {
        const float sc = ldexpf(1.0f, -7 * (g + 2));   // exact power of two
#pragma unroll
        for (int cb = 0; cb < OZ_BN; cb += 16) {
          float v[16];
          tmem_ld16(lane_addr + (uint32_t)g * OZ_BN + cb, v);
#pragma unroll
          for (int q = 0; q < 16; ++q) oz_add(hi[cb + q], lo[cb + q], __fmul_rn(v[q], sc));
        }
      }
      tc_before();
      mbar_arrive(&acc_free);
    }
    if (!ok && lane == 0) drain_fail = 1;
  }
  tc_before();
  __syncthreads();
  tc_after();
  const bool ok = !abort_flag && !drain_fail;
  if (!ok && threadIdx.x == 0) atomicExch(err, -5);
  // rows -> shared memory (the copies are complete), then coalesced scaled stores
  double* part = reinterpret_cast<double*>(smem);
  if (warp < OZ_EPI / 32) {
    const int row = warp * 32 + lane;
#pragma unroll
    for (int q = 0; q < OZ_BN; ++q) part[row * OZ_PART_LD + q] = (double)hi[q] + (double)lo[q];
  }
  __syncthreads();
  if (ok) {
    for (int e = threadIdx.x; e < OZ_BM * OZ_BN; e += OZ_THREADS) {
      const int lr = e / OZ_BN, col = e % OZ_BN;
      const int R = mt * OZ_BM + lr, c = nt * OZ_BN + col;
      if (R >= M2 || c >= n) continue;
      const int r = R < m ? R : R - m;
      const int er = eA[r], fc = fB[c];
      const double v = (er == INT_MIN || fc == INT_MIN) ? 0.0 : ldexp(part[lr * OZ_PART_LD + col], er + fc);
      double* out = reinterpret_cast<double*>(C + (long long)r * n + c);
      out[R < m ? 0 : 1] = v;
    }
  }
  __syncthreads();
  tc_after();
  if (warp == 0) tmem_free(tmem, OZ_TMEM_COLS);
}

__global__ void oz_fill_kernel(int* p, int count, int v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) p[i] = v;
}

}  // namespace

// ---- workspace layout: [error word | eA (m ints) | fB (n ints) | A slices | B slices] ----
namespace {
struct OzLayout {
  size_t eA, fB, pa, pb, total;
  long long pa_bytes, pb_bytes;
};
size_t oz_align(size_t x) { return (x + 1023) & ~(size_t)1023; }
OzLayout oz_layout(int m, int n, int k, int s) {
  OzLayout L;
  const long long nkt = ((2LL * k) + OZ_BK - 1) / OZ_BK;
  const long long mtiles = ((2LL * m) + OZ_BM - 1) / OZ_BM, ntiles = ((long long)n + OZ_BN - 1) / OZ_BN;
  L.pa_bytes = mtiles * nkt * s * OZ_A_PLANE;
  L.pb_bytes = ntiles * nkt * s * OZ_B_PLANE;
  L.eA = 1024;
  L.fB = oz_align(L.eA + sizeof(int) * (size_t)m);
  L.pa = oz_align(L.fB + sizeof(int) * (size_t)n);
  L.pb = oz_align(L.pa + (size_t)L.pa_bytes);
  L.total = oz_align(L.pb + (size_t)L.pb_bytes);
  return L;
}
bool oz_args_ok(int m, int n, int k, int s) {
  // grid limits: 2m / 128 and k / 64 blocks along y (<= 65535), the pack kernels' element counts
  // (4mk, 2kn) / 256 blocks along x (< 2^31)
  return m >= 1 && n >= 1 && k >= 1 && s >= 1 && s <= OZ_SMAX && m <= (1 << 21) && k <= (1 << 21) &&
         n <= (1 << 28) && 4LL * m * k <= (1LL << 36) && 2LL * k * n <= (1LL << 36);
}
bool oz_overlap(const void* a, size_t an, const void* b, size_t bn) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + bn && y < x + an;
}
}  // namespace

extern "C" size_t tdvp_zgemm_ozaki_workspace(int m, int n, int k, int slices) {
  if (!oz_args_ok(m, n, k, slices)) return 0;
  return oz_layout(m, n, k, slices).total;
}

extern "C" int tdvp_zgemm_ozaki(int m, int n, int k, const double* A, const double* B, double* C, int slices,
                                void* workspace, size_t workspace_bytes, void* cuda_stream) {
  if (!oz_args_ok(m, n, k, slices) || !A || !B || !C || !workspace) return TDVP_ERR_INVALID_ARG;
  const OzLayout L = oz_layout(m, n, k, slices);
  if (workspace_bytes < L.total) return TDVP_ERR_INVALID_ARG;
  if (((uintptr_t)workspace & 1023) || ((uintptr_t)A & 15) || ((uintptr_t)B & 15) || ((uintptr_t)C & 15))
    return TDVP_ERR_INVALID_ARG;
  const size_t abytes = 16 * (size_t)m * k, bbytes = 16 * (size_t)k * n, cbytes = 16 * (size_t)m * n;
  if (oz_overlap(C, cbytes, A, abytes) || oz_overlap(C, cbytes, B, bbytes) ||
      oz_overlap(workspace, L.total, A, abytes) || oz_overlap(workspace, L.total, B, bbytes) ||
      oz_overlap(workspace, L.total, C, cbytes))
    return TDVP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  unsigned char* ws = (unsigned char*)workspace;
  int* err = (int*)ws;
  int* eA = (int*)(ws + L.eA);
  int* fB = (int*)(ws + L.fB);
  unsigned char* PA = ws + L.pa;
  unsigned char* PB = ws + L.pb;
  const zc* Az = (const zc*)A;
  const zc* Bz = (const zc*)B;
  const int s = slices;
  const size_t smem = std::max<size_t>((size_t)OZ_STAGES * s * (OZ_A_PLANE + OZ_B_PLANE),
                                       (size_t)OZ_BM * OZ_PART_LD * sizeof(double));
  if (cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return TDVP_ERR_CUDA;
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return TDVP_ERR_CUDA;
  if (cudaMemsetAsync(PA, 0, (size_t)L.pa_bytes, st) != cudaSuccess) return TDVP_ERR_CUDA;
  if (cudaMemsetAsync(PB, 0, (size_t)L.pb_bytes, st) != cudaSuccess) return TDVP_ERR_CUDA;
  oz_row_exp_kernel<<<(m + 7) / 8, 256, 0, st>>>(m, k, Az, eA);
  oz_fill_kernel<<<(n + 255) / 256, 256, 0, st>>>(fB, n, INT_MIN);
  oz_col_exp_kernel<<<dim3((n + 127) / 128, (k + 63) / 64), 128, 0, st>>>(k, n, Bz, fB);
  const long long na = 4LL * m * k, nb = 2LL * k * n;
  oz_pack_a_kernel<<<(unsigned)((na + 255) / 256), 256, 0, st>>>(m, k, s, Az, eA, PA);
  oz_pack_b_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(k, n, s, Bz, fB, PB);
  const dim3 grid((n + OZ_BN - 1) / OZ_BN, (2 * m + OZ_BM - 1) / OZ_BM);
  oz_gemm_kernel<<<grid, OZ_THREADS, smem, st>>>(m, n, k, s, PA, PB, eA, fB, (zc*)C, err);
  return cudaGetLastError() == cudaSuccess ? TDVP_OK : TDVP_ERR_CUDA;
}

extern "C" int tdvp_zgemm_ozaki_status(const void* workspace, void* cuda_stream) {
  if (!workspace) return TDVP_ERR_INVALID_ARG;
  int e = 0;
  if (cudaMemcpyAsync(&e, workspace, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)cuda_stream) != cudaSuccess)
    return TDVP_ERR_CUDA;
  if (cudaStreamSynchronize((cudaStream_t)cuda_stream) != cudaSuccess) return TDVP_ERR_CUDA;
  return e == 0 ? TDVP_OK : TDVP_ERR_DEVICE_TIMEOUT;
}
