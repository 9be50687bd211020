// Mixed-precision contractions of the Lanczos matvecs on the 5th-generation tensor cores.
//
// H[i] C (Eq. tdvp2_C) and the zero-site H0 D (Eq. tdvp2_D) are complex GEMMs.  Each runs as real
// products on tcgen05 (kind::tf32 with TF32 operands, or kind::f16 with BF16 operands) with FP32
// accumulation in tensor memory.  A precision mode word selects the form (TC_PM_* bits):
//   4M:    Dr += Ar Br - Ai Bi,   Di += Ai Br + Ar Bi      (4 real products; A-negate gives -Ai)
//   3M:    P1 += Ar Br,  P2 += Ai Bi,  P3 += (Ar + Ai)(Br + Bi),  Dr = P1 - P2,  Di = P3 - P1 - P2
//          (Gauss: 3 real products; the sum planes are formed in FP64 and rounded once)
//   split: every operand a = a_hi + a_lo (a_hi = a rounded to the operand format) and the terms
//          hi*hi + hi*lo + lo*hi of the 4M form are accumulated (compensated products)
//
// Operands are produced by the pack kernels below directly in the tensor-core tile layout: a
// matrix with R rows (R = 128 for the A operand, 64 for B) and K columns is cut into R x 32 tiles,
// each stored contiguously in K-major "no swizzle" core-matrix order (8 rows x 16 bytes per core
// matrix; core matrices adjacent in K are 128 bytes apart, 8-row groups 1024 bytes apart for TF32
// and 512 for BF16), planes re_hi, im_hi, re_lo, im_lo (3M: re, im, re + im) one after another in
// slots of the TF32 tile size.  Padding rows/columns are zero.  A whole tile is therefore one
// contiguous block that a 1-D bulk TMA copy moves into shared memory.
//
// GEMM kernel: 160 threads per CTA and S CTAs per 128 x 64 output tile, each over its own range
// of K tiles (split-K; S = 1 when the output alone fills the GPU).  One thread of warp 4 issues
// the bulk copies (two-stage ring, mbarrier with transaction bytes) and the MMAs (tcgen05.mma,
// commit to mbarriers).  The main products of each K tile go into a fresh tensor-memory
// accumulator (two alternate), which warps 0-3 add into FP32 registers (tcgen05.ld) while the
// next tile is multiplied: the tensor cores accumulate with truncation, and a sum over all of K
// of same-signed terms (environment diagonals) would drift low by about K/8 half-ulps, whereas
// the register sums round to nearest.  The compensation terms keep one accumulator.  The rows
// then go into shared memory, which the copies no longer use.  The S CTAs of a tile form one thread-block cluster: after a cluster
// barrier CTA q sums rows [q*128/S, (q+1)*128/S) of all S partial tiles, read through distributed
// shared memory in the fixed order 0..S-1 (deterministic), and writes them with coalesced stores.
// Every wait is bounded: on timeout the CTA records an error, drains its copies and MMAs with
// bounded waits, still takes part in the cluster barriers, frees its tensor memory and returns.
#include "tdvp_internal.cuh"
#include "tc_pack.cuh"
#include "tc_ptx.cuh"
#include <cstdint>

namespace {

using tcpack::BM;
using tcpack::BN;
using tcpack::BK;
using tcpack::NPL;
using tcpack::pm_split;
using tcpack::pm_bf16;
using tcpack::pm_gauss;
using tcpack::pm_planes;
using tcpack::pk_store;
constexpr int A_TILE = BM * BK * 4;     // 16 KB per plane
constexpr int B_TILE = BN * BK * 4;     //  8 KB per plane
constexpr int STAGE_BYTES = NPL * (A_TILE + B_TILE);   // 96 KB
constexpr int STAGES = 2;
constexpr int TC_EPI = 128;             // warps 0-3: accumulator drains and epilogue (one TMEM lane each)
constexpr int TC_THREADS = TC_EPI + 32; // warp 4: bulk copies and MMAs
// tensor memory: main accumulators 0 and 1 (hi*hi products of alternate K tiles) at columns
// 0..127 and 128..255, the compensation terms (hi*lo + lo*hi) at 256..383; Dr then Di in each
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t ACC_SMALL = 256;

// instruction descriptor, D = F32, K-major, M = 128, N = 64: kind::tf32 with A = B = TF32 (format
// 2), or kind::f16 with A = B = BF16 (format 1)
__device__ __forceinline__ uint32_t idesc_tf32(bool negA) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((negA ? 1u : 0u) << 13) | ((uint32_t)(BN >> 3) << 17) |
         ((uint32_t)(BM >> 4) << 24);
}
__device__ __forceinline__ uint32_t idesc_bf16(bool negA) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((negA ? 1u : 0u) << 13) | ((uint32_t)(BN >> 3) << 17) |
         ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ int cdivd(int a, int b) { return (a + b - 1) / b; }

struct TcDesc {
  const char* A;     // packed, 128-row tiles
  const char* B;     // packed, 64-row tiles
  int M, N, K;       // logical sizes
  int mode;          // 0: planar FP32 (Cr, Ci), 1: complex FP64 (C64), 2: packed A of the next GEMM,
                     // 3: environment, column (w c) of row i to C64[(w Dc + i) Dc + c]
  int lanczos;       // 1: a stage of a Lanczos matvec (skipped once the solve is done)
  float* Cr;
  float* Ci;
  zc* C64;
  int ldc;
  char* P;           // mode 2 target
  int pDb, pnkt;     // mode 2: row m = w*Db + l' -> (l', w*Db + n); mode 3: pDb = Dc
};

// operands of the four tensor-core GEMMs, derived on the device from the site tables
__device__ bool tc_desc(int op, int site, const SiteDev* sdr, const WorkDev& W, TcDesc& g) {
  const SiteDev& s = sdr[site];
  g.lanczos = op <= TC_Z3 ? 1 : 0;
  switch (op) {
    case TC_MV1:   // T1[(w a')][(s b)] = sum_a L[w][a'][a] x[a][(s b)]
      g.A = W.tc_l; g.B = W.tc_x;
      g.M = s.Wl * s.Dl; g.N = s.d * s.Dr; g.K = s.Dl;
      g.mode = 0; g.Cr = W.tc_t1; g.Ci = W.tc_t1 + W.tc_t1_plane; g.ldc = s.d * s.Dr;
      return true;
    case TC_MV3:   // w[(a' s')][b'] = sum_{w',b} T2[(a' s')][(w' b)] R[w'][b'][b]
      g.A = W.tc_t2; g.B = W.tc_r;
      g.M = s.Dl * s.d; g.N = s.Dr; g.K = s.Wr * s.Dr;
      g.mode = 1; g.C64 = W.w; g.ldc = s.Dr;
      return true;
    case TC_Z1: {  // bond (site, site+1): T[(w l')][r] = sum_l Lb[w][l'][l] D[l][r]  -> packed A of Z3
      const int Db = s.Dr, Wb = s.Wr;
      g.A = W.tc_l; g.B = W.tc_x;
      g.M = Wb * Db; g.N = Db; g.K = Db;
      g.mode = 2; g.P = W.tc_t2; g.pDb = Db; g.pnkt = cdivd(Wb * Db, BK);
      return true;
    }
    case TC_Z3: {  // w[l'][r'] = sum_{w,r} T[l'][(w r)] Rb[w][r'][r]
      const int Db = s.Dr, Wb = s.Wr;
      g.A = W.tc_t2; g.B = W.tc_r;
      g.M = Db; g.N = Db; g.K = Wb * Db;
      g.mode = 1; g.C64 = W.w; g.ldc = Db;
      return true;
    }
    case TC_EL1:   // T1[(w l')][(s r)] = sum_l L[w][l'][l] A[l][(s r)]
      g.A = W.tc_l; g.B = W.tc_x;
      g.M = s.Wl * s.Dl; g.N = s.d * s.Dr; g.K = s.Dl;
      g.mode = 0; g.Cr = W.tc_t1; g.Ci = W.tc_t1 + W.tc_t1_plane; g.ldc = s.d * s.Dr;
      return true;
    case TC_EL3:   // Lenv(i+1)[w'][r'][r] = sum_{(l' s')} conj(A[(l' s')][r']) T2[(l' s')][(w' r)]
      g.A = W.tc_e1; g.B = W.tc_e2;
      g.M = s.Dr; g.N = s.Wr * s.Dr; g.K = s.Dl * s.d;
      g.mode = 3; g.C64 = sdr[site + 1].Lenv; g.pDb = s.Dr;
      return true;
    case TC_ER1:   // T1[(l s)][(w' r')] = sum_r A[(l s)][r] R[w'][r'][r]
      g.A = W.tc_e1; g.B = W.tc_e2;
      g.M = s.Dl * s.d; g.N = s.Wr * s.Dr; g.K = s.Dr;
      g.mode = 0; g.Cr = W.tc_t1; g.Ci = W.tc_t1 + W.tc_t1_plane; g.ldc = s.Wr * s.Dr;
      return true;
    case TC_ER3:   // Renv(i-1)[w][l'][l] = sum_{(s' r')} conj(A[l'][(s' r')]) T2[w][l][(s' r')]
      g.A = W.tc_e1; g.B = W.tc_e2;
      g.M = s.Dl; g.N = s.Wl * s.Dl; g.K = s.d * s.Dr;
      g.mode = 3; g.C64 = sdr[site - 1].Renv; g.pDb = s.Dl;
      return true;
  }
  return false;
}

constexpr int PART_LD = BN + 1;       // partial tile row stride in floats (conflict-free columns)
constexpr int MAX_SPLIT = 8;
static_assert(2 * BM * PART_LD * 4 <= STAGE_BYTES, "partial tile must fit in the first stage");

// PM: precision mode word (TC_PM_* bits), a template parameter so that every mode gets its own
// register allocation
template <int PM>
__global__ void __launch_bounds__(TC_THREADS, 1)
tc_cgemm_kernel(int op, int site, const SiteDev* __restrict__ sd, const WorkDev* __restrict__ wk, int N_sites,
                int S) {
  constexpr int pm = PM;
  pdl_enter();
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ TcDesc g;
  __shared__ uint64_t full_bar[STAGES];
  __shared__ uint64_t done_bar[STAGES];
  __shared__ uint64_t acc_full[2];     // main accumulator b holds a finished K tile
  __shared__ uint64_t acc_free[2];     // main accumulator b has been drained
  __shared__ uint64_t drain_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int live;
  __shared__ volatile int abort_flag, drain_fail;
  const int r = blockIdx.z / S;
  const int sidx = S > 1 ? (int)cluster_rank() : 0;
  const WorkDev& W = wk[r];
  if (threadIdx.x == 0) {
    const SiteDev* sdr = sd + (long long)r * N_sites;
    live = tc_desc(op, site, sdr, W, g) && !(g.lanczos && W.ks->done) && (int)blockIdx.y * BM < g.M &&
           (int)blockIdx.x * BN < g.N;
    abort_flag = 0;
    drain_fail = 0;
  }
  __syncthreads();
  // the S CTAs of a cluster share realisation and output tile, so all of them leave here or none
  if (!live) return;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (warp == 0) tmem_alloc(&tmem_base, TMEM_COLS);
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&done_bar[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&acc_full[b], 1); mbar_init(&acc_free[b], TC_EPI); }
    mbar_init(&drain_bar, 1);
    mbar_fence_init();
  }
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = tmem_base;
  const int nkt_all = cdivd(g.K, BK);
  const int kt0 = (int)((long long)nkt_all * sidx / S);
  const int nkt = (int)((long long)nkt_all * (sidx + 1) / S) - kt0;
  const int mt = blockIdx.y, nt = blockIdx.x;
  constexpr bool split = pm_split(pm), bf = pm_bf16(pm), gauss = pm_gauss(pm);
  constexpr int npl = pm_planes(pm);
  const uint32_t plane_a = bf ? A_TILE / 2 : A_TILE, plane_b = bf ? B_TILE / 2 : B_TILE;
  const uint32_t stage_tx = (uint32_t)npl * (plane_a + plane_b);
  // main accumulators: 4M Dr, Di (2 x BN columns); 3M P1, P2, P3 (3 x BN), at b * bstride
  const uint32_t bstride = gauss ? 3 * BN : 2 * BN;
  // The tensor cores add into an FP32 accumulator with truncation, so a long sum of same-signed
  // terms (the diagonal of an environment, sum_k |A_k|^2 weighted by the MPO) loses about half an
  // ulp per addition, always downward.  The main products of each K tile therefore go into a fresh
  // accumulator (two, alternating), which warps 0-3 add into FP32 registers with rounding to
  // nearest while the next tile is multiplied; the compensation terms, 2^-11 smaller, keep one
  // accumulator for the whole K range.
  float ar[BN], ai[BN];
#pragma unroll
  for (int q = 0; q < BN; ++q) { ar[q] = 0.f; ai[q] = 0.f; }
  if (warp == TC_EPI / 32) {
    if (lane == 0) {
      auto issue = [&](int kt) {
        const int s = kt % STAGES;
        unsigned char* st = smem + s * STAGE_BYTES;
        mbar_expect_tx(&full_bar[s], stage_tx);
        for (int p = 0; p < npl; ++p) {
          bulk_load(st + p * A_TILE, g.A + ((long long)(mt * nkt_all + kt0 + kt) * NPL + p) * A_TILE, plane_a,
                    &full_bar[s]);
          bulk_load(st + NPL * A_TILE + p * B_TILE, g.B + ((long long)(nt * nkt_all + kt0 + kt) * NPL + p) * B_TILE,
                    plane_b, &full_bar[s]);
        }
      };
      const uint32_t id_pos = bf ? idesc_bf16(false) : idesc_tf32(false);
      const uint32_t id_neg = bf ? idesc_bf16(true) : idesc_tf32(true);
      const uint32_t sbo = bf ? 512u : 1024u;
      // one instruction covers 32 bytes of K per row (8 TF32 or 16 BF16 = 2 core matrices)
      constexpr int ksteps = bf ? BK / 16 : BK / 8;
      const uint32_t sr = tmem + ACC_SMALL, si = sr + BN;
      int issued = 0;
      for (; issued < STAGES && issued < nkt; ++issued) issue(issued);
      for (int kt = 0; kt < nkt && !abort_flag; ++kt) {
        const int s = kt % STAGES, b = kt & 1;
        const uint32_t par = (uint32_t)((kt / STAGES) & 1);
        if (!mbar_wait(&full_bar[s], par)) { abort_flag = 1; break; }
        // main accumulator b is free once the drain of tile kt - 2 has read it
        if (kt >= 2 && !mbar_wait_or(&acc_free[b], (uint32_t)(((kt - 2) >> 1) & 1), &drain_fail)) {
          abort_flag = 1;
          break;
        }
        tc_after();
        const uint32_t dr = tmem + (uint32_t)b * bstride, di = dr + BN, d3 = dr + 2 * BN;
        const uint32_t abase = su32(smem + s * STAGE_BYTES);
        const uint32_t bbase = abase + NPL * A_TILE;
#pragma unroll
        for (int ks = 0; ks < ksteps; ++ks) {
          const uint32_t ko = ks * 256;   // 32 bytes of K per row = 2 core matrices of 128 B
          const uint64_t arh = sdesc(abase + 0 * A_TILE + ko, sbo), aih = sdesc(abase + 1 * A_TILE + ko, sbo);
          const uint64_t brh = sdesc(bbase + 0 * B_TILE + ko, sbo), bih = sdesc(bbase + 1 * B_TILE + ko, sbo);
          const uint32_t acc = ks > 0 ? 1u : 0u;
          if constexpr (gauss) {
            // P1 = Ar Br, P2 = Ai Bi, P3 = (Ar + Ai)(Br + Bi)
            const uint64_t as = sdesc(abase + 2 * A_TILE + ko, sbo), bs = sdesc(bbase + 2 * B_TILE + ko, sbo);
            mma_fmt(bf, dr, arh, brh, id_pos, acc);
            mma_fmt(bf, di, aih, bih, id_pos, acc);
            mma_fmt(bf, d3, as, bs, id_pos, acc);
          } else {
          mma_fmt(bf, dr, arh, brh, id_pos, acc);
          mma_fmt(bf, dr, aih, bih, id_neg, 1u);
          mma_fmt(bf, di, aih, brh, id_pos, acc);
          mma_fmt(bf, di, arh, bih, id_pos, 1u);
          }
          if constexpr (split) {
            const uint32_t accs = (kt > 0 || ks > 0) ? 1u : 0u;
            const uint64_t arl = sdesc(abase + 2 * A_TILE + ko, sbo), ail = sdesc(abase + 3 * A_TILE + ko, sbo);
            const uint64_t brl = sdesc(bbase + 2 * B_TILE + ko, sbo), bil = sdesc(bbase + 3 * B_TILE + ko, sbo);
            mma_fmt(bf, sr, arh, brl, id_pos, accs);
            mma_fmt(bf, sr, arl, brh, id_pos, 1u);
            mma_fmt(bf, sr, aih, bil, id_neg, 1u);
            mma_fmt(bf, sr, ail, bih, id_neg, 1u);
            mma_fmt(bf, si, aih, brl, id_pos, accs);
            mma_fmt(bf, si, ail, brh, id_pos, 1u);
            mma_fmt(bf, si, arh, bil, id_pos, 1u);
            mma_fmt(bf, si, arl, bih, id_pos, 1u);
          }
        }
        mma_commit(&done_bar[s]);
        mma_commit(&acc_full[b]);
        if (issued < nkt) {
          // stage s is refilled once the MMAs that read it have completed
          if (!mbar_wait(&done_bar[s], par)) { abort_flag = 1; break; }
          issue(issued);
          ++issued;
        }
      }
      if (abort_flag) {
        // drain (bounded): the newest copy of every stage, then every MMA issued so far
        for (int s = 0; s < STAGES; ++s) {
          int last = -1;
          for (int kt = 0; kt < issued; ++kt) if (kt % STAGES == s) last = kt;
          if (last >= 0) mbar_wait(&full_bar[s], (uint32_t)((last / STAGES) & 1));
        }
        mma_commit(&drain_bar);
        mbar_wait(&drain_bar, 0);
        atomicExch(W.err, -5);
      }
    }
    __syncwarp();
  } else {
    // drains: warp w reads TMEM lanes 32w..32w+31, thread = output row of the tile
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
    bool ok = true;
    for (int kt = 0; kt < nkt; ++kt) {
      const int b = kt & 1;
      const bool got = mbar_wait_or(&acc_full[b], (uint32_t)((kt >> 1) & 1), &abort_flag);
      if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
      tc_after();
      if constexpr (gauss) {
        // Dr += P1 - P2, Di += P3 - P1 - P2 (in FP32 registers, round to nearest)
#pragma unroll
        for (int cb = 0; cb < BN; cb += 16) {
          float v1[16], v2[16], v3[16];
          tmem_ld16(lane_addr + (uint32_t)b * bstride + cb, v1);
          tmem_ld16(lane_addr + (uint32_t)b * bstride + BN + cb, v2);
          tmem_ld16(lane_addr + (uint32_t)b * bstride + 2 * BN + cb, v3);
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            ar[cb + q] += v1[q] - v2[q];
            ai[cb + q] += v3[q] - v1[q] - v2[q];
          }
        }
      } else {
#pragma unroll
        for (int cb = 0; cb < BN; cb += 16) {
          float v[16];
          tmem_ld16(lane_addr + (uint32_t)b * bstride + cb, v);
#pragma unroll
          for (int q = 0; q < 16; ++q) ar[cb + q] += v[q];
          tmem_ld16(lane_addr + (uint32_t)b * bstride + BN + cb, v);
#pragma unroll
          for (int q = 0; q < 16; ++q) ai[cb + q] += v[q];
        }
      }
      tc_before();
      mbar_arrive(&acc_free[b]);
    }
    if (!ok) {
      if (lane == 0) drain_fail = 1;
    } else if (split && nkt > 0) {
      // every MMA has completed with the last tile's commit
#pragma unroll
      for (int cb = 0; cb < BN; cb += 16) {
        float v[16];
        tmem_ld16(lane_addr + ACC_SMALL + cb, v);
#pragma unroll
        for (int q = 0; q < 16; ++q) ar[cb + q] += v[q];
        tmem_ld16(lane_addr + ACC_SMALL + BN + cb, v);
#pragma unroll
        for (int q = 0; q < 16; ++q) ai[cb + q] += v[q];
      }
    }
  }
  tc_before();
  __syncthreads();
  tc_after();
  // copies and MMAs are all complete here (or drained after an abort)
  const bool ok = !abort_flag && !drain_fail;
  if (!ok && threadIdx.x == 0) atomicExch(W.err, -5);
  // ---- accumulated rows -> shared memory partial tile part[plane][row][col] ----
  float* part = reinterpret_cast<float*>(smem);
  if (warp < TC_EPI / 32) {
    const int row = warp * 32 + lane;
#pragma unroll
    for (int q = 0; q < BN; ++q) {
      part[row * PART_LD + q] = ok ? ar[q] : 0.f;
      part[BM * PART_LD + row * PART_LD + q] = ok ? ai[q] : 0.f;
    }
  }
  tc_before();
  if (S > 1) cluster_sync_all(); else __syncthreads();
  // ---- sum of the S partials over this CTA's rows, coalesced epilogue ----
  {
    const int rows = BM / S, row0 = sidx * rows;
    const uint32_t pbase = su32(part);
    uint32_t rbase[MAX_SPLIT];
#pragma unroll
    for (int q = 0; q < MAX_SPLIT; ++q) rbase[q] = (S > 1 && q < S) ? mapa(pbase, (uint32_t)q) : 0u;
    for (int e = threadIdx.x; e < rows * BN; e += TC_THREADS) {
      const int lr = row0 + e / BN, col = e % BN;
      const uint32_t off = (uint32_t)(lr * PART_LD + col) * 4u, offi = off + (uint32_t)(BM * PART_LD) * 4u;
      float vr, vi;
      if (S == 1) {
        vr = part[lr * PART_LD + col];
        vi = part[BM * PART_LD + lr * PART_LD + col];
      } else {
        float ar[MAX_SPLIT], ai[MAX_SPLIT];
#pragma unroll
        for (int q = 0; q < MAX_SPLIT; ++q) {
          ar[q] = q < S ? ld_cluster_f32(rbase[q] + off) : 0.f;
          ai[q] = q < S ? ld_cluster_f32(rbase[q] + offi) : 0.f;
        }
        vr = ar[0];
        vi = ai[0];
#pragma unroll
        for (int q = 1; q < MAX_SPLIT; ++q)
          if (q < S) { vr += ar[q]; vi += ai[q]; }
      }
      const int row = mt * BM + lr, gcol = nt * BN + col;
      if (ok && row < g.M && gcol < g.N) {
        if (g.mode == 0) {
          g.Cr[(long long)row * g.ldc + gcol] = vr;
          g.Ci[(long long)row * g.ldc + gcol] = vi;
        } else if (g.mode == 1) {
          g.C64[(long long)row * g.ldc + gcol] = zmake((double)vr, (double)vi);
        } else if (g.mode == 3) {
          const int Dc = g.pDb, w = gcol / Dc, c = gcol % Dc;
          g.C64[((long long)w * Dc + row) * Dc + c] = zmake((double)vr, (double)vi);
        } else {
          const int w = row / g.pDb, lp = row % g.pDb;
          pk_store(g.P, BM, g.pnkt, lp, w * g.pDb + gcol, (double)vr, (double)vi, pm);
        }
      }
    }
  }
  // no CTA leaves (or frees its tensor memory) while another may still read its shared memory
  if (S > 1) cluster_sync_all(); else __syncthreads();
  tc_after();
  if (warp == 0) tmem_free(tmem, TMEM_COLS);
}

// ---- pack kernels (all write only the valid region; the targets are zeroed beforehand) ----

// Lenv[site] stacked as the A operand: row = w*Dl + a', k = a
__global__ void pack_env_l_kernel(int site, const SiteDev* __restrict__ sd, const WorkDev* __restrict__ wk,
                                  int N_sites, int pm) {
  pdl_enter();
  const int r = blockIdx.y;
  const SiteDev& s = sd[(long long)r * N_sites + site];
  const WorkDev& W = wk[r];
  const int M = s.Wl * s.Dl, K = s.Dl, nkt = cdivd(K, BK);
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)M * K) return;
  const int row = (int)(e / K), k = (int)(e % K);
  const zc v = s.Lenv[e];          // [w][a'][a] row-major = [(w a')][a]
  pk_store(W.tc_l, BM, nkt, row, k, v.x, v.y, pm);
}

// Renv[site] as the B operand: row = b', k = w*Dr + b
__global__ void pack_env_r_kernel(int site, const SiteDev* __restrict__ sd, const WorkDev* __restrict__ wk,
                                  int N_sites, int pm) {
  pdl_enter();
  const int r = blockIdx.y;
  const SiteDev& s = sd[(long long)r * N_sites + site];
  const WorkDev& W = wk[r];
  const int Dr = s.Dr, K = s.Wr * Dr, nkt = cdivd(K, BK);
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)s.Wr * Dr * Dr) return;
  const int w = (int)(e / ((long long)Dr * Dr)), rem = (int)(e % ((long long)Dr * Dr));
  const int bp = rem / Dr, b = rem % Dr;
  const zc v = s.Renv[e];          // [w][b'][b]
  pk_store(W.tc_r, BN, nkt, bp, w * Dr + b, v.x, v.y, pm);
}

// x as the B operand.  kind 0 (site): row = (s b), k = a;  kind 1 (bond D[l][r]): row = r, k = l
__global__ void pack_x_kernel(int kind, int site, const SiteDev* __restrict__ sd, const WorkDev* __restrict__ wk,
                              int N_sites, int pm) {
  pdl_enter();
  const int r = blockIdx.y;
  const SiteDev& s = sd[(long long)r * N_sites + site];
  const WorkDev& W = wk[r];
  if (W.ks->done) return;
  const int Kd = kind == 0 ? s.Dl : s.Dr;
  const int Nn = kind == 0 ? s.d * s.Dr : s.Dr;
  const int nkt = cdivd(Kd, BK);
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)Kd * Nn) return;
  const int k = (int)(e / Nn), n = (int)(e % Nn);
  const zc v = W.x[e];
  pk_store(W.tc_x, BN, nkt, n, k, v.x, v.y, pm);
}

// Sparse MPO middle stage from the planar FP32 T1 into the packed A operand of the third GEMM:
// T2[(a' s')][(w' b)] = sum_e val * T1[(w a')][(s b)]  over the CSR row (w', s').
__global__ void wapply_tc_kernel(int site, const SiteDev* __restrict__ sd, const WorkDev* __restrict__ wk,
                                 int N_sites, int pm) {
  pdl_wait();
  const int r = blockIdx.z;
  const SiteDev& s = sd[(long long)r * N_sites + site];
  const WorkDev& W = wk[r];
  if (W.ks->done) return;
  const int row = blockIdx.y;           // (w', s')
  const int d = s.d, Dl = s.Dl, Dr = s.Dr;
  if (row >= s.Wr * d) return;
  const int xy = blockIdx.x * blockDim.x + threadIdx.x;
  if (xy >= Dl * Dr) return;
  const int ap = xy / Dr, b = xy % Dr;
  const int wp = row / d, sp = row % d;
  const float* T1r = W.tc_t1;
  const float* T1i = W.tc_t1 + W.tc_t1_plane;
  const long long ld = (long long)d * Dr;
  double ar = 0, ai = 0;
  for (int e = s.fw.ptr[row]; e < s.fw.ptr[row + 1]; ++e) {
    const long long off = ((long long)s.fw.ci[e] * Dl + ap) * ld + (long long)s.fw.si[e] * Dr + b;
    ar += s.fw.val[e] * (double)T1r[off];
    ai += s.fw.val[e] * (double)T1i[off];
  }
  const int nkt = cdivd(s.Wr * Dr, BK);
  pk_store(W.tc_t2, BM, nkt, ap * d + sp, wp * Dr + b, ar, ai, pm);
}

// Site tensor of an environment update as a packed operand; the grid covers the padded tiles.
//   kind 0: A^H as A operand, row r', k (l s);    kind 1: A as A operand, row (l s), k r
//   kind 2: conj(A) as A operand, row l', k (s r); kind 3: A as B operand, row (s r), k l
__global__ void pack_site_kernel(int kind, int site, const SiteDev* __restrict__ sd, const WorkDev* __restrict__ wk,
                                 int N_sites, int pm) {
  pdl_wait();
  const int r = blockIdx.y;
  const SiteDev& s = sd[(long long)r * N_sites + site];
  const WorkDev& W = wk[r];
  const int Dl = s.Dl, d = s.d, Dr = s.Dr;
  int rows, K, RT;
  char* dst;
  switch (kind) {
    case 0: rows = Dr; K = Dl * d; RT = BM; dst = W.tc_e1; break;
    case 1: rows = Dl * d; K = Dr; RT = BM; dst = W.tc_e1; break;
    case 2: rows = Dl; K = d * Dr; RT = BM; dst = W.tc_e1; break;
    default: rows = d * Dr; K = Dl; RT = BN; dst = W.tc_x; break;
  }
  const int rp = cdivd(rows, RT) * RT, kp = cdivd(K, BK) * BK;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rp * kp) return;
  const int row = (int)(e / kp), k = (int)(e % kp);
  zc v = zmake(0, 0);
  if (row < rows && k < K) {
    switch (kind) {
      case 0: v = zconj(s.A[(long long)k * Dr + row]); break;
      case 1: v = s.A[(long long)row * Dr + k]; break;
      case 2: v = zconj(s.A[(long long)row * d * Dr + k]); break;
      default: v = s.A[(long long)k * d * Dr + row]; break;
    }
  }
  pk_store(dst, RT, cdivd(K, BK), row, k, v.x, v.y, pm);
}

// Renv[site] as the B operand of the right-update first stage: row (w' r'), k r.
__global__ void pack_renv_rows_kernel(int site, const SiteDev* __restrict__ sd, const WorkDev* __restrict__ wk,
                                      int N_sites, int pm) {
  pdl_wait();
  const int r = blockIdx.y;
  const SiteDev& s = sd[(long long)r * N_sites + site];
  const WorkDev& W = wk[r];
  const int Dr = s.Dr, rows = s.Wr * Dr, K = Dr;
  const int rp = cdivd(rows, BN) * BN, kp = cdivd(K, BK) * BK;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rp * kp) return;
  const int row = (int)(e / kp), k = (int)(e % kp);
  const zc v = (row < rows && k < K) ? s.Renv[(long long)row * Dr + k] : zmake(0, 0);
  pk_store(W.tc_e2, BN, cdivd(K, BK), row, k, v.x, v.y, pm);
}

// Sparse MPO stage of an environment update from the planar FP32 first-stage output, written as
// the packed B operand of the last stage (one output element per thread, padded tiles included).
//   which 0 (left):  T2[(l' s')][(w' r)] = sum_e val T1[(w l')][(s r)] over the forward CSR row
//                    (w', s'); B row (w' r), k (l' s').
//   which 1 (right): T2[w][(l s')][r'] = sum_e val T1[(l s)][(w' r')] over the backward CSR row
//                    (w, s'); B row (w l), k (s' r').
__global__ void wapply_env_kernel(int which, int site, const SiteDev* __restrict__ sd,
                                  const WorkDev* __restrict__ wk, int N_sites, int pm) {
  pdl_wait();
  const int r = blockIdx.y;
  const SiteDev& s = sd[(long long)r * N_sites + site];
  const WorkDev& W = wk[r];
  const int Dl = s.Dl, d = s.d, Dr = s.Dr;
  const int rows = which == 0 ? s.Wr * Dr : s.Wl * Dl;
  const int K = which == 0 ? Dl * d : d * Dr;
  const int rp = cdivd(rows, BN) * BN, kp = cdivd(K, BK) * BK;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rp * kp) return;
  const int row = (int)(e / kp), k = (int)(e % kp);
  double ar = 0, ai = 0;
  if (row < rows && k < K) {
    const float* T1r = W.tc_t1;
    const float* T1i = W.tc_t1 + W.tc_t1_plane;
    if (which == 0) {
      const int wp = row / Dr, b = row % Dr, ap = k / d, sp = k % d;
      const int crow = wp * d + sp;
      const long long ld = (long long)d * Dr;
      for (int q = s.fw.ptr[crow]; q < s.fw.ptr[crow + 1]; ++q) {
        const long long off = ((long long)s.fw.ci[q] * Dl + ap) * ld + (long long)s.fw.si[q] * Dr + b;
        ar += s.fw.val[q] * (double)T1r[off];
        ai += s.fw.val[q] * (double)T1i[off];
      }
    } else {
      const int w = row / Dl, l = row % Dl, sp = k / Dr, rr = k % Dr;
      const int crow = w * d + sp;
      const long long ld = (long long)s.Wr * Dr;
      for (int q = s.bw.ptr[crow]; q < s.bw.ptr[crow + 1]; ++q) {
        const long long off = ((long long)l * d + s.bw.si[q]) * ld + (long long)s.bw.ci[q] * Dr + rr;
        ar += s.bw.val[q] * (double)T1r[off];
        ai += s.bw.val[q] * (double)T1i[off];
      }
    }
  }
  pk_store(W.tc_e2, BN, cdivd(K, BK), row, k, ar, ai, pm);
}

inline int cdivh(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace

long long tc_pack_bytes(int rows_tile, long long rows, long long K) {
  return (long long)cdivh(rows, rows_tile) * cdivh(K, BK) * NPL * rows_tile * BK * 4;
}

cudaError_t tc_setup() {
  const int smem = STAGES * STAGE_BYTES;
  cudaError_t e = cudaFuncSetAttribute(tc_cgemm_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_cgemm_kernel<TC_PM_SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_cgemm_kernel<TC_PM_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_cgemm_kernel<TC_PM_BF16 | TC_PM_SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_cgemm_kernel<TC_PM_GAUSS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_cgemm_kernel<TC_PM_BF16 | TC_PM_GAUSS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem);
  return e;
}

// K splits per output tile: the largest power of two <= 8 that keeps at least two K tiles per
// CTA and the whole grid within one CTA per SM of the 148
int tc_splits(int tiles, int R, int maxK) {
  const int nkt = cdivh(maxK, BK);
  int S = 1;
  while (2 * S <= MAX_SPLIT && (long long)2 * S * tiles * R <= 148 && nkt >= 4 * S) S *= 2;
  return S;
}

cudaError_t launch_tc_gemm(int op, int site, const SiteDev* sd, const WorkDev* wk, int R, int N_sites, int maxM,
                           int maxN, int maxK, int pm, cudaStream_t st, int S_force) {
  const int tn = cdivh(maxN, BN), tm = cdivh(maxM, BM);
  int S = tc_splits(tn * tm, R, maxK);
  if (S_force > 0) {
    if (S_force > MAX_SPLIT || (S_force & (S_force - 1)) || S_force > cdivh(maxK, BK)) return cudaErrorInvalidValue;
    S = S_force;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  if (S > 1) {
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 1;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = S;
  } else {
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
  }
  cfg.gridDim = dim3(tn, tm, R * S);
  cfg.blockDim = dim3(TC_THREADS);
  cfg.dynamicSmemBytes = STAGES * STAGE_BYTES;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = (S > 1 || g_tdvp_pdl) ? 1 : 0;
  switch (pm) {
    case 0: return cudaLaunchKernelEx(&cfg, tc_cgemm_kernel<0>, op, site, sd, wk, N_sites, S);
    case TC_PM_SPLIT: return cudaLaunchKernelEx(&cfg, tc_cgemm_kernel<TC_PM_SPLIT>, op, site, sd, wk, N_sites, S);
    case TC_PM_BF16: return cudaLaunchKernelEx(&cfg, tc_cgemm_kernel<TC_PM_BF16>, op, site, sd, wk, N_sites, S);
    case TC_PM_BF16 | TC_PM_SPLIT:
      return cudaLaunchKernelEx(&cfg, tc_cgemm_kernel<TC_PM_BF16 | TC_PM_SPLIT>, op, site, sd, wk, N_sites, S);
    case TC_PM_GAUSS: return cudaLaunchKernelEx(&cfg, tc_cgemm_kernel<TC_PM_GAUSS>, op, site, sd, wk, N_sites, S);
    case TC_PM_BF16 | TC_PM_GAUSS:
      return cudaLaunchKernelEx(&cfg, tc_cgemm_kernel<TC_PM_BF16 | TC_PM_GAUSS>, op, site, sd, wk, N_sites, S);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_pack_env(int which, int site, const SiteDev* sd, const WorkDev* wk, int R, int N_sites,
                            long long max_elems, int pm, cudaStream_t st) {
  dim3 grid(cdivh(max_elems, 256), R);
  if (which == 0) { const cudaError_t e_ = launch_pdl(pack_env_l_kernel, grid, 256, 0, st, site, sd, wk, N_sites, pm); if (e_ != cudaSuccess) return e_; }
  else { const cudaError_t e_ = launch_pdl(pack_env_r_kernel, grid, 256, 0, st, site, sd, wk, N_sites, pm); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

cudaError_t launch_pack_x(int kind, int site, const SiteDev* sd, const WorkDev* wk, int R, int N_sites,
                          long long max_elems, int pm, cudaStream_t st) {
  dim3 grid(cdivh(max_elems, 256), R);
  { const cudaError_t e_ = launch_pdl(pack_x_kernel, grid, 256, 0, st, kind, site, sd, wk, N_sites, pm); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

cudaError_t launch_pack_site(int kind, int site, const SiteDev* sd, const WorkDev* wk, int R, int N_sites,
                             long long max_rows, long long max_k, int pm, cudaStream_t st) {
  const int RT = kind == 3 ? BN : BM;
  const long long total = (long long)cdivh(max_rows, RT) * RT * cdivh(max_k, BK) * BK;
  dim3 grid(cdivh(total, 256), R);
  { const cudaError_t e_ = launch_pdl(pack_site_kernel, grid, 256, 0, st, kind, site, sd, wk, N_sites, pm); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

cudaError_t launch_pack_renv_rows(int site, const SiteDev* sd, const WorkDev* wk, int R, int N_sites,
                                  long long max_rows, long long max_k, int pm, cudaStream_t st) {
  const long long total = (long long)cdivh(max_rows, BN) * BN * cdivh(max_k, BK) * BK;
  dim3 grid(cdivh(total, 256), R);
  { const cudaError_t e_ = launch_pdl(pack_renv_rows_kernel, grid, 256, 0, st, site, sd, wk, N_sites, pm); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

cudaError_t launch_wapply_env(int which, int site, const SiteDev* sd, const WorkDev* wk, int R, int N_sites,
                              long long max_rows, long long max_k, int pm, cudaStream_t st) {
  const long long total = (long long)cdivh(max_rows, BN) * BN * cdivh(max_k, BK) * BK;
  dim3 grid(cdivh(total, 256), R);
  { const cudaError_t e_ = launch_pdl(wapply_env_kernel, grid, 256, 0, st, which, site, sd, wk, N_sites, pm); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

cudaError_t launch_wapply_tc(int site, const SiteDev* sd, const WorkDev* wk, int R, int N_sites, int max_xy,
                             int n_rows, int pm, cudaStream_t st) {
  dim3 grid(cdivh(max_xy, 256), n_rows, R);
  { const cudaError_t e_ = launch_pdl(wapply_tc_kernel, grid, 256, 0, st, site, sd, wk, N_sites, pm); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}
