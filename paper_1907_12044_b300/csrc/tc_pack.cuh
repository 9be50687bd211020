// Tensor-core operand packing shared by the tensor-core GEMMs (kernels_tc.cu) and the Lanczos
// kernels (kernels_lanczos.cu), which write the next Krylov vector straight into its packed form.
//
// A matrix with R rows (R = 128 for the A operand, 64 for B) and K columns is cut into R x 32
// tiles, each stored contiguously in K-major "no swizzle" core-matrix order (8 rows x 16 bytes per
// core matrix; core matrices adjacent in K are 128 bytes apart, 8-row groups 1024 bytes apart for
// TF32 and 512 for BF16).  Each tile has NPL plane slots of the TF32 tile size: re_hi, im_hi,
// re_lo, im_lo (split modes), re, im, re + im (3M), or re, im; a BF16 tile fills the first half of
// its slot.  The precision mode word pm holds the TC_PM_* bits.
#pragma once
#include "tdvp_internal.cuh"
#include <cuda_bf16.h>

namespace tcpack {

constexpr int BM = 128, BN = 64, BK = 32;
constexpr int NPL = 4;                  // plane slots per tile

__host__ __device__ constexpr bool pm_split(int pm) { return (pm & TC_PM_SPLIT) != 0; }
__host__ __device__ constexpr bool pm_bf16(int pm) { return (pm & TC_PM_BF16) != 0; }
__host__ __device__ constexpr bool pm_gauss(int pm) { return (pm & TC_PM_GAUSS) != 0; }
// planes of a packed operand: 2 (4M), 3 (3M: re, im, re + im), 4 (split: re_hi, im_hi, re_lo, im_lo)
__host__ __device__ constexpr int pm_planes(int pm) { return pm_split(pm) ? 4 : (pm_gauss(pm) ? 3 : 2); }

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// byte offset of element (row, k) in a packed operand with RT-row tiles and nkt K-tiles; every
// plane of a tile has a slot of the TF32 tile size, a BF16 tile fills the first half of it
__device__ __forceinline__ long long pk_off(int RT, int nkt, int row, int k, int plane, bool bf16) {
  const int rt = row / RT, r = row % RT, kt = k / BK, kk = k % BK;
  const long long tile = ((long long)(rt * nkt + kt) * NPL + plane) * (RT * BK * 4);
  if (bf16) return tile + (r / 8) * 512 + (kk / 8) * 128 + (r % 8) * 16 + (kk % 8) * 2;
  return tile + (r / 8) * 1024 + (kk / 4) * 128 + (r % 8) * 16 + (kk % 4) * 4;
}

__device__ __forceinline__ void pk_put(char* base, long long off, bool bf16, double v, double* rounded) {
  if (bf16) {
    const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
    *reinterpret_cast<__nv_bfloat16*>(base + off) = h;
    if (rounded) *rounded = (double)__bfloat162float(h);
  } else {
    const float h = tf32_round((float)v);
    *reinterpret_cast<float*>(base + off) = h;
    if (rounded) *rounded = (double)h;
  }
}

// store a complex value into the packed planes of precision mode pm
__device__ __forceinline__ void pk_store(char* base, int RT, int nkt, int row, int k, double re, double im, int pm) {
  const bool bf = pm_bf16(pm);
  double rh, ih;
  pk_put(base, pk_off(RT, nkt, row, k, 0, bf), bf, re, &rh);
  pk_put(base, pk_off(RT, nkt, row, k, 1, bf), bf, im, &ih);
  if (pm_split(pm)) {
    if (bf) {
      pk_put(base, pk_off(RT, nkt, row, k, 2, bf), bf, re - rh, nullptr);
      pk_put(base, pk_off(RT, nkt, row, k, 3, bf), bf, im - ih, nullptr);
    } else {
      // the tensor cores read the leading TF32 bits of the FP32 low part
      *reinterpret_cast<float*>(base + pk_off(RT, nkt, row, k, 2, bf)) = (float)(re - rh);
      *reinterpret_cast<float*>(base + pk_off(RT, nkt, row, k, 3, bf)) = (float)(im - ih);
    }
  } else if (pm_gauss(pm)) {
    pk_put(base, pk_off(RT, nkt, row, k, 2, bf), bf, re + im, nullptr);
  }
}

}  // namespace tcpack
