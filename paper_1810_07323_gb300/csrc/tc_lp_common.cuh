// Shared pieces of the kind::f16 streaming passes (pass_tc_lp.cu: one problem,
// Stream-K; pass_tc_lp_grouped.cu: a table of problems, fixed work units): tile
// shapes, the BF16 instruction descriptor and MMA, FP8 e4m3 -> BF16 conversion,
// and one stage of the converter warps (FP8 dequantisation with the 128 x 128
// tile scales into the BF16 operand tile, and/or the sum of squares of A).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "tc_common.cuh"

namespace corutv {
namespace lpk {

constexpr int kBN = 256;             // output positions per tile (MMA N)
constexpr int kM = 128;              // MMA M (sketch columns, padded)
constexpr int kBK = 64;              // elements of K per stage (one 128-byte row of BF16)
constexpr int kATile = kBN * kBK * 2;        // 32 KB BF16 A tile (K-major, 128-byte swizzle)
constexpr int kXTile = kM * kBK * 2;         // 16 KB per BF16 X part
constexpr int kF8Tile = kBN * kBK;           // 16 KB FP8 staging tile
constexpr int kMaxThreads = 448;     // 0 TMA, 1 MMA, 2..5 epilogue, 6.. converter (4 BF16, 8 FP8 warps)

template <bool FP8>
struct LpCfg {
  static constexpr int kStage = kATile + 2 * kXTile + (FP8 ? kF8Tile : 0);
  static constexpr int kStages = FP8 ? 2 : 3;
  static constexpr int kTx = (FP8 ? kF8Tile : kATile) + 2 * kXTile;
  static constexpr int kSmem = kStages * kStage + 1024 + 512;
  // FP8 tiles are dequantised element by element: twice the converter warps keep two per SM
  // sub-partition issuing; BF16 converters only sum squares
  static constexpr int kConvWarps = FP8 ? 8 : 4;
  static constexpr int kThreads = 192 + 32 * kConvWarps;
};

// kind::f16 instruction descriptor: D fp32, A/B BF16 (1), A K-major, B K-major or (b_mn) MN-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool b_mn = false) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((b_mn ? 1u : 0u) << 16) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ float bf16lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

// 8 FP8 e4m3 values (a uint2) times `s` -> 8 floats
__device__ __forceinline__ void fp8x8_to_float(uint2 raw, float s, float (&f)[8]) {
  const uint32_t w[2] = {raw.x, raw.y};
#pragma unroll
  for (int q = 0; q < 2; ++q) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const __nv_fp8x2_storage_t pair = (__nv_fp8x2_storage_t)((w[q] >> (16 * h)) & 0xFFFFu);
      const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(pair, __NV_E4M3);
      __half2 h2;
      h2 = *reinterpret_cast<const __half2*>(&hr);
      const float2 v = __half22float2(h2);
      f[4 * q + 2 * h] = v.x * s;
      f[4 * q + 2 * h + 1] = v.y * s;
    }
  }
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 p = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&p);
}

// FP8 tile scales a converter thread needs for the stage at k-block kb of the output tile that
// starts at position p0 -- A X (dir 0): the two 128-row tile rows of the 256 positions; A^T Y
// (dir 1): the tile column of the thread's eight positions (c8 = ct mod 32 in every stage).
__device__ __forceinline__ void lp_stage_scales(const float* scales, int64_t sld, int64_t srows, int64_t scols,
                                                int dir, int64_t kb, int64_t p0, int ct, float& a, float& b) {
  const int64_t kcol = (kb * kBK) >> 7;
  if (dir == 0) {
    const int64_t tr0 = p0 >> 7, tr1 = tr0 + 1 < srows ? tr0 + 1 : tr0;
    a = scales[tr0 * sld + kcol];
    b = scales[tr1 * sld + kcol];
  } else {
    int64_t tc = (p0 + 8 * (ct & 31)) >> 7;
    if (tc >= scols) tc = scols - 1;
    a = b = scales[kcol * sld + tc];
  }
}

// One stage of the CT converter threads (ct in [0, CT)).  BF16: the tile is read as TMA landed it
// and only sum(a^2) is formed.  FP8, A X: staging [256 rows][64 B] -> BF16 [256 rows][64] with the
// 128-byte swizzle, times the tile scale (rows < 128: sca, else scb; the 64 columns lie in one tile
// column).  FP8, A^T Y: staging [64 k][256 B] -> BF16 MN-major, row k of the 64-position block c at
// c * 8 KB + 128 k (128-byte swizzle), times sca (the 64 k rows lie in one tile row and 8
// consecutive positions in one tile column).  Returns this thread's FP32 sum of squares (FRO).
template <bool FP8, bool FRO, int CT>
__device__ __forceinline__ float lp_convert_stage(uint8_t* at, const uint8_t* f8, int dir, float sca, float scb,
                                                  int ct) {
  float part = 0.f;
  if (!FP8) {
    if (!FRO) return 0.f;
    const uint4* a4 = reinterpret_cast<const uint4*>(at);
#pragma unroll 4
    for (int q = ct; q < kATile / 16; q += CT) {
      const uint4 v = a4[q];
      const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float lo = bf16lo(w[i]), hi = bf16hi(w[i]);
        part = fmaf(lo, lo, fmaf(hi, hi, part));
      }
    }
  } else if (dir == 0) {
#pragma unroll 4
    for (int u = ct; u < kBN * 8; u += CT) {
      const int r = u >> 3, c8 = u & 7;
      const float sc = r < 128 ? sca : scb;
      float f[8];
      fp8x8_to_float(*reinterpret_cast<const uint2*>(f8 + r * 64 + 8 * c8), sc, f);
      if (FRO)
#pragma unroll
        for (int i = 0; i < 8; ++i) part = fmaf(f[i], f[i], part);
      uint4 o;
      o.x = pack_bf16(f[0], f[1]); o.y = pack_bf16(f[2], f[3]);
      o.z = pack_bf16(f[4], f[5]); o.w = pack_bf16(f[6], f[7]);
      *reinterpret_cast<uint4*>(at + r * 128 + ((c8 ^ (r & 7)) << 4)) = o;
    }
  } else {
#pragma unroll 4
    for (int u = ct; u < kBK * (kBN / 8); u += CT) {
      const int k = u >> 5, c8 = u & 31;
      float f[8];
      fp8x8_to_float(*reinterpret_cast<const uint2*>(f8 + k * kBN + 8 * c8), sca, f);
      if (FRO)
#pragma unroll
        for (int i = 0; i < 8; ++i) part = fmaf(f[i], f[i], part);
      uint4 o;
      o.x = pack_bf16(f[0], f[1]); o.y = pack_bf16(f[2], f[3]);
      o.z = pack_bf16(f[4], f[5]); o.w = pack_bf16(f[6], f[7]);
      const int c = c8 >> 3, ch = c8 & 7;
      *reinterpret_cast<uint4*>(at + c * (kBK * 128) + k * 128 + ((ch ^ (k & 7)) << 4)) = o;
    }
  }
  return part;
}

}  // namespace lpk
}  // namespace corutv
