// Tensor-core streaming passes for A stored in BF16 or in FP8 e4m3 with one
// FP32 scale per 128 x 128 tile (the precision modes of the hot path):
//     Ct (l x len) = X^T op(A)   as in pass_tc.cu,
// with tcgen05.mma kind::f16 on BF16 operands and FP32 accumulation in TMEM.
// A in BF16 is exact; the FP32 sketch operand is split X = X_hi + X_lo into two
// BF16 parts (both products accumulate in the same TMEM tile), so each product
// keeps ~16 bits of X.  FP8 tiles are dequantised with their tile scale into
// BF16 in shared memory by converter warps.  A X reads A tiles K-major (rows of
// A); A^T Y reads them MN-major (the tile as TMA lands it: rows of A are the K
// direction, 64 positions per 128-byte swizzled row, four such 8 KB blocks side
// by side), so no tile is transposed.  Stream-K split, bounded waits and the
// epilogue are those of pass_tc.cu.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace corutv {

namespace {

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

struct LpArgs {
  float* Ct;
  int64_t ldc;
  float* partials;
  int64_t len, K;
  int l;
  DevStatus* status;
  double* fro_parts;
  const float* scales;   // FP8 tile scales, row-major srows x scols, leading dimension sld
  int64_t sld;
  int64_t srows, scols;  // ceil(m/128), ceil(n/128)
};

template <int DIR, bool FP8, bool FRO>
__global__ void __launch_bounds__(kMaxThreads, 1)
    pass_tc_lp_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapXh,
                      const __grid_constant__ CUtensorMap mapXl, LpArgs args) {
  using Cfg = LpCfg<FP8>;
  constexpr int S = Cfg::kStages;
  constexpr bool kConv = FP8 || FRO;
  extern __shared__ uint8_t smem_dyn[];
  uint8_t* smem = smem_dyn + ((1024u - (smem_u32(smem_dyn) & 1023u)) & 1023u);
  // stage s: [A bf16 | X_hi | X_lo | (FP8 staging)]
  auto a_tile = [&](int st) { return smem + st * Cfg::kStage; };
  auto xh_tile = [&](int st) { return smem + st * Cfg::kStage + kATile; };
  auto xl_tile = [&](int st) { return smem + st * Cfg::kStage + kATile + kXTile; };
  auto f8_tile = [&](int st) { return smem + st * Cfg::kStage + kATile + 2 * kXTile; };
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * Cfg::kStage);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * S + 4);
  double* fro_red = reinterpret_cast<double*>(bars + 3 * S + 6);
  volatile int* conv_abort = reinterpret_cast<volatile int*>(fro_red + 8);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + S), conv0 = smem_u32(bars + 2 * S);
  const uint32_t tfull0 = smem_u32(bars + 3 * S), tempty0 = smem_u32(bars + 3 * S + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t KB = cdiv(args.K, kBK);
  StreamK sk(cdiv(args.len, kBN), KB, gridDim.x);
  const int64_t s = sk.start(blockIdx.x), e = sk.start(blockIdx.x + 1);

  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(full0 + 8 * i, 1);
      mbar_init(empty0 + 8 * i, 1);
      mbar_init(conv0 + 8 * i, Cfg::kConvWarps);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      mbar_init(tempty0 + 8 * b, 4);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      const uint64_t pol_a = policy_evict_first(), pol_x = policy_evict_last();
      int64_t n = 0;
      bool ok = true;
      for (int64_t it = s; it < e; ++it, ++n) {
        const int stage = (int)(n % S);
        const uint32_t ph = (uint32_t)((n / S) & 1);
        if (!mbar_wait(empty0 + 8 * stage, ph ^ 1, args.status)) { ok = false; break; }
        const int64_t t = it / KB, kb = it - t * KB;
        const int k0 = (int)(kb * kBK);
        const int p0 = (int)(t * kBN);
        const uint32_t fb = full0 + 8 * stage;
        mbar_arrive_expect_tx(fb, Cfg::kTx);
        if (FP8) {
          if (DIR == 0) tma_load_2d(smem_u32(f8_tile(stage)), &mapA, fb, k0, p0, pol_a);    // 256 rows x 64 B
          else tma_load_2d(smem_u32(f8_tile(stage)), &mapA, fb, p0, k0, pol_a);             // 64 rows x 256 B
        } else {
          if (DIR == 0) {
            tma_load_2d(smem_u32(a_tile(stage)), &mapA, fb, k0, p0, pol_a);                 // 256 rows x 64
          } else {
#pragma unroll
            for (int c = 0; c < kBN / 64; ++c)                                              // 4 x (64 rows x 64)
              tma_load_2d(smem_u32(a_tile(stage)) + c * (kBK * 128), &mapA, fb, p0 + 64 * c, k0, pol_a);
          }
        }
        tma_load_2d(smem_u32(xh_tile(stage)), &mapXh, fb, k0, 0, pol_x);
        tma_load_2d(smem_u32(xl_tile(stage)), &mapXl, fb, k0, 0, pol_x);
      }
      const int64_t first = n > S ? n - S : 0;
      for (int64_t f = first; f < n; ++f) {
        const int stage = (int)(f % S);
        const uint32_t ph = (uint32_t)((f / S) & 1);
        if (ok) {
          if (!mbar_wait(empty0 + 8 * stage, ph, args.status)) ok = false;
        }
        if (!ok) mbar_wait(full0 + 8 * stage, ph, args.status);
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(kM, kBN, DIR == 1);
      const uint32_t ready0 = kConv ? conv0 : full0;
      int64_t n = 0;
      int seg = 0;
      bool ok = true;
      int64_t it = s;
      while (it < e && ok) {
        const int64_t t = it / KB;
        const int64_t kb1 = (e - t * KB < KB) ? (e - t * KB) : KB;
        const int b = seg & 1;
        const uint32_t tph = (uint32_t)((seg >> 1) & 1);
        if (!mbar_wait(tempty0 + 8 * b, tph ^ 1, args.status)) { ok = false; break; }
        tc_fence_after();
        const uint32_t tacc = tmem_base + (uint32_t)(b * kBN);
        bool first = true;
        for (; it < t * KB + kb1; ++it, ++n) {
          const int stage = (int)(n % S);
          const uint32_t ph = (uint32_t)((n / S) & 1);
          if (!mbar_wait(ready0 + 8 * stage, ph, args.status)) { ok = false; break; }
          tc_fence_after();
          const uint32_t abase = smem_u32(a_tile(stage));
          const uint32_t hbase = smem_u32(xh_tile(stage)), lbase = smem_u32(xl_tile(stage));
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk) {
            // K-major: the k-step is 32 bytes inside the swizzled rows; MN-major: 16 rows (2 KB), the
            // next 8-row group 1 KB on (SBO) and the next 64 positions 8 KB on (LBO)
            const uint64_t bdesc =
                DIR == 0 ? smem_desc(abase + kk * 32, 16, 1024) : smem_desc(abase + kk * 2048, kBK * 128, 1024);
            mma_f16(tacc, smem_desc(hbase + kk * 32, 16, 1024), bdesc, idesc, (first && kk == 0) ? 0u : 1u);
            mma_f16(tacc, smem_desc(lbase + kk * 32, 16, 1024), bdesc, idesc, 1u);
          }
          first = false;
          mma_commit(empty0 + 8 * stage);
        }
        if (!ok) break;
        mma_commit(tfull0 + 8 * b);
        ++seg;
      }
    }
  } else if (warp < 6) {
    // ---------------------------------------------------------------- epilogue (warps 2..5)
    tc_epilogue<kBN, kM>(args.Ct, args.ldc, args.partials, args.len, args.l, KB, sk, s, e, tmem_base, tfull0,
                         tempty0, args.status);
  } else if (kConv) {
    // ---------------------------------------------------------------- converter (warps 6..9)
    constexpr int CT = 32 * Cfg::kConvWarps;   // converter threads
    const int ct = threadIdx.x - 192;
    if (ct == 0) *conv_abort = 0;
    asm volatile("bar.sync 1, %0;" ::"n"(CT) : "memory");
    double fro = 0.0;
    // FP8 tile scales of iteration i2 for this thread -- A X: the two 128-row tile rows of the 256
    // positions; A^T Y: the tile column of the thread's eight positions (c8 = ct mod 32 in every
    // stage) -- loaded one iteration ahead, so their latency hides behind a stage's conversion
    auto scales_of = [&](int64_t i2, float& a, float& b) {
      const int64_t t2 = i2 / KB, kb2 = i2 - t2 * KB;
      const int64_t kcol = (kb2 * kBK) >> 7, p02 = t2 * kBN;
      if (DIR == 0) {
        const int64_t tr0 = p02 >> 7, tr1 = tr0 + 1 < args.srows ? tr0 + 1 : tr0;
        a = args.scales[tr0 * args.sld + kcol];
        b = args.scales[tr1 * args.sld + kcol];
      } else {
        int64_t tc = (p02 + 8 * (ct & 31)) >> 7;
        if (tc >= args.scols) tc = args.scols - 1;
        a = b = args.scales[kcol * args.sld + tc];
      }
    };
    float sca = 1.f, scb = 1.f;
    if (FP8 && s < e) scales_of(s, sca, scb);
    int64_t n = 0;
    for (int64_t it = s; it < e; ++it, ++n) {
      const int stage = (int)(n % S);
      const uint32_t ph = (uint32_t)((n / S) & 1);
      float nsa = 1.f, nsb = 1.f;
      if (FP8 && it + 1 < e) scales_of(it + 1, nsa, nsb);
      // the converter warps give up together (one abort flag per stage)
      if (!mbar_wait(full0 + 8 * stage, ph, args.status)) *conv_abort = 1;
      asm volatile("bar.sync 1, %0;" ::"n"(CT) : "memory");
      if (*conv_abort) break;
      uint8_t* at = a_tile(stage);
      float part = 0.f;
      if (!FP8) {
        // BF16 tiles are read as TMA lands them: only ||A||^2
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
      } else if (DIR == 0) {
        // staging [256 rows][64 B] -> BF16 [256 rows][64] (128-byte swizzle), times the tile scale
        // the 256 rows span two 128-row tile rows; the 64 columns lie in one tile column
        const uint8_t* f8 = f8_tile(stage);
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
        // staging [64 k][256 B] -> BF16 MN-major: row k of the 64-position block c at c * 8 KB + 128 k
        // (128-byte swizzle), times the tile scale; the 64 k rows lie in one 128-row tile row and 8
        // consecutive positions in one tile column
        const uint8_t* f8 = f8_tile(stage);
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
      fro += (double)part;
      sca = nsa;
      scb = nsb;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(conv0 + 8 * stage);
    }
    if (FRO) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
      if (lane == 0) fro_red[warp - 6] = fro;
    }
  }

  tc_fence_before();
  __syncthreads();
  if (FRO && threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < Cfg::kConvWarps; ++w) t += fro_red[w];
    args.fro_parts[blockIdx.x] = t;
  }
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem_base) : "memory");
  }
}

// X (FP32 ST) -> X_hi = bf16(X), X_lo = bf16(X - X_hi)
__global__ void split_bf16_kernel(const float* __restrict__ X, int64_t ldx, __nv_bfloat16* __restrict__ Xh,
                                  __nv_bfloat16* __restrict__ Xl, int64_t ldo, int l, int64_t len) {
  const int j = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
    const float x = X[j * ldx + i];
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    Xh[j * ldo + i] = h;
    Xl[j * ldo + i] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}

template <int DIR, bool FP8, bool FRO>
cudaError_t launch_lp_variant(const CUtensorMap& mA, const CUtensorMap& mH, const CUtensorMap& mL, const LpArgs& la,
                              int64_t G, cudaStream_t st) {
  auto kern = pass_tc_lp_kernel<DIR, FP8, FRO>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, LpCfg<FP8>::kSmem);
  if (err != cudaSuccess) return err;
  constexpr bool conv = FP8 || FRO;
  kern<<<(unsigned)G, conv ? LpCfg<FP8>::kThreads : 192, LpCfg<FP8>::kSmem, st>>>(mA, mH, mL, la);
  CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

template <int DIR, bool FP8>
cudaError_t launch_lp_dir(const CUtensorMap& mA, const CUtensorMap& mH, const CUtensorMap& mL, const LpArgs& la,
                          bool fro, int64_t G, cudaStream_t st) {
  return fro ? launch_lp_variant<DIR, FP8, true>(mA, mH, mL, la, G, st)
             : launch_lp_variant<DIR, FP8, false>(mA, mH, mL, la, G, st);
}

}  // namespace

size_t tc_lp_partial_bytes(int sms) { return (size_t)2 * sms * kM * kBN * sizeof(float); }

int tc_lp_grid(int64_t len, int64_t K, int sms) {
  const int64_t total = cdiv(len, kBN) * cdiv(K, kBK);
  return (int)(sms < total ? sms : total);
}

bool tc_lp_supported(int dir, int a_dtype, int l) {
  return (dir == 0 || dir == 1) && (a_dtype == 2 || a_dtype == 3) && l >= 1 && l <= kM;
}

cudaError_t launch_pass_tc_lp(const PassArgs& a, int dir, int a_dtype, int sms, DevStatus* status,
                              double* fro_parts, void* Xh_, void* Xl_, int64_t ldxs, cudaStream_t st) {
  __nv_bfloat16* Xh = static_cast<__nv_bfloat16*>(Xh_);
  __nv_bfloat16* Xl = static_cast<__nv_bfloat16*>(Xl_);
  if (!tc_lp_supported(dir, a_dtype, a.l)) return cudaErrorInvalidValue;
  const bool fp8 = a_dtype == 3;
  // split the FP32 sketch operand into BF16 hi / lo parts
  {
    dim3 grid((unsigned)(cdiv(a.K, 256) < 64 ? cdiv(a.K, 256) : 64), (unsigned)a.l);
    if (grid.x > 0) {
      split_bf16_kernel<<<grid, 256, 0, st>>>(static_cast<const float*>(a.Xt), a.ldx, Xh, Xl, ldxs, a.l, a.K);
      CORUTV_COUNT_LAUNCH();
    }
  }
  CUtensorMap mA, mH, mL;
  bool ok;
  if (fp8) {
    // raw bytes, no swizzle: DIR 0 boxes of 64 columns x 256 rows, DIR 1 of 256 columns x 64 rows
    ok = dir == 0 ? make_map_2d(&mA, a.A, a.m, a.n, a.lda, 1, CU_TENSOR_MAP_DATA_TYPE_UINT8, kBK, kBN, false)
                  : make_map_2d(&mA, a.A, a.m, a.n, a.lda, 1, CU_TENSOR_MAP_DATA_TYPE_UINT8, kBN, kBK, false);
  } else {
    ok = dir == 0 ? make_map_2d(&mA, a.A, a.m, a.n, a.lda, 2, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, kBK, kBN, true)
                  : make_map_2d(&mA, a.A, a.m, a.n, a.lda, 2, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 64, kBK, true);
  }
  ok = ok && make_map_2d(&mH, Xh, a.l, a.K, ldxs, 2, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, kBK, kM, true);
  ok = ok && make_map_2d(&mL, Xl, a.l, a.K, ldxs, 2, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, kBK, kM, true);
  if (!ok) return cudaErrorInvalidValue;
  const int64_t G = tc_lp_grid(a.len_out, a.K, sms);
  if (G <= 0) return cudaSuccess;
  LpArgs la{static_cast<float*>(a.Ct), a.ldc, static_cast<float*>(a.partials), a.len_out, a.K, a.l, status,
            fro_parts, a.scales, a.scale_ld, cdiv(a.m, 128), cdiv(a.n, 128)};
  const bool fro = fro_parts != nullptr;
  cudaError_t err;
  if (fp8) err = dir == 0 ? launch_lp_dir<0, true>(mA, mH, mL, la, fro, G, st) : launch_lp_dir<1, true>(mA, mH, mL, la, fro, G, st);
  else err = dir == 0 ? launch_lp_dir<0, false>(mA, mH, mL, la, fro, G, st) : launch_lp_dir<1, false>(mA, mH, mL, la, fro, G, st);
  if (err != cudaSuccess) return err;
  return launch_streamk_reduce_f32(static_cast<float*>(a.Ct), a.ldc, static_cast<const float*>(a.partials), a.l,
                                   kM, kBN, a.len_out, cdiv(a.K, kBK), G, st);
}

}  // namespace corutv
