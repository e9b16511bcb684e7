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
#include "tc_lp_common.cuh"

namespace corutv {

namespace {

using namespace lpk;

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
    // FP8 tile scales of iteration i2, loaded one iteration ahead so their latency hides behind a
    // stage's conversion
    auto scales_of = [&](int64_t i2, float& a, float& b) {
      const int64_t t2 = i2 / KB, kb2 = i2 - t2 * KB;
      lp_stage_scales(args.scales, args.sld, args.srows, args.scols, DIR, kb2, t2 * kBN, ct, a, b);
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
      const float part = lp_convert_stage<FP8, FRO, CT>(a_tile(stage), f8_tile(stage), DIR, sca, scb, ct);
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

// FP8 A with decoupled rings.  The FP8 tiles, the dequantised BF16 tiles and the sketch tiles
// each get their own ring, so a stage no longer holds its shared memory from the TMA copy
// through the conversion to the MMA: FP8 copies (16 KB) run four ahead of the converter warps,
// the converters fill two BF16 slots ahead of the MMA, and a second producer warp keeps three
// sketch stages ahead of the MMA.  (One 80 KB stage per iteration allows only two in flight,
// and the DRAM latency then bounds the pass.)  Warps: 0 FP8 TMA, 1 MMA, 2..5 epilogue, 6..13
// converters, 14 sketch TMA.
constexpr int k8S = 4;                     // FP8 staging slots
constexpr int k8A = 2;                     // BF16 A slots
constexpr int k8X = 3;                     // sketch (X_hi + X_lo) slots
constexpr int k8ConvWarps = 8;
constexpr int k8XWarp = 6 + k8ConvWarps;
constexpr int k8Threads = 32 * (k8XWarp + 1);
constexpr int k8Smem = k8S * kF8Tile + k8A * kATile + k8X * 2 * kXTile + 1024 + 512;
static_assert(k8Smem <= 232448, "shared memory");

template <int DIR, bool FRO>
__global__ void __launch_bounds__(k8Threads, 1)
    pass_tc_lp8_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapXh,
                       const __grid_constant__ CUtensorMap mapXl, LpArgs args) {
  extern __shared__ uint8_t smem_dyn[];
  uint8_t* smem = smem_dyn + ((1024u - (smem_u32(smem_dyn) & 1023u)) & 1023u);
  uint8_t* a_slots = smem;                                   // k8A x 32 KB (1024-aligned)
  uint8_t* x_slots = a_slots + k8A * kATile;                 // k8X x (X_hi 16 KB | X_lo 16 KB)
  uint8_t* f_slots = x_slots + k8X * 2 * kXTile;             // k8S x 16 KB
  auto a_tile = [&](int q) { return a_slots + q * kATile; };
  auto xh_tile = [&](int q) { return x_slots + q * 2 * kXTile; };
  auto xl_tile = [&](int q) { return x_slots + q * 2 * kXTile + kXTile; };
  auto f8_tile = [&](int q) { return f_slots + q * kF8Tile; };
  uint64_t* bars = reinterpret_cast<uint64_t*>(f_slots + k8S * kF8Tile);
  // ffull/fempty[k8S], afull/aempty[k8A], xfull/xempty[k8X], tfull/tempty[2]
  constexpr int kBars = 2 * k8S + 2 * k8A + 2 * k8X + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + kBars);
  double* fro_red = reinterpret_cast<double*>(bars + kBars + 2);
  volatile int* conv_abort = reinterpret_cast<volatile int*>(fro_red + k8ConvWarps);
  const uint32_t ffull0 = smem_u32(bars), fempty0 = ffull0 + 8 * k8S;
  const uint32_t afull0 = fempty0 + 8 * k8S, aempty0 = afull0 + 8 * k8A;
  const uint32_t xfull0 = aempty0 + 8 * k8A, xempty0 = xfull0 + 8 * k8X;
  const uint32_t tfull0 = xempty0 + 8 * k8X, tempty0 = tfull0 + 16;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t KB = cdiv(args.K, kBK);
  StreamK sk(cdiv(args.len, kBN), KB, gridDim.x);
  const int64_t s = sk.start(blockIdx.x), e = sk.start(blockIdx.x + 1);

  if (threadIdx.x == 0) {
    for (int i = 0; i < k8S; ++i) {
      mbar_init(ffull0 + 8 * i, 1);
      mbar_init(fempty0 + 8 * i, k8ConvWarps);
    }
    for (int i = 0; i < k8A; ++i) {
      mbar_init(afull0 + 8 * i, k8ConvWarps);
      mbar_init(aempty0 + 8 * i, 1);
    }
    for (int i = 0; i < k8X; ++i) {
      mbar_init(xfull0 + 8 * i, 1);
      mbar_init(xempty0 + 8 * i, 1);
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

  if (warp == 0 || warp == k8XWarp) {
    // ---------------------------------------------------------------- TMA producers
    // warp 0: FP8 tiles of A, paced by the converters; the last warp: the sketch tiles, paced by the MMA
    if (lane == 0) {
      const bool isA = warp == 0;
      const int S = isA ? k8S : k8X;
      const uint32_t full0 = isA ? ffull0 : xfull0, empty0 = isA ? fempty0 : xempty0;
      const uint64_t pol = isA ? policy_evict_first() : policy_evict_last();
      int64_t n = 0;
      bool ok = true;
      for (int64_t it = s; it < e; ++it, ++n) {
        const int q = (int)(n % S);
        const uint32_t ph = (uint32_t)((n / S) & 1);
        if (!mbar_wait(empty0 + 8 * q, ph ^ 1, args.status)) { ok = false; break; }
        const int64_t t = it / KB, kb = it - t * KB;
        const int k0 = (int)(kb * kBK), p0 = (int)(t * kBN);
        const uint32_t fb = full0 + 8 * q;
        if (isA) {
          mbar_arrive_expect_tx(fb, kF8Tile);
          if (DIR == 0) tma_load_2d(smem_u32(f8_tile(q)), &mapA, fb, k0, p0, pol);   // 256 rows x 64 B
          else tma_load_2d(smem_u32(f8_tile(q)), &mapA, fb, p0, k0, pol);            // 64 rows x 256 B
        } else {
          mbar_arrive_expect_tx(fb, 2 * kXTile);
          tma_load_2d(smem_u32(xh_tile(q)), &mapXh, fb, k0, 0, pol);
          tma_load_2d(smem_u32(xl_tile(q)), &mapXl, fb, k0, 0, pol);
        }
      }
      // drain: every issued copy is consumed (or, after a timeout, has landed) before the exit
      const int64_t first = n > S ? n - S : 0;
      for (int64_t f = first; f < n; ++f) {
        const int q = (int)(f % S);
        const uint32_t ph = (uint32_t)((f / S) & 1);
        if (ok) {
          if (!mbar_wait(empty0 + 8 * q, ph, args.status)) ok = false;
        }
        if (!ok) mbar_wait(full0 + 8 * q, ph, args.status);
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(kM, kBN, DIR == 1);
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
          const int qa = (int)(n % k8A), qx = (int)(n % k8X);
          if (!mbar_wait(afull0 + 8 * qa, (uint32_t)((n / k8A) & 1), args.status) ||
              !mbar_wait(xfull0 + 8 * qx, (uint32_t)((n / k8X) & 1), args.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t abase = smem_u32(a_tile(qa));
          const uint32_t hbase = smem_u32(xh_tile(qx)), lbase = smem_u32(xl_tile(qx));
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk) {
            const uint64_t bdesc =
                DIR == 0 ? smem_desc(abase + kk * 32, 16, 1024) : smem_desc(abase + kk * 2048, kBK * 128, 1024);
            mma_f16(tacc, smem_desc(hbase + kk * 32, 16, 1024), bdesc, idesc, (first && kk == 0) ? 0u : 1u);
            mma_f16(tacc, smem_desc(lbase + kk * 32, 16, 1024), bdesc, idesc, 1u);
          }
          first = false;
          mma_commit(aempty0 + 8 * qa);
          mma_commit(xempty0 + 8 * qx);
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
  } else {
    // ---------------------------------------------------------------- converters (warps 6..13)
    constexpr int CT = 32 * k8ConvWarps;
    const int ct = threadIdx.x - 192;
    if (ct == 0) *conv_abort = 0;
    asm volatile("bar.sync 1, %0;" ::"n"(CT) : "memory");
    double fro = 0.0;
    // FP8 tile scales of iteration i2, loaded one iteration ahead
    auto scales_of = [&](int64_t i2, float& a, float& b) {
      const int64_t t2 = i2 / KB, kb2 = i2 - t2 * KB;
      lp_stage_scales(args.scales, args.sld, args.srows, args.scols, DIR, kb2, t2 * kBN, ct, a, b);
    };
    float sca = 1.f, scb = 1.f;
    if (s < e) scales_of(s, sca, scb);
    int64_t n = 0;
    for (int64_t it = s; it < e; ++it, ++n) {
      const int qf = (int)(n % k8S), qa = (int)(n % k8A);
      float nsa = 1.f, nsb = 1.f;
      if (it + 1 < e) scales_of(it + 1, nsa, nsb);
      // the FP8 tile has landed and the MMA has released the BF16 slot; the converter warps give
      // up together (one abort flag per stage)
      if (!mbar_wait(ffull0 + 8 * qf, (uint32_t)((n / k8S) & 1), args.status) ||
          !mbar_wait(aempty0 + 8 * qa, (uint32_t)(((n / k8A) & 1) ^ 1), args.status))
        *conv_abort = 1;
      asm volatile("bar.sync 1, %0;" ::"n"(CT) : "memory");
      if (*conv_abort) break;
      tc_fence_after();
      fro += (double)lp_convert_stage<true, FRO, CT>(a_tile(qa), f8_tile(qf), DIR, sca, scb, ct);
      sca = nsa;
      scb = nsb;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(afull0 + 8 * qa);
        mbar_arrive(fempty0 + 8 * qf);
      }
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
    for (int w = 0; w < k8ConvWarps; ++w) t += fro_red[w];
    args.fro_parts[blockIdx.x] = t;
  }
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem_base) : "memory");
  }
}

template <int DIR, bool FRO>
cudaError_t launch_lp8_variant(const CUtensorMap& mA, const CUtensorMap& mH, const CUtensorMap& mL,
                               const LpArgs& la, int64_t G, cudaStream_t st) {
  auto kern = pass_tc_lp8_kernel<DIR, FRO>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, k8Smem);
  if (err != cudaSuccess) return err;
  kern<<<(unsigned)G, k8Threads, k8Smem, st>>>(mA, mH, mL, la);
  CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
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
  if (a.kmark) a.kmark->start(st);
  if (fp8) {
    if (dir == 0) err = fro ? launch_lp8_variant<0, true>(mA, mH, mL, la, G, st) : launch_lp8_variant<0, false>(mA, mH, mL, la, G, st);
    else err = fro ? launch_lp8_variant<1, true>(mA, mH, mL, la, G, st) : launch_lp8_variant<1, false>(mA, mH, mL, la, G, st);
  }
  else {
    err = dir == 0 ? launch_lp_dir<0, false>(mA, mH, mL, la, fro, G, st) : launch_lp_dir<1, false>(mA, mH, mL, la, fro, G, st);
  }
  if (err != cudaSuccess) return err;
  if (a.kmark) a.kmark->stop(st);
  return launch_streamk_reduce_f32(static_cast<float*>(a.Ct), a.ldc, static_cast<const float*>(a.partials), a.l,
                                   kM, kBN, a.len_out, cdiv(a.K, kBK), G, st);
}

}  // namespace corutv
