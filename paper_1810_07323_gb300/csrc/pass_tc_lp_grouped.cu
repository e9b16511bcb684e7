// Grouped kind::f16 tensor-core passes for batched BF16 / FP8 problems: one
// launch computes Ct_p (l_p x len_p) = Xt_p (l_p x K_p) op_p(A_p) for every
// problem p of a table (the products of Sec. III: A X and A^T Y with A stored
// in BF16, or in FP8 e4m3 with one scale per 128 x 128 tile), with the roles
// of the single-problem kernel in pass_tc_lp.cu: a TMA producer warp, one MMA
// issuing thread, four TMEM epilogue warps and, for FP8 tiles or when sum(a^2)
// is folded in, converter warps.  The FP32 sketch operand is split into BF16
// parts X = X_hi + X_lo first (both products accumulate in the same TMEM tile).
//
// Unlike the Stream-K single-problem kernel, work is cut into units that depend
// on the problem alone: one 256-position output tile and one K range of whole
// 64-element k-blocks.  Each unit starts its accumulator from zero and writes
// either the tile itself or, when the tile's K is cut into S ranges, the
// range's partial; a second kernel adds the S partials in range order.  A
// problem's result is therefore the same bits whichever batch it runs in.  Each
// CTA runs the contiguous run of units cta_first[c] .. cta_first[c + 1] - 1 (the
// host balances the runs by k-blocks), its pipeline running on across units.
// Every wait is bounded (DevStatus on timeout).
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
static_assert(kBN == kLpUnitBN && kBK == kLpUnitBK, "unit tile of the grouped kind::f16 pass");

// problem of global unit u (largest p with unit_base <= u)
__device__ inline int find_unit_problem(const GLpProb* __restrict__ gp, int np, int64_t u) {
  int lo = 0, hi = np - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (gp[mid].unit_base <= u) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// unit u of problem P: output tile t, K range s, k-blocks [kb0, kb1)
struct UnitPos {
  int64_t t, kb0, kb1;
  int s;
};
__device__ inline UnitPos unit_pos(const GLpProb& P, int64_t u) {
  const int64_t local = u - P.unit_base;
  UnitPos r;
  r.s = (int)(local / P.tiles);
  r.t = local - (int64_t)r.s * P.tiles;
  r.kb0 = (int64_t)r.s * P.kbc;
  r.kb1 = r.kb0 + P.kbc < P.KB ? r.kb0 + P.kbc : P.KB;
  return r;
}

template <bool FP8, bool FRO>
__global__ void __launch_bounds__(kMaxThreads, 1)
    pass_lp_grouped_kernel(const GLpProb* __restrict__ gp, int np, const int* __restrict__ cta_first,
                           DevStatus* status, int keep_a) {
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
  const int64_t ub = cta_first[blockIdx.x], ue = cta_first[blockIdx.x + 1];

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
  int pi = ub < ue ? find_unit_problem(gp, np, ub) : 0;
  auto advance = [&](int64_t u) -> const GLpProb& {
    while (u >= gp[pi].unit_base + gp[pi].units) ++pi;
    return gp[pi];
  };

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      // keep_a: A is read again by the next launch (fused power steps), so it stays in L2
      const uint64_t pol_a = keep_a ? policy_evict_last() : policy_evict_first(), pol_x = policy_evict_last();
      int64_t n = 0;
      bool ok = true;
      for (int64_t u = ub; u < ue && ok; ++u) {
        const GLpProb& P = advance(u);
        const UnitPos U = unit_pos(P, u);
        const CUtensorMap* mA = static_cast<const CUtensorMap*>(P.mapA);
        const CUtensorMap* mH = static_cast<const CUtensorMap*>(P.mapXh);
        const CUtensorMap* mL = static_cast<const CUtensorMap*>(P.mapXl);
        const int p0 = (int)(U.t * kBN);
        for (int64_t kb = U.kb0; kb < U.kb1; ++kb, ++n) {
          const int stage = (int)(n % S);
          const uint32_t ph = (uint32_t)((n / S) & 1);
          if (!mbar_wait(empty0 + 8 * stage, ph ^ 1, status)) { ok = false; break; }
          const int k0 = (int)(kb * kBK);
          const uint32_t fb = full0 + 8 * stage;
          mbar_arrive_expect_tx(fb, Cfg::kTx);
          if (FP8) {
            if (P.dir == 0) tma_load_2d(smem_u32(f8_tile(stage)), mA, fb, k0, p0, pol_a);   // 256 rows x 64 B
            else tma_load_2d(smem_u32(f8_tile(stage)), mA, fb, p0, k0, pol_a);              // 64 rows x 256 B
          } else if (P.dir == 0) {
            tma_load_2d(smem_u32(a_tile(stage)), mA, fb, k0, p0, pol_a);                    // 256 rows x 64
          } else {
#pragma unroll
            for (int c = 0; c < kBN / 64; ++c)                                              // 4 x (64 rows x 64)
              tma_load_2d(smem_u32(a_tile(stage)) + c * (kBK * 128), mA, fb, p0 + 64 * c, k0, pol_a);
          }
          tma_load_2d(smem_u32(xh_tile(stage)), mH, fb, k0, 0, pol_x);
          tma_load_2d(smem_u32(xl_tile(stage)), mL, fb, k0, 0, pol_x);
        }
      }
      // wait for the last stages' MMAs (or, after a timeout, for the copies in flight)
      const int64_t first = n > S ? n - S : 0;
      for (int64_t f = first; f < n; ++f) {
        const int stage = (int)(f % S);
        const uint32_t ph = (uint32_t)((f / S) & 1);
        if (ok) {
          if (!mbar_wait(empty0 + 8 * stage, ph, status)) ok = false;
        }
        if (!ok) mbar_wait(full0 + 8 * stage, ph, status);
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t ready0 = kConv ? conv0 : full0;
      int64_t n = 0;
      int seg = 0;
      bool ok = true;
      for (int64_t u = ub; u < ue && ok; ++u) {
        const GLpProb& P = advance(u);
        const UnitPos U = unit_pos(P, u);
        const int b = seg & 1;
        const uint32_t tph = (uint32_t)((seg >> 1) & 1);
        if (!mbar_wait(tempty0 + 8 * b, tph ^ 1, status)) break;
        tc_fence_after();
        const uint32_t tacc = tmem_base + (uint32_t)(b * kBN);
        const bool mn = P.dir == 1;
        const uint32_t idesc = mn ? idesc_bf16(kM, kBN, true) : idesc_bf16(kM, kBN, false);
        for (int64_t kb = U.kb0; kb < U.kb1; ++kb, ++n) {
          const int stage = (int)(n % S);
          const uint32_t ph = (uint32_t)((n / S) & 1);
          if (!mbar_wait(ready0 + 8 * stage, ph, status)) { ok = false; break; }
          tc_fence_after();
          const uint32_t abase = smem_u32(a_tile(stage));
          const uint32_t hbase = smem_u32(xh_tile(stage)), lbase = smem_u32(xl_tile(stage));
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk) {
            // K-major: the k-step is 32 bytes inside the swizzled rows; MN-major: 16 rows (2 KB), the
            // next 8-row group 1 KB on (SBO) and the next 64 positions 8 KB on (LBO)
            const uint64_t bdesc = mn ? smem_desc(abase + kk * 2048, kBK * 128, 1024) : smem_desc(abase + kk * 32, 16, 1024);
            mma_f16(tacc, smem_desc(hbase + kk * 32, 16, 1024), bdesc, idesc, (kb == U.kb0 && kk == 0) ? 0u : 1u);
            mma_f16(tacc, smem_desc(lbase + kk * 32, 16, 1024), bdesc, idesc, 1u);
          }
          mma_commit(empty0 + 8 * stage);
        }
        if (!ok) break;
        mma_commit(tfull0 + 8 * b);
        ++seg;
      }
    }
  } else if (warp < 6) {
    // ---------------------------------------------------------------- epilogue (warps 2..5)
    const int g = warp & 3, j = 32 * g + lane;
    int seg = 0;
    for (int64_t u = ub; u < ue; ++u) {
      const GLpProb& P = advance(u);
      const UnitPos U = unit_pos(P, u);
      const int b = seg & 1;
      const uint32_t tph = (uint32_t)((seg >> 1) & 1);
      if (!mbar_wait(tfull0 + 8 * b, tph, status)) break;
      tc_fence_after();
      const int64_t p0 = U.t * kBN, lim = P.len - p0;
      float* dst = P.S == 1 ? P.Ct + (int64_t)j * P.ldc + p0 : P.kparts + ((int64_t)U.s * P.l + j) * P.ldk + p0;
#pragma unroll 1
      for (int c = 0; c < kBN / 32; ++c) {
        float v[32];
        tmem_ld32(tmem_base + (uint32_t)(b * kBN + 32 * c) + ((uint32_t)(32 * g) << 16), v);
        if (j < P.l) {
          const int64_t col0 = 32 * c;
          if (col0 + 32 <= lim) {
            float4* d4 = reinterpret_cast<float4*>(dst + col0);
#pragma unroll
            for (int q = 0; q < 8; ++q) d4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
          } else {
#pragma unroll
            for (int q = 0; q < 32; ++q)
              if (col0 + q < lim) dst[col0 + q] = v[q];
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty0 + 8 * b);
      ++seg;
    }
  } else if (kConv) {
    // ---------------------------------------------------------------- converter (warps 6..)
    constexpr int CT = 32 * Cfg::kConvWarps;
    const int ct = threadIdx.x - 192;
    if (ct == 0) *conv_abort = 0;
    asm volatile("bar.sync 1, %0;" ::"n"(CT) : "memory");
    int64_t n = 0;
    bool stop = false;
    for (int64_t u = ub; u < ue && !stop; ++u) {
      const GLpProb& P = advance(u);
      const UnitPos U = unit_pos(P, u);
      const int64_t p0 = U.t * kBN;
      double fro = 0.0;
      float sca = 1.f, scb = 1.f;
      if (FP8) lp_stage_scales(P.scales, P.sld, P.srows, P.scols, P.dir, U.kb0, p0, ct, sca, scb);
      for (int64_t kb = U.kb0; kb < U.kb1; ++kb, ++n) {
        const int stage = (int)(n % S);
        const uint32_t ph = (uint32_t)((n / S) & 1);
        // the next stage's tile scales, loaded ahead so their latency hides behind this stage
        float nsa = 1.f, nsb = 1.f;
        if (FP8 && kb + 1 < U.kb1) lp_stage_scales(P.scales, P.sld, P.srows, P.scols, P.dir, kb + 1, p0, ct, nsa, nsb);
        // the converter warps give up together (one abort flag per stage)
        if (!mbar_wait(full0 + 8 * stage, ph, status)) *conv_abort = 1;
        asm volatile("bar.sync 1, %0;" ::"n"(CT) : "memory");
        if (*conv_abort) { stop = true; break; }
        fro += (double)lp_convert_stage<FP8, FRO, CT>(a_tile(stage), f8_tile(stage), P.dir, sca, scb, ct);
        sca = nsa;
        scb = nsb;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(conv0 + 8 * stage);
      }
      if (FRO && !stop) {
        // the unit's sum(a^2): per warp, then over the warps in order (one FP64 value per unit)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
        if (lane == 0) fro_red[warp - 6] = fro;
        asm volatile("bar.sync 1, %0;" ::"n"(CT) : "memory");
        if (ct == 0 && P.fro) {
          double t = 0.0;
          for (int w = 0; w < Cfg::kConvWarps; ++w) t += fro_red[w];
          P.fro[u - P.unit_base] = t;
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem_base) : "memory");
  }
}

// X (FP32 ST) -> X_hi = bf16(X), X_lo = bf16(X - X_hi) for every problem of the table; block
// (map[b].x, map[b].y) covers 256 columns of one problem's sketch operand, four consecutive
// columns per thread and step (one 16-byte load, two 8-byte stores; rows are 16-byte aligned)
__global__ void __launch_bounds__(256) lp_grouped_split_kernel(const GLpProb* __restrict__ gp,
                                                               const int2* __restrict__ map) {
  const int2 pm = map[blockIdx.x];
  const GLpProb& P = gp[pm.x];
  __nv_bfloat16* Xh = static_cast<__nv_bfloat16*>(P.Xh);
  __nv_bfloat16* Xl = static_cast<__nv_bfloat16*>(P.Xl);
  const int64_t i0 = (int64_t)pm.y * 256;
  for (int e = threadIdx.x; e < P.l * 64; e += blockDim.x) {
    const int j = e >> 6;
    const int64_t i = i0 + 4 * (e & 63);
    if (i >= P.K) continue;
    float x[4];
    if (i + 3 < P.K) {
      const float4 v = *reinterpret_cast<const float4*>(P.X + j * P.ldx + i);
      x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) x[q] = i + q < P.K ? P.X[j * P.ldx + i + q] : 0.f;
    }
    __nv_bfloat16 h[4], lo[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      h[q] = __float2bfloat16_rn(x[q]);
      lo[q] = __float2bfloat16_rn(x[q] - __bfloat162float(h[q]));
    }
    if (i + 3 < P.K) {
      *reinterpret_cast<uint2*>(Xh + j * P.ldxs + i) = *reinterpret_cast<const uint2*>(h);
      *reinterpret_cast<uint2*>(Xl + j * P.ldxs + i) = *reinterpret_cast<const uint2*>(lo);
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (i + q < P.K) {
          Xh[j * P.ldxs + i + q] = h[q];
          Xl[j * P.ldxs + i + q] = lo[q];
        }
    }
  }
}

// Tiles cut into S K ranges: Ct = sum of the S partials in range order.  Block (map[b], y) covers
// rows 16 y .. 16 y + 15 of tile map[b].y of problem map[b].x.
__global__ void __launch_bounds__(256) lp_grouped_reduce_kernel(const GLpProb* __restrict__ gp,
                                                                const int2* __restrict__ map) {
  const int2 pm = map[blockIdx.x];
  const GLpProb& P = gp[pm.x];
  const int row0 = blockIdx.y * 16;
  if (row0 >= P.l) return;
  const int64_t p0 = (int64_t)pm.y * kBN;
  for (int x = threadIdx.x; x < 16 * kBN; x += blockDim.x) {
    const int j = row0 + x / kBN, ii = x % kBN;
    if (j >= P.l || p0 + ii >= P.len) continue;
    float acc = 0.f;
    for (int s = 0; s < P.S; ++s) acc += P.kparts[((int64_t)s * P.l + j) * P.ldk + p0 + ii];
    P.Ct[(int64_t)j * P.ldc + p0 + ii] = acc;
  }
}

template <bool FP8, bool FRO>
cudaError_t launch_variant(const GLpProb* gp, int np, const int* cta_first, int G, DevStatus* status, int keep_a,
                           cudaStream_t st) {
  auto kern = pass_lp_grouped_kernel<FP8, FRO>;
  // raised once per device (the first, uncaptured run of a batch)
  static bool attr_set[64] = {};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, LpCfg<FP8>::kSmem);
    if (err != cudaSuccess) return err;
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  constexpr bool conv = FP8 || FRO;
  kern<<<(unsigned)G, conv ? LpCfg<FP8>::kThreads : 192, LpCfg<FP8>::kSmem, st>>>(gp, np, cta_first, status,
                                                                                   keep_a);
  CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pass_lp_grouped(const GLpProb* gp, int np, bool fp8, bool fro, const int* cta_first, int G,
                                   const int2* split_map, int nsplit, const int2* red_map, int nred, int lmax,
                                   DevStatus* status, bool keep_a, cudaStream_t st, KernelMark* km) {
  if (np <= 0 || G <= 0) return cudaSuccess;
  if (nsplit > 0) {
    lp_grouped_split_kernel<<<nsplit, 256, 0, st>>>(gp, split_map);
    CORUTV_COUNT_LAUNCH();
  }
  cudaError_t err;
  const int ka = keep_a ? 1 : 0;
  if (km) km->start(st);
  if (fp8) err = fro ? launch_variant<true, true>(gp, np, cta_first, G, status, ka, st)
                     : launch_variant<true, false>(gp, np, cta_first, G, status, ka, st);
  else err = fro ? launch_variant<false, true>(gp, np, cta_first, G, status, ka, st)
                 : launch_variant<false, false>(gp, np, cta_first, G, status, ka, st);
  if (err != cudaSuccess) return err;
  if (km) km->stop(st);
  if (nred > 0) {
    lp_grouped_reduce_kernel<<<dim3((unsigned)nred, (unsigned)cdiv(lmax, 16)), 256, 0, st>>>(gp, red_map);
    CORUTV_COUNT_LAUNCH();
  }
  return cudaGetLastError();
}

}  // namespace corutv
