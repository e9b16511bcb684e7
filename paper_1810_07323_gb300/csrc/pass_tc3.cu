// FP32-faithful tensor-core streaming passes over A for sm_103a: the skinny
// products of Sec. III (C1 = A Psi, C2 = A^T C1) and Alg. 3 steps 3-4 with
// split operands.  Each FP32 value v is split as v = h + c with h = TF32(v) and
// c = BF16(v - h) (both to nearest: |v - h - c| <= 2^-21 |v|), and
//     a x ~ a_h x_h  +  [c_a, bf16(a_h)] . [bf16(x_h), c_x]
// -- one kind::tf32 MMA (TF32 x TF32 products are exact in FP32) plus ONE
// kind::f16 MMA of twice the K that carries both cross terms, c_a x_h and a_h c_x
// (each within 2^-9 of its exact value, itself ~2^-12 of a x) -- so every product
// carries at most ~2^-19 relative error instead of TF32's 2^-11, for two MMAs per
// k-step.  (Three TF32 MMAs -- h h + l h + h l -- measured 1.3x slower: the
// tensor core re-reads the sketch tile from shared memory for every MMA, and that
// traffic, with the TMA fills, is what binds.)
//
// Orientation: A is the MMA M operand and lives in TENSOR MEMORY.  A tile is 256
// output positions: two sub-tiles of 128 (the MMA M = TMEM lanes) that share every
// staged k-block of the sketch operand, which halves its shared-memory fills and L2
// reads against 128-position tiles.  Per 256 x 32 block of A, two groups of four
// converter warps (one group per sub-tile) read it from shared memory (one
// position per thread: a row of A for dir AX, a column for dir ATY, so the A^T
// direction needs no shared-memory transpose -- the TMEM lane of a thread is its
// position), split it and store a_h (TF32, 32 columns) and the packed BF16 pairs
// [c_a, bf16(a_h)] of each k-step (32 columns) with tcgen05.st.  The sketch
// operand arrives pre-split (l rows of K, ST layout): Xh = TF32(x) and Xc, whose
// row holds, per group of 8 consecutive k, bf16(x_h) of the 8 then c_x of the 8.
// Both are N x K operands in shared memory (N = l rounded up to 16, TMA with
// 128-byte swizzle).  The MMAs accumulate into a 128 x N FP32 TMEM accumulator
// whose lane is the output position, so the epilogue writes Ct (l x len) row by
// row with coalesced stores.
// Shared memory: three stages of A 32 KB + Xh 16 KB + Xc 16 KB.  TMEM: the two
// sub-tiles' accumulators (columns 0..255; one set, so the products of the next
// tile segment wait for the epilogue of the last) and two slots of converted A,
// 64 columns per sub-tile (256..511), released by the MMA's commit.
//
// Work split, partial tiles, bounded waits and the timeout protocol are those of
// the TF32 pass (pass_tc.cu): Stream-K over one CTA per SM, ordered reduction of
// split tiles, every mbarrier wait bounded by %globaltimer.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace corutv {

namespace {

constexpr int kBM = 128;                    // positions per sub-tile (MMA M = TMEM lanes)
constexpr int kSub = 2;                     // sub-tiles per tile
constexpr int kBT = kSub * kBM;             // output positions per tile
constexpr int kBK = 32;                     // FP32 elements along K per stage
constexpr int kNP = 128;                    // sketch rows held per stage (MMA N <= 128)
constexpr int kAStages = 4;                 // shared-memory stages of A (released by the converters)
constexpr int kXStages = 3;                 // shared-memory stages of the sketch operand (released by the MMA)
constexpr int kSlots = 2;                   // TMEM slots of converted A
constexpr int kATileBytes = kBT * kBK * 4;  // 32 KB
constexpr int kXTileBytes = kNP * kBK * 4;  // 16 KB (Xh: 32 FP32, or Xc: 64 BF16 per row)
constexpr int kConvWarps = 4 * kSub;
// warp 0 TMA of A, 1 MMA, 2..5 epilogue, 6..13 converters, 14 TMA of the sketch operand
constexpr int kXWarp = 6 + kConvWarps;
constexpr int kThreads = 32 * (kXWarp + 1);
constexpr int kSmemBytes = kAStages * kATileBytes + kXStages * 2 * kXTileBytes + 1024 /*align*/ + 512 /*barriers*/;
static_assert(kSmemBytes <= 232448, "shared memory");
constexpr uint32_t kAccCols = 128;          // accumulator of a sub-tile: 128 lanes x N <= 128 columns
constexpr uint32_t kACol0 = kSub * kAccCols;   // first TMEM column of the A slots
constexpr uint32_t kASubCols = 2 * kBK;     // a_h (32 TF32 columns) + BF16 pairs (32 columns)
constexpr uint32_t kASlotCols = kSub * kASubCols;
static_assert(kACol0 + kSlots * kASlotCols <= 512, "TMEM columns");

struct Tc3Args {
  float* Ct;
  int64_t ldc;
  float* partials;
  int64_t len, K;
  int l, np;
  DevStatus* status;
  double* fro_parts;
};

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}

// D (TMEM) (+)= A (TMEM, M x K) * B (shared memory descriptor, N x K), kind::tf32
__device__ __forceinline__ void mma_tf32_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n"
      "}\n" ::"r"(tmem_d),
      "r"(tmem_a), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// the same for kind::f16 (BF16 operands, FP32 accumulation), K = 16
__device__ __forceinline__ void mma_bf16_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t idesc) {
  asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, 1;" ::"r"(tmem_d), "r"(tmem_a), "l"(bdesc),
               "r"(idesc)
               : "memory");
}

// kind::f16 instruction descriptor: D FP32 (bit 4), A / B BF16 (1 at bits 7, 10), both K-major,
// N >> 3 (bits 17-22), M >> 4 (bits 24-28)
__host__ __device__ constexpr uint32_t idesc_bf16_kk(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// two floats -> packed BF16 pair (round to nearest even), `lo` in the low half
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

// Epilogue (four consecutive warps; warp & 3 selects the TMEM lane quarter = 32
// positions of each sub-tile).  A thread owns position pl of both sub-tiles; the
// accumulator row of a position holds its l outputs, read 32 columns at a time.  A
// segment covering all k-blocks of its tile goes to Ct, any other to the CTA's
// partial slot ([j][position], 256 positions).
__device__ __noinline__ void tc3_epilogue(const Tc3Args& a, int KB, int s, int e, uint32_t tmem_base,
                                             uint32_t tfull, uint32_t tempty) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = warp & 3;
  const int pl = 32 * g + lane;
  const int chunks = (a.l + 31) / 32;
  const int first_tile = s / KB;               // partial slots as StreamK::slot: 2 c (first tile), 2 c + 1
  int seg = 0;
  int it = s;
  while (it < e) {
    const int t = it / KB;
    const int kb0 = it - t * KB;
    const int kb1 = (e - t * KB < KB) ? (e - t * KB) : KB;
    if (!mbar_wait(tfull, (uint32_t)(seg & 1), a.status)) break;
    tc_fence_after();
    const bool complete = (kb0 == 0 && kb1 == KB);
    const int slot = 2 * (int)blockIdx.x + (t == first_tile ? 0 : 1);
#pragma unroll 1
    for (int u = 0; u < kSub; ++u) {
      const int64_t p = (int64_t)t * kBT + u * kBM + pl;
      float* dst;
      int64_t ld;
      bool live;
      if (complete) {
        dst = a.Ct + p;
        ld = a.ldc;
        live = p < a.len;
      } else {
        dst = a.partials + (int64_t)slot * kNP * kBT + u * kBM + pl;
        ld = kBT;
        live = true;
      }
#pragma unroll 1
      for (int c = 0; c < chunks; ++c) {
        float v[32];
        tmem_ld32(tmem_base + (uint32_t)(u * kAccCols + 32 * c) + ((uint32_t)(32 * g) << 16), v);
        if (live) {
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int j = 32 * c + i;
            if (j < a.l) dst[(int64_t)j * ld] = v[i];
          }
        }
      }
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(tempty);
    ++seg;
    it = t * KB + kb1;
  }
}

// FRO: the converter warps also accumulate sum(a^2) of the tiles (FP32 per stage,
// folded into FP64), one partial per CTA.
template <int DIR, bool FRO>
__global__ void __launch_bounds__(kThreads, 1)
    pass_tc3_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapXh,
                    const __grid_constant__ CUtensorMap mapXc, Tc3Args args) {
  extern __shared__ uint8_t smem_dyn[];
  uint8_t* smem = smem_dyn + ((1024u - (smem_u32(smem_dyn) & 1023u)) & 1023u);
  uint8_t* a_tiles = smem;                                   // kAStages x 32 KB
  uint8_t* xh_tiles = smem + kAStages * kATileBytes;         // kXStages x 16 KB
  uint8_t* xc_tiles = xh_tiles + kXStages * kXTileBytes;     // kXStages x 16 KB
  uint64_t* bars = reinterpret_cast<uint64_t*>(xc_tiles + kXStages * kXTileBytes);
  // bars: afull[AS], aempty[AS], xfull[XS], xempty[XS], conv[kSlots], tfree[kSlots], tfull, tempty;
  // then the TMEM address and the ||A||^2 partials
  constexpr int kBars = 2 * kAStages + 2 * kXStages + 2 * kSlots + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + kBars);
  double* fro_red = reinterpret_cast<double*>(bars + kBars + 1);   // one double per converter warp
  const uint32_t afull0 = smem_u32(bars), aempty0 = afull0 + 8 * kAStages;
  const uint32_t xfull0 = aempty0 + 8 * kAStages, xempty0 = xfull0 + 8 * kXStages;
  const uint32_t conv0 = xempty0 + 8 * kXStages, tfree0 = conv0 + 8 * kSlots;
  const uint32_t tfull = tfree0 + 8 * kSlots, tempty = tfull + 8;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // iteration indices fit 32 bits (the host checks tiles x k-blocks < 2^31): 32-bit divisions
  const int KB = (int)cdiv(args.K, kBK);
  const StreamK sk(cdiv(args.len, kBT), KB, gridDim.x);
  const int s = (int)sk.start(blockIdx.x), e = (int)sk.start(blockIdx.x + 1);

  if (threadIdx.x == 0) {
    for (int i = 0; i < kAStages; ++i) {
      mbar_init(afull0 + 8 * i, 1);
      mbar_init(aempty0 + 8 * i, kConvWarps);
    }
    for (int i = 0; i < kXStages; ++i) {
      mbar_init(xfull0 + 8 * i, 1);
      mbar_init(xempty0 + 8 * i, 1);
    }
    for (int q = 0; q < kSlots; ++q) {
      mbar_init(conv0 + 8 * q, kConvWarps);
      mbar_init(tfree0 + 8 * q, 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, 4);
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

  if (warp == 0 || warp == kXWarp) {
    // ---------------------------------------------------------------- TMA producers
    // warp 0 fills the A stages as the converters free them (they run ahead of the MMA by
    // the TMEM slots, so A is prefetched several stages ahead); warp kXWarp fills the
    // sketch stages as the MMA frees them (L2-resident data, a short lead suffices)
    if (lane == 0) {
      const bool isA = warp == 0;
      const int S = isA ? kAStages : kXStages;
      const uint32_t full0 = isA ? afull0 : xfull0, empty0 = isA ? aempty0 : xempty0;
      const uint64_t pol = isA ? policy_evict_first() : policy_evict_last();
      int n = 0;
      bool ok = true;
      for (int it = s; it < e; ++it, ++n) {
        const int stage = n % S;
        const uint32_t ph = (uint32_t)((n / S) & 1);
        if (!mbar_wait(empty0 + 8 * stage, ph ^ 1, args.status)) { ok = false; break; }
        const int t = it / KB, kb = it - t * KB;
        const int k0 = kb * kBK;
        const int p0 = t * kBT;
        const uint32_t fb = full0 + 8 * stage;
        if (isA) {
          mbar_arrive_expect_tx(fb, kATileBytes);
          const uint32_t adst = smem_u32(a_tiles + stage * kATileBytes);
          if (DIR == 0)
            tma_load_2d(adst, &mapA, fb, k0, p0, pol);     // 256 rows of A x 32 columns (swizzled)
          else
            tma_load_2d(adst, &mapA, fb, p0, k0, pol);     // 32 rows of A x 256 columns (plain)
        } else {
          mbar_arrive_expect_tx(fb, 2 * kXTileBytes);
          tma_load_2d(smem_u32(xh_tiles + stage * kXTileBytes), &mapXh, fb, k0, 0, pol);
          tma_load_2d(smem_u32(xc_tiles + stage * kXTileBytes), &mapXc, fb, 2 * k0, 0, pol);
        }
      }
      // drain: every issued fill must be consumed before the CTA exits; on an aborted run
      // wait (bounded) for the copies themselves
      const int first = n > S ? n - S : 0;
      for (int f = first; f < n; ++f) {
        const int stage = f % S;
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
      const uint32_t idesc = idesc_tf32(kBM, args.np, 0, 0);   // A from TMEM, B K-major
      const uint32_t idesc_x = idesc_bf16_kk(kBM, args.np);
      int n = 0;
      int seg = 0;
      bool ok = true;
      int it = s;
      while (it < e && ok) {
        const int t = it / KB;
        const int kb1 = (e - t * KB < KB) ? (e - t * KB) : KB;
        // the accumulators are free once the epilogue has drained the previous segment
        if (!mbar_wait(tempty, (uint32_t)((seg & 1) ^ 1), args.status)) { ok = false; break; }
        tc_fence_after();
        bool first = true;
        for (; it < t * KB + kb1; ++it, ++n) {
          const int xs = n % kXStages, q = n % kSlots;
          if (!mbar_wait(conv0 + 8 * q, (uint32_t)((n / kSlots) & 1), args.status) ||
              !mbar_wait(xfull0 + 8 * xs, (uint32_t)((n / kXStages) & 1), args.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t xh = smem_u32(xh_tiles + xs * kXTileBytes);
          const uint32_t xc = smem_u32(xc_tiles + xs * kXTileBytes);
          const uint32_t ta = tmem_base + kACol0 + (uint32_t)q * kASlotCols;
#pragma unroll
          for (int kk = 0; kk < kBK / 8; ++kk) {
            // k-step kk: 8 values of K; TF32 rows are 32 bytes per k-step, so are the BF16 pairs
            const uint64_t bh = smem_desc(xh + kk * 32, 16, 1024), bc = smem_desc(xc + kk * 32, 16, 1024);
#pragma unroll
            for (int u = 0; u < kSub; ++u) {
              const uint32_t tacc = tmem_base + (uint32_t)u * kAccCols;
              const uint32_t tau = ta + (uint32_t)u * kASubCols;
              mma_tf32_ts(tacc, tau + (uint32_t)(8 * kk), bh, idesc, (first && kk == 0) ? 0u : 1u);
              mma_bf16_ts(tacc, tau + (uint32_t)(kBK + 8 * kk), bc, idesc_x);
            }
          }
          first = false;
          mma_commit(xempty0 + 8 * xs);
          mma_commit(tfree0 + 8 * q);
        }
        if (!ok) break;
        mma_commit(tfull);
        ++seg;
      }
    }
  } else if (warp < 6) {
    // ---------------------------------------------------------------- epilogue (warps 2..5)
    tc3_epilogue(args, KB, s, e, tmem_base, tfull, tempty);
  } else {
    // ---------------------------------------------------------------- converters (warps 6..13)
    // group u converts sub-tile u (positions 128 u .. 128 u + 127) of every staged block
    const int u = (warp - 6) >> 2;
    const int g = warp & 3;
    const int pl = 32 * g + lane;                 // this thread's position in the sub-tile
    double fro = 0.0;
    int n = 0;
    for (int it = s; it < e; ++it, ++n) {
      const int as = n % kAStages, q = n % kSlots;
      // the TMEM slot is free once the products of fill n - kSlots have completed
      if (!mbar_wait(tfree0 + 8 * q, (uint32_t)(((n / kSlots) & 1) ^ 1), args.status)) break;
      if (!mbar_wait(afull0 + 8 * as, (uint32_t)((n / kAStages) & 1), args.status)) break;
      tc_fence_after();
      const uint8_t* tile = a_tiles + as * kATileBytes;
      const uint32_t ta = tmem_base + kACol0 + (uint32_t)q * kASlotCols + (uint32_t)u * kASubCols +
                          ((uint32_t)(32 * g) << 16);
      // the 32 values of this position: a row of the block (dir AX) or a column (dir ATY)
      float v[32];
      if (DIR == 0) {
        // row 128 u + pl of the swizzled 256 x 32 block: chunk c (4 floats) sits at c ^ (pl & 7)
        const uint8_t* row = tile + (u * kBM + pl) * 128;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float4 w = *reinterpret_cast<const float4*>(row + ((c ^ (pl & 7)) << 4));
          v[4 * c] = w.x; v[4 * c + 1] = w.y; v[4 * c + 2] = w.z; v[4 * c + 3] = w.w;
        }
      } else {
        // column 128 u + pl of the plain 32 x 256 block
        const float* col = reinterpret_cast<const float*>(tile) + u * kBM + pl;
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = col[k * kBT];
      }
      // the A stage is released as soon as it has been read (the next copy may land in it)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(aempty0 + 8 * as);
      float part = 0.f;
      // two halves of 16 values of K (k-steps 2 hf, 2 hf + 1): a_h = TF32(a) into columns
      // 16 hf .. 16 hf + 15 of the sub-tile's slot; per k-step kk the BF16 pairs
      // [c_a(k) ..., bf16(a_h)(k) ...] of its 8 values into columns 32 + 8 kk .. 32 + 8 kk + 7
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        uint32_t hi[16], cr[16];
#pragma unroll
        for (int k2 = 0; k2 < 2; ++k2) {
          float h[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const float a = v[16 * hf + 8 * k2 + i];
            if (FRO) part = fmaf(a, a, part);
            h[i] = to_tf32(a);
            hi[8 * k2 + i] = __float_as_uint(h[i]);
          }
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            const int k = 16 * hf + 8 * k2 + 2 * w;
            cr[8 * k2 + w] = pack_bf16(v[k] - h[2 * w], v[k + 1] - h[2 * w + 1]);
            cr[8 * k2 + 4 + w] = pack_bf16(h[2 * w], h[2 * w + 1]);
          }
        }
        tmem_st16(ta + (uint32_t)(16 * hf), hi);
        tmem_st16(ta + (uint32_t)(kBK + 16 * hf), cr);
      }
      if (FRO) fro += (double)part;
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(conv0 + 8 * q);
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
    double f = 0.0;
    for (int w = 0; w < kConvWarps; ++w) f += fro_red[w];
    args.fro_parts[blockIdx.x] = f;
  }
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem_base) : "memory");
  }
}

template <int DIR, bool FRO>
cudaError_t launch_variant(const CUtensorMap& mapA, const CUtensorMap& mapXh, const CUtensorMap& mapXc,
                           const Tc3Args& ta, int64_t G, cudaStream_t st) {
  auto kern = pass_tc3_kernel<DIR, FRO>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (err != cudaSuccess) return err;
  kern<<<(unsigned)G, kThreads, kSmemBytes, st>>>(mapA, mapXh, mapXc, ta);
  CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

// Xh = TF32(X) (nearest) and Xc: for every group of 8 consecutive positions k of a row,
// bf16(Xh) of the 8 then bf16(X - Xh) of the 8 (the BF16 operand of the cross-term MMA).
// A thread takes one group (two 16-byte loads, two 16-byte stores to Xh, two to Xc);
// positions len .. round_up(len, 8) - 1 of Xc are written as zeros.  Rows of X, Xh and
// Xc start 16-byte aligned (ST layouts).
__global__ void split_tf32_kernel(const float* __restrict__ X, int64_t ldx, float* __restrict__ Xh,
                                  __nv_bfloat16* __restrict__ Xc, int64_t ldr, int l, int64_t len) {
  const int j = blockIdx.y;
  if (j >= l) return;
  const int64_t groups = (len + 7) / 8;
  const float* xr = X + j * ldx;
  float* hr = Xh + j * ldr;
  uint4* cr = reinterpret_cast<uint4*>(Xc + j * 2 * ldr);
  for (int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gi < groups;
       gi += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = 8 * gi;
    float x[8];
    if (i0 + 8 <= len) {
      const float4 a = *reinterpret_cast<const float4*>(xr + i0);
      const float4 b = *reinterpret_cast<const float4*>(xr + i0 + 4);
      x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) x[q] = i0 + q < len ? xr[i0 + q] : 0.f;
    }
    float h[8];
    uint32_t hb[4], cb[4];
#pragma unroll
    for (int q = 0; q < 8; ++q) h[q] = to_tf32(x[q]);
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      hb[w] = pack_bf16(h[2 * w], h[2 * w + 1]);
      cb[w] = pack_bf16(x[2 * w] - h[2 * w], x[2 * w + 1] - h[2 * w + 1]);
    }
    if (i0 + 8 <= len) {
      *reinterpret_cast<float4*>(hr + i0) = make_float4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<float4*>(hr + i0 + 4) = make_float4(h[4], h[5], h[6], h[7]);
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (i0 + q < len) hr[i0 + q] = h[q];
    }
    cr[2 * gi] = make_uint4(hb[0], hb[1], hb[2], hb[3]);
    cr[2 * gi + 1] = make_uint4(cb[0], cb[1], cb[2], cb[3]);
  }
}

}  // namespace

size_t tc3_pass_partial_bytes(int sms) { return (size_t)2 * sms * kNP * kBT * sizeof(float); }

int tc3_pass_grid(int64_t len, int64_t K, int sms) {
  const int64_t total = cdiv(len, kBT) * cdiv(K, kBK);
  return (int)(sms < total ? sms : total);
}

bool tc3_pass_supported(int dir, int a_dtype, int l) {
  return (dir == 0 || dir == 1) && a_dtype == 1 && l >= 1 && l <= kNP;
}

cudaError_t launch_split_tf32(const float* X, int64_t ldx, float* Xh, void* Xc, int64_t ldr, int l, int64_t len,
                              cudaStream_t st) {
  const int64_t blocks = cdiv(cdiv(len, 8), 128);
  dim3 grid((unsigned)(blocks < 64 ? blocks : 64), (unsigned)l);
  if (grid.x == 0 || l <= 0) return cudaSuccess;
  split_tf32_kernel<<<grid, 128, 0, st>>>(X, ldx, Xh, static_cast<__nv_bfloat16*>(Xc), ldr, l, len);
  CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t launch_pass_tc3(const PassArgs& a, int dir, int sms, DevStatus* status, double* fro_parts,
                            const float* Xh, const void* Xc, int64_t ldxs, cudaStream_t st) {
  if (!tc3_pass_supported(dir, 1, a.l)) return cudaErrorInvalidValue;
  CUtensorMap mapA, mapXh, mapXc;
  if (dir == 0) {
    // rows of A: 256 rows x 32 columns, 128-byte swizzle (a converter thread reads one row)
    if (!make_map_2d(&mapA, a.A, a.m, a.n, a.lda, 4, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, kBK, kBT, true))
      return cudaErrorInvalidValue;
  } else {
    // columns of A: 32 rows x 256 columns, unswizzled (a converter thread reads one column)
    if (!make_map_2d(&mapA, a.A, a.m, a.n, a.lda, 4, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, kBT, kBK, false))
      return cudaErrorInvalidValue;
  }
  // Xh: l rows x K FP32, Xc: l rows x 2 round_up(K, 8) BF16 (leading dimension 2 ldxs); the
  // 128-row boxes read zeros below row l
  if (!make_map_2d(&mapXh, Xh, a.l, a.K, ldxs, 4, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, kBK, kNP, true) ||
      !make_map_2d(&mapXc, Xc, a.l, 2 * round_up(a.K, 8), 2 * ldxs, 2, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2 * kBK,
                   kNP, true))
    return cudaErrorInvalidValue;
  const int64_t G = tc3_pass_grid(a.len_out, a.K, sms);
  if (G <= 0) return cudaSuccess;
  if (cdiv(a.len_out, kBT) * cdiv(a.K, kBK) >= (int64_t)1 << 31) return cudaErrorInvalidValue;   // 32-bit indices
  Tc3Args ta{static_cast<float*>(a.Ct), a.ldc, static_cast<float*>(a.partials), a.len_out, a.K, a.l,
             (int)round_up(a.l, 16), status, fro_parts};
  cudaError_t err;
  if (a.kmark) a.kmark->start(st);
  if (dir == 0)
    err = fro_parts ? launch_variant<0, true>(mapA, mapXh, mapXc, ta, G, st)
                    : launch_variant<0, false>(mapA, mapXh, mapXc, ta, G, st);
  else
    err = fro_parts ? launch_variant<1, true>(mapA, mapXh, mapXc, ta, G, st)
                    : launch_variant<1, false>(mapA, mapXh, mapXc, ta, G, st);
  if (err != cudaSuccess) return err;
  if (a.kmark) a.kmark->stop(st);
  return launch_streamk_reduce_f32(static_cast<float*>(a.Ct), a.ldc, static_cast<const float*>(a.partials), a.l,
                                   kNP, kBT, a.len_out, cdiv(a.K, kBK), G, st);
}

}  // namespace corutv
