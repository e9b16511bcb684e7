// Tensor-core streaming passes over A for sm_103a: the skinny products of
// Sec. III (C1 = A Psi, C2 = A^T C1) and Alg. 3 steps 3-4, as
//     Ct (l x len) = Xt (l x K) * op(A)
// with the l sketch columns as the MMA M dimension (M = 128) and A as the
// N x K operand, K-major in shared memory for both directions:
//   dir AX : op(A) = A^T, B operand = A rows (TMA delivers them K-major, K = n)
//   dir ATY: op(A) = A,   B operand = A columns (TMA delivers 32-row x 32-column
//            boxes; the converter warps transpose each tile in shared memory, K = m)
// A is streamed HBM -> shared memory by TMA (128-byte swizzle), consumed by
// tcgen05.mma kind::tf32 issued from one thread, accumulated in TMEM (two
// 128 x 256 FP32 accumulators, so the epilogue of one tile overlaps the
// products of the next), and written out by four epilogue warps.  Converter
// warps round A tiles to TF32 (nearest), transpose A^T tiles and accumulate
// ||A||_F^2 where those are asked for.
// The (tile, k-block) space is split Stream-K style over one CTA per SM;
// tiles shared by several CTAs go through the ordered partial reduction.
//
// Every wait is bounded (kWaitBudgetNs of %globaltimer): on expiry the
// thread records kStatTimeout in the status word and stops its role; the
// producer then waits (bounded) for its copies in flight and the CTA frees
// its TMEM before returning.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace corutv {

namespace {

constexpr int kTcBN = 256;          // output positions per tile (MMA N)
constexpr int kTcM = 128;           // MMA M (sketch columns, padded)
constexpr int kTcBK = 32;           // fp32 elements per stage along K (one 128-byte swizzle row)
constexpr int kStages = 4;
constexpr int kATileBytes = kTcBN * kTcBK * 4;   // 32 KB
constexpr int kXTileBytes = kTcM * kTcBK * 4;    // 16 KB
constexpr int kStageBytes = kATileBytes + kXTileBytes;
constexpr int kThreads = 192;       // warp 0 TMA, warp 1 MMA, warps 2..5 epilogue
constexpr int kThreadsMax = 320;    // + warps 6..9: TF32 rounding / ||A||^2 of each A tile
constexpr int kSmemBytes = kStages * kStageBytes + 1024 /*align*/ + 512 /*barriers, reductions*/;

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false (and the timeout bit set) if the phase did not complete in time.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, DevStatus* st) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  uint32_t spins = 0;
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((++spins & 255u) == 0 && globaltimer_ns() - t0 > kWaitBudgetNs) {
      if (st) {
        atomicOr(&st->flags, kStatTimeout);
        atomicAdd(&st->timeouts, 1);
      }
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y,
                                            uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%3, %4}], [%2], %5;" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y), "l"(policy)
      : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// Shared-memory matrix descriptor (sm_100 family): start, leading / stride byte
// offsets (>> 4), version 1 at bit 46, 128-byte swizzle (layout 2) at bits 61-63.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor, kind::tf32: D fp32 (bit 4), A/B tf32 (2 at bits 7, 10),
// A major (bit 15), B major (bit 16), N >> 3 (bits 17-22), M >> 4 (bits 24-28).
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N, int a_mn_major, int b_mn_major) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)a_mn_major << 15) | ((uint32_t)b_mn_major << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float sel_comp(const float4& v, int j) {
  float r = v.x;
  r = (j == 1) ? v.y : r;
  r = (j == 2) ? v.z : r;
  r = (j == 3) ? v.w : r;
  return r;
}

// FP32 -> TF32, round to nearest (ties away from zero); low 13 bits become zero.
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

struct TcArgs {
  float* Ct;
  int64_t ldc;
  float* partials;
  int64_t len, K;
  int l;
  DevStatus* status;
  double* fro_parts;   // per-CTA sum(a^2) when fused, else null
};

// ------------------------------------------------------------------ kernel
// CONV: warps 6..9 round every A tile in shared memory to TF32 (round to
//       nearest, ties away) before the MMA reads it, so the tensor core's
//       truncation of the low 13 bits is exact and the products carry no
//       systematic shrink.
// FRO:  the same warps accumulate sum(a^2) of the original tile values
//       (FP32 per stage, folded into FP64), one partial per CTA.
template <int DIR, bool CONV, bool FRO>
__global__ void __launch_bounds__(kThreadsMax, 1)
    pass_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapX, TcArgs args) {
  constexpr bool kConvWarps = CONV || FRO || DIR == 1;   // A^T tiles are always transposed in shared memory
  extern __shared__ uint8_t smem_dyn[];
  // 128-byte-swizzled tiles need 1024-byte aligned shared addresses
  uint8_t* smem = smem_dyn + ((1024u - (smem_u32(smem_dyn) & 1023u)) & 1023u);
  uint8_t* a_tiles = smem;                                   // kStages x 32 KB
  uint8_t* x_tiles = smem + kStages * kATileBytes;           // kStages x 16 KB
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
  // bars: full[S], empty[S], conv[S], tfull[2], tempty[2]; then the TMEM address
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * kStages + 4);
  double* fro_red = reinterpret_cast<double*>(bars + 3 * kStages + 6);   // 4 doubles + abort flag
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + kStages), conv0 = smem_u32(bars + 2 * kStages);
  const uint32_t tfull0 = smem_u32(bars + 3 * kStages), tempty0 = smem_u32(bars + 3 * kStages + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t KB = cdiv(args.K, kTcBK);
  StreamK sk(cdiv(args.len, kTcBN), KB, gridDim.x);
  const int64_t s = sk.start(blockIdx.x), e = sk.start(blockIdx.x + 1);

  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(full0 + 8 * i, 1);
      mbar_init(empty0 + 8 * i, 1);
      mbar_init(conv0 + 8 * i, 4);
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
      int64_t n = 0;       // fills issued by this CTA
      bool ok = true;
      for (int64_t it = s; it < e; ++it, ++n) {
        const int stage = (int)(n % kStages);
        const uint32_t ph = (uint32_t)((n / kStages) & 1);
        if (!mbar_wait(empty0 + 8 * stage, ph ^ 1, args.status)) { ok = false; break; }
        const int64_t t = it / KB, kb = it - t * KB;
        const int k0 = (int)(kb * kTcBK);
        const int p0 = (int)(t * kTcBN);
        const uint32_t fb = full0 + 8 * stage;
        mbar_arrive_expect_tx(fb, kStageBytes);
        const uint32_t adst = smem_u32(a_tiles + stage * kATileBytes);
        if (DIR == 0) {
          tma_load_2d(adst, &mapA, fb, k0, p0, pol_a);                       // 256 rows x 32 cols
        } else {
#pragma unroll
          for (int c = 0; c < kTcBN / 32; ++c)                               // 8 x (32 rows x 32 cols)
            tma_load_2d(adst + c * (kTcBK * 128), &mapA, fb, p0 + 32 * c, k0, pol_a);
        }
        tma_load_2d(smem_u32(x_tiles + stage * kXTileBytes), &mapX, fb, k0, 0, pol_x);
      }
      // drain: every issued fill must have been consumed (released by the MMA
      // commit) before the CTA may exit; on an aborted run wait for the copies.
      const int64_t first = n > kStages ? n - kStages : 0;
      for (int64_t f = first; f < n; ++f) {
        const int stage = (int)(f % kStages);
        const uint32_t ph = (uint32_t)((f / kStages) & 1);
        if (ok) {
          if (!mbar_wait(empty0 + 8 * stage, ph, args.status)) ok = false;
        }
        if (!ok) mbar_wait(full0 + 8 * stage, ph, args.status);
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_tf32(kTcM, kTcBN, 0, 0);   // both operands K-major
      const uint32_t ready0 = kConvWarps ? conv0 : full0;
      int64_t n = 0;     // fills consumed
      int seg = 0;       // tile segments started
      bool ok = true;
      int64_t it = s;
      while (it < e && ok) {
        const int64_t t = it / KB;
        const int64_t kb1 = (e - t * KB < KB) ? (e - t * KB) : KB;
        const int b = seg & 1;
        const uint32_t tph = (uint32_t)((seg >> 1) & 1);
        if (!mbar_wait(tempty0 + 8 * b, tph ^ 1, args.status)) { ok = false; break; }
        tc_fence_after();
        const uint32_t tacc = tmem_base + (uint32_t)(b * kTcBN);
        bool first = true;
        for (; it < t * KB + kb1; ++it, ++n) {
          const int stage = (int)(n % kStages);
          const uint32_t ph = (uint32_t)((n / kStages) & 1);
          if (!mbar_wait(ready0 + 8 * stage, ph, args.status)) { ok = false; break; }
          tc_fence_after();
          const uint32_t abase = smem_u32(a_tiles + stage * kATileBytes);
          const uint32_t xbase = smem_u32(x_tiles + stage * kXTileBytes);
#pragma unroll
          for (int kk = 0; kk < kTcBK / 8; ++kk) {
            const uint64_t adesc = smem_desc(xbase + kk * 32, 16, 1024);
            const uint64_t bdesc = smem_desc(abase + kk * 32, 16, 1024);
            mma_tf32(tacc, adesc, bdesc, idesc, (first && kk == 0) ? 0u : 1u);
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
    const int g = warp & 3;                  // TMEM lane quarter this warp may access
    const int j = 32 * g + lane;             // output row (sketch column)
    int seg = 0;
    int64_t it = s;
    while (it < e) {
      const int64_t t = it / KB;
      const int64_t kb0 = it - t * KB;
      const int64_t kb1 = (e - t * KB < KB) ? (e - t * KB) : KB;
      const int b = seg & 1;
      const uint32_t tph = (uint32_t)((seg >> 1) & 1);
      if (!mbar_wait(tfull0 + 8 * b, tph, args.status)) break;
      tc_fence_after();
      const bool complete = (kb0 == 0 && kb1 == KB);
      const int64_t p0 = t * kTcBN;
      float* dst;
      int64_t lim;
      if (complete) {
        dst = args.Ct + (int64_t)j * args.ldc + p0;
        lim = args.len - p0;
      } else {
        dst = args.partials + ((int64_t)sk.slot(blockIdx.x, t) * kTcM + j) * kTcBN;
        lim = kTcBN;
      }
#pragma unroll 1
      for (int c = 0; c < kTcBN / 32; ++c) {
        float v[32];
        tmem_ld32(tmem_base + (uint32_t)(b * kTcBN + 32 * c) + ((uint32_t)(32 * g) << 16), v);
        if (j < args.l) {
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
      it = t * KB + kb1;
    }
  } else if (kConvWarps) {
    // ---------------------------------------------------------------- converter (warps 6..9)
    const int ct = threadIdx.x - 192;       // 0..127
    volatile int* conv_abort = reinterpret_cast<volatile int*>(fro_red + 4);
    if (ct == 0) *conv_abort = 0;
    asm volatile("bar.sync 1, 128;" ::: "memory");
    double fro = 0.0;
    int64_t n = 0;
    for (int64_t it = s; it < e; ++it, ++n) {
      const int stage = (int)(n % kStages);
      const uint32_t ph = (uint32_t)((n / kStages) & 1);
      if (DIR == 0) {
        if (!mbar_wait(full0 + 8 * stage, ph, args.status)) break;
      } else {
        // the transpose synchronises the four converter warps: they give up together
        if (!mbar_wait(full0 + 8 * stage, ph, args.status)) *conv_abort = 1;
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (*conv_abort) break;
      }
      uint8_t* tile = a_tiles + stage * kATileBytes;
      float part = 0.f;
      if (DIR == 0) {
        // rows of A are already K-major: round in place
        float4* a4 = reinterpret_cast<float4*>(tile);
#pragma unroll 4
        for (int q = ct; q < kATileBytes / 16; q += 128) {
          float4 v = a4[q];
          if (FRO) part = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, part))));
          if (CONV) {
            v.x = to_tf32(v.x); v.y = to_tf32(v.y); v.z = to_tf32(v.z); v.w = to_tf32(v.w);
            a4[q] = v;
          }
        }
      } else {
        // A^T tile: loaded as 8 column chunks [c][k][32 n] (128-byte swizzle); rewrite it in
        // place as the K-major tile [n][32 k] the MMA reads.  Thread block b covers
        // k = 4 kb .. 4 kb + 3, n = 4 nb .. 4 nb + 3 (kb = q / 64, nb = q % 64).
        float4 blk[4][4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int q = ct + 128 * b, kb = q >> 6, nb = q & 63;
          const int c = nb >> 3, ch = nb & 7;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int k = 4 * kb + i;
            blk[b][i] = *reinterpret_cast<const float4*>(tile + c * 4096 + k * 128 + ((ch ^ (k & 7)) << 4));
          }
        }
        // all four converter warps must finish reading before anyone overwrites the tile
        asm volatile("bar.sync 1, 128;" ::: "memory");
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int q = ct + 128 * b, kb = q >> 6, nb = q & 63;
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const int j = (jj + (nb >> 1)) & 3;        // rotate rows: conflict-free stores
            float4 v;
            v.x = sel_comp(blk[b][0], j); v.y = sel_comp(blk[b][1], j);
            v.z = sel_comp(blk[b][2], j); v.w = sel_comp(blk[b][3], j);
            if (FRO) part = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, part))));
            if (CONV) { v.x = to_tf32(v.x); v.y = to_tf32(v.y); v.z = to_tf32(v.z); v.w = to_tf32(v.w); }
            const int nrow = 4 * nb + j;
            *reinterpret_cast<float4*>(tile + nrow * 128 + ((kb ^ (nrow & 7)) << 4)) = v;
          }
        }
      }
      fro += (double)part;
      // generic-proxy writes must be visible to the tensor core (async proxy)
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
  if (FRO && threadIdx.x == 0) args.fro_parts[blockIdx.x] = (fro_red[0] + fro_red[1]) + (fro_red[2] + fro_red[3]);
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem_base) : "memory");
  }
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2-D row-major fp32 matrix (rows x cols, leading dimension ld elements), box
// (box_cols x box_rows), 128-byte swizzle, zero fill out of bounds.
bool make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_cols,
              int box_rows) {
  auto enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

size_t tc_pass_partial_bytes(int64_t len, int64_t K, int sms) {
  (void)len;
  (void)K;
  return (size_t)2 * sms * kTcM * kTcBN * sizeof(float);
}

int tc_pass_grid(int64_t len, int64_t K, int sms) {
  const int64_t total = cdiv(len, kTcBN) * cdiv(K, kTcBK);
  return (int)(sms < total ? sms : total);
}

// mma 1: TF32 with operands rounded to nearest (A in shared memory, X by the caller);
// mma 4: TF32 as the tensor core truncates (no conversion).
bool tc_pass_supported(int dir, int a_dtype, int mma, int l) {
  return (dir == 0 || dir == 1) && a_dtype == 1 && (mma == 1 || mma == 4) && l >= 1 && l <= kTcM;
}

template <int DIR, bool CONV, bool FRO>
static cudaError_t launch_variant(const CUtensorMap& mapA, const CUtensorMap& mapX, const TcArgs& ta, int64_t G,
                                  cudaStream_t st) {
  auto kern = pass_tc_kernel<DIR, CONV, FRO>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (err != cudaSuccess) return err;
  const int threads = (CONV || FRO || DIR == 1) ? kThreadsMax : kThreads;
  kern<<<(unsigned)G, threads, kSmemBytes, st>>>(mapA, mapX, ta);
  CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

template <int DIR>
static cudaError_t launch_dir_tc(const CUtensorMap& mapA, const CUtensorMap& mapX, const TcArgs& ta, bool conv,
                                 bool fro, int64_t G, cudaStream_t st) {
  if (conv && fro) return launch_variant<DIR, true, true>(mapA, mapX, ta, G, st);
  if (conv) return launch_variant<DIR, true, false>(mapA, mapX, ta, G, st);
  if (fro) return launch_variant<DIR, false, true>(mapA, mapX, ta, G, st);
  return launch_variant<DIR, false, false>(mapA, mapX, ta, G, st);
}

cudaError_t launch_pass_tc(const PassArgs& a, int dir, int a_dtype, int mma, int sms, DevStatus* status,
                           double* fro_parts, cudaStream_t st) {
  if (!tc_pass_supported(dir, a_dtype, mma, a.l)) return cudaErrorInvalidValue;
  CUtensorMap mapA, mapX;
  // A: m rows x n cols (row-major, lda)
  if (dir == 0) {
    if (!make_map(&mapA, a.A, a.m, a.n, a.lda, kTcBK, kTcBN)) return cudaErrorInvalidValue;
  } else {
    if (!make_map(&mapA, a.A, a.m, a.n, a.lda, 32, kTcBK)) return cudaErrorInvalidValue;
  }
  // Xt: l rows x K cols; the 128-row box reads zeros below row l
  if (!make_map(&mapX, a.Xt, a.l, a.K, a.ldx, kTcBK, kTcM)) return cudaErrorInvalidValue;
  const int64_t G = tc_pass_grid(a.len_out, a.K, sms);
  if (G <= 0) return cudaSuccess;
  TcArgs ta{static_cast<float*>(a.Ct), a.ldc, static_cast<float*>(a.partials), a.len_out, a.K, a.l, status,
            fro_parts};
  const bool conv = (mma == 1), fro = fro_parts != nullptr;
  cudaError_t err = dir == 0 ? launch_dir_tc<0>(mapA, mapX, ta, conv, fro, G, st)
                             : launch_dir_tc<1>(mapA, mapX, ta, conv, fro, G, st);
  if (err != cudaSuccess) return err;
  // ordered reduction of split tiles
  return launch_streamk_reduce_f32(static_cast<float*>(a.Ct), a.ldc, static_cast<const float*>(a.partials), a.l,
                                   kTcM, kTcBN, a.len_out, cdiv(a.K, kTcBK), G, st);
}

// Xr = TF32(X) rounded to nearest, l rows of `len` (the sketch operand of a rounded pass).
__global__ void round_tf32_kernel(const float* __restrict__ X, int64_t ldx, float* __restrict__ Xr, int64_t ldr,
                                  int l, int64_t len) {
  const int j = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    Xr[j * ldr + i] = to_tf32(X[j * ldx + i]);
}

cudaError_t launch_round_tf32(const float* X, int64_t ldx, float* Xr, int64_t ldr, int l, int64_t len,
                              cudaStream_t st) {
  dim3 grid((unsigned)(cdiv(len, 256) < 64 ? cdiv(len, 256) : 64), (unsigned)l);
  if (grid.x == 0) return cudaSuccess;
  round_tf32_kernel<<<grid, 256, 0, st>>>(X, ldx, Xr, ldr, l, len);
  CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

}  // namespace corutv
