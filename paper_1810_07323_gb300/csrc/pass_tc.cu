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
#include "tc_common.cuh"

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
    tc_epilogue<kTcBN, kTcM>(args.Ct, args.ldc, args.partials, args.len, args.l, KB, sk, s, e, tmem_base, tfull0,
                             tempty0, args.status);
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
      const float part = DIR == 0 ? tc_conv_rows_tf32<CONV, FRO>(tile, ct) : tc_conv_transpose_tf32<CONV, FRO>(tile, ct);
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
// 2-D row-major fp32 matrix, box (box_cols x box_rows), 128-byte swizzle.
bool make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_cols,
              int box_rows) {
  return make_map_2d(map, base, rows, cols, ld, 4, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, box_cols, box_rows, true);
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
  if (a.kmark) a.kmark->start(st);
  cudaError_t err = dir == 0 ? launch_dir_tc<0>(mapA, mapX, ta, conv, fro, G, st)
                             : launch_dir_tc<1>(mapA, mapX, ta, conv, fro, G, st);
  if (err != cudaSuccess) return err;
  if (a.kmark) a.kmark->stop(st);
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
