// Gram partials on the tensor cores: parts[c] = X[:, cols_c] Y[:, cols_c]^T for
// two skinny-transposed blocks (l <= 128 rows of `len` FP32 columns), the
// C^T C of CholeskyQR (Sec. III, QR of C1 and C2) and the core Q1^T (A Q2)
// (Alg. 2 step 5), to FP32 accuracy with three TF32 products ("3xTF32"):
// every operand element is split x = hi + lo, hi = TF32(x) and lo = TF32(x - hi)
// (both rounded to nearest), and X Y^T ~ Xhi Yhi^T + Xhi Ylo^T + Xlo Yhi^T,
// the dropped Xlo Ylo^T being ~2^-22 of |X||Y|.
//
// One CTA per contiguous range of 32-column k-blocks: warp 0 loads the X (and
// Y) blocks by TMA (128 rows x 32 columns, 128-byte swizzle, rows >= l read
// as zero), warps 2..5 split them into hi / lo tiles in shared memory, warp 1
// issues tcgen05.mma.kind::tf32 (M = N = 128, K = 8) into a 128 x 128 FP32
// TMEM accumulator, and warps 2..5 write it out as the CTA's partial (the
// ordered compensated reduction of small.cu sums the partials).  Every wait
// is bounded; on expiry the status word records a timeout and the CTA frees
// its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace corutv {

namespace {

constexpr int kGM = 128;                       // rows of X (MMA M) and of Y (MMA N)
constexpr int kGK = 32;                        // FP32 columns per k-block (one swizzle row)
constexpr int kGStages = 3;
constexpr int kGTile = kGM * kGK * 4;          // 16 KB
constexpr int kGStageBytes = 4 * kGTile;       // X hi, X lo, Y hi, Y lo
constexpr int kGSmem = kGStages * kGStageBytes + 1024 /*align*/ + 256 /*barriers*/;
constexpr int kGThreads = 192;                 // warp 0 TMA, warp 1 MMA, warps 2..5 split + epilogue
constexpr int kGMinKb = 16;                    // k-blocks per CTA at least (fewer, fuller partials)

// hi = TF32(x), lo = TF32(x - hi) over one 128 x 32 tile (element-wise: the swizzle does not matter)
__device__ __forceinline__ void split_tile(uint8_t* hi_tile, uint8_t* lo_tile, int ct) {
  float4* h4 = reinterpret_cast<float4*>(hi_tile);
  float4* l4 = reinterpret_cast<float4*>(lo_tile);
#pragma unroll
  for (int q = 0; q < kGTile / 16 / 128; ++q) {
    const int e = ct + 128 * q;
    const float4 x = h4[e];
    const float4 h = make_float4(to_tf32(x.x), to_tf32(x.y), to_tf32(x.z), to_tf32(x.w));
    l4[e] = make_float4(to_tf32(x.x - h.x), to_tf32(x.y - h.y), to_tf32(x.z - h.z), to_tf32(x.w - h.w));
    h4[e] = h;
  }
}

template <bool SAME>
__global__ void __launch_bounds__(kGThreads, 1)
    gram_tc_kernel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapY, int64_t KB,
                   int64_t chunk, float* __restrict__ parts, DevStatus* status) {
  pdl_enter();
  extern __shared__ uint8_t smem_dyn[];
  uint8_t* smem = smem_dyn + ((1024u - (smem_u32(smem_dyn) & 1023u)) & 1023u);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kGStages * kGStageBytes);
  // bars: full[S], conv[S], empty[S], done; then the TMEM address
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * kGStages + 1);
  const uint32_t full0 = smem_u32(bars), conv0 = smem_u32(bars + kGStages), empty0 = smem_u32(bars + 2 * kGStages);
  const uint32_t done = smem_u32(bars + 3 * kGStages);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t kb0 = blockIdx.x * chunk;
  const int64_t kb1 = (kb0 + chunk < KB) ? kb0 + chunk : KB;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kGStages; ++i) {
      mbar_init(full0 + 8 * i, 1);
      mbar_init(conv0 + 8 * i, 4);
      mbar_init(empty0 + 8 * i, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(tmem_slot))
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
      const uint64_t pol = policy_evict_first();
      int64_t n = 0;
      bool ok = true;
      for (int64_t kb = kb0; kb < kb1; ++kb, ++n) {
        const int stage = (int)(n % kGStages);
        const uint32_t ph = (uint32_t)((n / kGStages) & 1);
        if (!mbar_wait(empty0 + 8 * stage, ph ^ 1, status)) { ok = false; break; }
        uint8_t* st = smem + stage * kGStageBytes;
        const uint32_t fb = full0 + 8 * stage;
        mbar_arrive_expect_tx(fb, SAME ? kGTile : 2 * kGTile);
        tma_load_2d(smem_u32(st), &mapX, fb, (int)(kb * kGK), 0, pol);
        if (!SAME) tma_load_2d(smem_u32(st + 2 * kGTile), &mapY, fb, (int)(kb * kGK), 0, pol);
      }
      // every issued fill must have been consumed before the CTA exits; on an abort wait for the copies
      const int64_t first = n > kGStages ? n - kGStages : 0;
      for (int64_t f = first; f < n; ++f) {
        const int stage = (int)(f % kGStages);
        const uint32_t ph = (uint32_t)((f / kGStages) & 1);
        if (ok) {
          if (!mbar_wait(empty0 + 8 * stage, ph, status)) ok = false;
        }
        if (!ok) mbar_wait(full0 + 8 * stage, ph, status);
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_tf32(kGM, kGM, 0, 0);   // both operands K-major
      int64_t n = 0;
      bool ok = true, first = true;
      for (int64_t kb = kb0; kb < kb1; ++kb, ++n) {
        const int stage = (int)(n % kGStages);
        const uint32_t ph = (uint32_t)((n / kGStages) & 1);
        if (!mbar_wait(conv0 + 8 * stage, ph, status)) { ok = false; break; }
        tc_fence_after();
        const uint32_t st = smem_u32(smem + stage * kGStageBytes);
        const uint32_t xh = st, xl = st + kGTile;
        const uint32_t yh = SAME ? xh : st + 2 * kGTile, yl = SAME ? xl : st + 3 * kGTile;
#pragma unroll
        for (int kk = 0; kk < kGK / 8; ++kk) {
          const uint32_t o = kk * 32;
          mma_tf32(tmem_base, smem_desc(xh + o, 16, 1024), smem_desc(yh + o, 16, 1024), idesc, first ? 0u : 1u);
          first = false;
          mma_tf32(tmem_base, smem_desc(xh + o, 16, 1024), smem_desc(yl + o, 16, 1024), idesc, 1u);
          mma_tf32(tmem_base, smem_desc(xl + o, 16, 1024), smem_desc(yh + o, 16, 1024), idesc, 1u);
        }
        mma_commit(empty0 + 8 * stage);
      }
      if (ok && kb1 > kb0) mma_commit(done);
    }
  } else {
    // ---------------------------------------------------------------- split (warps 2..5)
    const int ct = threadIdx.x - 64;   // 0..127
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    if (ct == 0) *abort_flag = 0;
    asm volatile("bar.sync 1, 128;" ::: "memory");
    int64_t n = 0;
    for (int64_t kb = kb0; kb < kb1; ++kb, ++n) {
      const int stage = (int)(n % kGStages);
      const uint32_t ph = (uint32_t)((n / kGStages) & 1);
      if (!mbar_wait(full0 + 8 * stage, ph, status)) *abort_flag = 1;
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (*abort_flag) break;
      uint8_t* st = smem + stage * kGStageBytes;
      split_tile(st, st + kGTile, ct);
      if (!SAME) split_tile(st + 2 * kGTile, st + 3 * kGTile, ct);
      // generic-proxy writes must be visible to the tensor core (async proxy)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(conv0 + 8 * stage);
    }
    // ---------------------------------------------------------------- epilogue: the CTA's partial
    const int g = warp & 3;                 // TMEM lane quarter of this warp
    const int j = 32 * g + lane;            // row of X
    float* dst = parts + ((int64_t)blockIdx.x * kGM + j) * kGM;
    const bool have = (kb1 > kb0) && !*abort_flag && mbar_wait(done, 0, status);
    if (have) tc_fence_after();
#pragma unroll 1
    for (int c = 0; c < kGM / 32; ++c) {
      float v[32];
      if (have) {
        tmem_ld32(tmem_base + (uint32_t)(32 * c) + ((uint32_t)(32 * g) << 16), v);
      } else {
#pragma unroll
        for (int q = 0; q < 32; ++q) v[q] = 0.f;
      }
      float4* d4 = reinterpret_cast<float4*>(dst + 32 * c);
#pragma unroll
      for (int q = 0; q < 8; ++q) d4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem_base) : "memory");
  }
}

}  // namespace

int gram_tc_parts(int64_t len, int sms) {
  const int64_t KB = cdiv(len, kGK);
  int64_t g = cdiv(KB, kGMinKb);
  if (g > sms) g = sms;
  return (int)(g < 1 ? 1 : g);
}

bool gram_tc_ok(const float* X, int64_t ldx, const float* Y, int64_t ldy, int l) {
  return l >= 1 && l <= kGM && ((uintptr_t)X & 15) == 0 && ((uintptr_t)Y & 15) == 0 && (ldx & 3) == 0 &&
         (ldy & 3) == 0;
}

// parts: gram_tc_parts(len, sms) blocks of 128 x 128 FP32
cudaError_t launch_gram_tc_partials(const float* X, int64_t ldx, const float* Y, int64_t ldy, int64_t len, int l,
                                    float* parts, int sms, DevStatus* status, cudaStream_t st) {
  CUtensorMap mapX, mapY;
  if (!make_map_2d(&mapX, X, l, len, ldx, 4, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, kGK, kGM, true))
    return cudaErrorInvalidValue;
  const bool same = X == Y && ldx == ldy;
  if (!same && !make_map_2d(&mapY, Y, l, len, ldy, 4, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, kGK, kGM, true))
    return cudaErrorInvalidValue;
  if (same) mapY = mapX;
  const int64_t KB = cdiv(len, kGK);
  const int G = gram_tc_parts(len, sms);
  const int64_t chunk = cdiv(KB, G);
  // the shared-memory limit is raised once per kernel and device
  constexpr int kDev = 64;
  static bool attr_done[2][kDev] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  bool* flag = (dev >= 0 && dev < kDev) ? &attr_done[same ? 0 : 1][dev] : nullptr;
  if (!flag || !*flag) {
    e = cudaFuncSetAttribute(same ? gram_tc_kernel<true> : gram_tc_kernel<false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kGSmem);
    if (e != cudaSuccess) return e;
    if (flag) *flag = true;
  }
  if (same)
    e = launch_pdl(gram_tc_kernel<true>, G, kGThreads, kGSmem, st, mapX, mapY, KB, chunk, parts, status);
  else
    e = launch_pdl(gram_tc_kernel<false>, G, kGThreads, kGSmem, st, mapX, mapY, KB, chunk, parts, status);
  if (e != cudaSuccess) return e;
  CORUTV_COUNT_LAUNCH();
  return cudaSuccess;
}

}  // namespace corutv
