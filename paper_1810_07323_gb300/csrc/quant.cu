// Storage conversion of A for the low-precision passes: FP32 -> BF16 (round to
// nearest even), or FP32 -> FP8 e4m3 with one FP32 scale per 128 x 128 tile.
// The tile scale is the smallest power of two >= fl32(amax / 448), so that
// a / scale is exact, lies in [-448, 448] and rounds once (to nearest even,
// saturating) to e4m3; dequantisation e4m3 * scale is then exact in BF16 and
// FP32.  One CTA per tile.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace corutv {
namespace {

constexpr int kQT = 128;       // tile edge
constexpr int kQThreads = 256;

// smallest power of two >= x for finite x > 0 (FP32, normal range of the result)
__device__ __forceinline__ float pow2_ceil(float x) {
  const uint32_t b = __float_as_uint(x);
  uint32_t e = (b >> 23) & 0xFFu;
  if (e == 0) return __uint_as_float(1u << 23);         // subnormal quotient: 2^-126
  if (b & 0x7FFFFFu) ++e;
  return __uint_as_float(e << 23);
}

__global__ void __launch_bounds__(kQThreads) quant_fp8_kernel(const float* __restrict__ A, int64_t lda, int64_t m,
                                                              int64_t n, uint8_t* __restrict__ out, int64_t ldo,
                                                              float* __restrict__ scales, int64_t sld) {
  const int64_t r0 = (int64_t)blockIdx.y * kQT, c0 = (int64_t)blockIdx.x * kQT;
  const int c = threadIdx.x & (kQT - 1), rr = threadIdx.x >> 7;   // column, row parity
  const bool col_ok = c0 + c < n;
  float amax = 0.f;
  for (int r = rr; r < kQT; r += 2) {
    const int64_t i = r0 + r;
    if (i < m && col_ok) amax = fmaxf(amax, fabsf(A[i * lda + c0 + c]));
  }
  __shared__ float red[kQThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = amax;
  __syncthreads();
  float t = red[0];
#pragma unroll
  for (int w = 1; w < kQThreads / 32; ++w) t = fmaxf(t, red[w]);
  const float scale = t > 0.f ? pow2_ceil(t / 448.f) : 1.f;
  const float inv = __uint_as_float((254u - ((__float_as_uint(scale) >> 23) & 0xFFu)) << 23);   // 1 / scale, exact
  if (threadIdx.x == 0) scales[blockIdx.y * sld + blockIdx.x] = scale;
  for (int r = rr; r < kQT; r += 2) {
    const int64_t i = r0 + r;
    if (i < m && col_ok)
      out[i * ldo + c0 + c] = (uint8_t)__nv_cvt_float_to_fp8(A[i * lda + c0 + c] * inv, __NV_SATFINITE, __NV_E4M3);
  }
}

__global__ void __launch_bounds__(kQThreads) quant_bf16_kernel(const float* __restrict__ A, int64_t lda, int64_t m,
                                                               int64_t n, __nv_bfloat16* __restrict__ out,
                                                               int64_t ldo) {
  const int64_t r0 = (int64_t)blockIdx.y * kQT, c0 = (int64_t)blockIdx.x * kQT;
  const int c = threadIdx.x & (kQT - 1), rr = threadIdx.x >> 7;
  if (c0 + c >= n) return;
  for (int r = rr; r < kQT; r += 2) {
    const int64_t i = r0 + r;
    if (i < m) out[i * ldo + c0 + c] = __float2bfloat16_rn(A[i * lda + c0 + c]);
  }
}

}  // namespace

cudaError_t launch_quantize(int dtype, const float* A, int64_t lda, int64_t m, int64_t n, void* out, int64_t ldo,
                            float* scales, cudaStream_t st) {
  const dim3 grid((unsigned)cdiv(n, kQT), (unsigned)cdiv(m, kQT));
  if (dtype == 3) {
    quant_fp8_kernel<<<grid, kQThreads, 0, st>>>(A, lda, m, n, static_cast<uint8_t*>(out), ldo, scales, cdiv(n, kQT));
  } else if (dtype == 2) {
    quant_bf16_kernel<<<grid, kQThreads, 0, st>>>(A, lda, m, n, static_cast<__nv_bfloat16*>(out), ldo);
  } else {
    return cudaErrorInvalidValue;
  }
  CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

}  // namespace corutv
