// Element access for the storage types of A (FP64, FP32, BF16, FP8 e4m3 with
// per-128x128-tile scales).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace corutv {

template <typename T> struct Elem;

template <> struct Elem<double> {
  using acc = double;
  __device__ static double load(const double* p, int64_t i, int64_t j, int64_t ld, const float*, int64_t) {
    return p[i * ld + j];
  }
};
template <> struct Elem<float> {
  using acc = float;
  __device__ static float load(const float* p, int64_t i, int64_t j, int64_t ld, const float*, int64_t) {
    return p[i * ld + j];
  }
};
template <> struct Elem<__nv_bfloat16> {
  using acc = float;
  __device__ static float load(const __nv_bfloat16* p, int64_t i, int64_t j, int64_t ld, const float*, int64_t) {
    return __bfloat162float(p[i * ld + j]);
  }
};
template <> struct Elem<__nv_fp8_e4m3> {
  using acc = float;
  // scales: ceil(m/128) x ceil(n/128), row-major with `sld` columns
  __device__ static float load(const __nv_fp8_e4m3* p, int64_t i, int64_t j, int64_t ld, const float* scales,
                               int64_t sld) {
    return float(p[i * ld + j]) * scales[(i >> 7) * sld + (j >> 7)];
  }
};

}  // namespace corutv
