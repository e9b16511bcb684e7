// Spectral readout of a factorisation (the quality measure of Sec. VI-B, e_k,2):
//     ||R||_2,  R = A - U(:, 1:k) T(1:k, :) V^T,
// estimated by power iteration on R^T R with R applied as an operator (never
// formed): per step y = R x, ||y||, x = R^T y / ||R^T y||; the estimate is
// ||R x|| for the last x.  A X-type products read A once each (HBM-bound).
//
// FP32 A: the long dot products use Ogita-Rump-Oishi Dot2 (TwoProd by FMA,
// TwoSum of the running sum; "Accurate sum and dot product", SIAM J. Sci.
// Comput. 26, 2005), so A x carries about twice the working precision before
// the low-rank part U_k (T_k V^T x) -- formed in FP64 -- is subtracted: the
// residual is orders of magnitude smaller than A x, and a plain FP32 sum would
// leave its error amplified by that ratio.  The vectors are stored in the
// storage precision; norms and the l-vectors are FP64.  FP64 A: FP64
// throughout.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "handle.h"
#include "internal.h"

namespace corutv {

namespace {

constexpr int kResRows = 8;        // warps (rows) per CTA of the row products
constexpr int kResColChunks = 32;  // row ranges of the column products
constexpr int kResParts = 152;     // CTAs of the l-vector partial sums

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void add2(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// Dot2 step: (s, c) += a x with the product and the sum error kept
struct Dot2 {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float a, float x) {
    const float p = __fmul_rn(a, x);
    const float pe = fmaf(a, x, -p);
    float t, e;
    add2(s, p, t, e);
    s = t;
    c = __fadd_rn(c, __fadd_rn(e, pe));
  }
  __device__ __forceinline__ void merge(const Dot2& o) {
    float t, e;
    add2(s, o.s, t, e);
    s = t;
    c = __fadd_rn(c, __fadd_rn(e, o.c));
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

template <typename TA>
struct RowAcc;                       // accumulator of one dot product in the storage type's scheme
template <>
struct RowAcc<float> {
  Dot2 d;
  __device__ __forceinline__ void add(float a, float x) { d.add(a, x); }
  __device__ __forceinline__ void shfl_merge(int o) {
    Dot2 t;
    t.s = __shfl_xor_sync(0xffffffffu, d.s, o);
    t.c = __shfl_xor_sync(0xffffffffu, d.c, o);
    d.merge(t);
  }
  __device__ __forceinline__ double value() const { return d.value(); }
};
template <>
struct RowAcc<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double a, double x) { v = fma(a, x, v); }
  __device__ __forceinline__ void shfl_merge(int o) { v += __shfl_xor_sync(0xffffffffu, v, o); }
  __device__ __forceinline__ double value() const { return v; }
};

// w partials: part[b][a] = sum over rows r of chunk b of M[r][a] v[r], a < na (M row-major, ld ldm)
template <typename TA>
__global__ void __launch_bounds__(256) resid_mtv_part_kernel(const TA* __restrict__ M, int64_t ldm, int64_t rows,
                                                             int na, const TA* __restrict__ v,
                                                             double* __restrict__ part) {
  __shared__ double acc[8][kMaxL];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int a = lane; a < kMaxL; a += 32) acc[warp][a] = 0.0;
  const int64_t chunk = cdiv(rows, (int64_t)gridDim.x);
  const int64_t r0 = blockIdx.x * chunk, r1 = r0 + chunk < rows ? r0 + chunk : rows;
  double mine[kMaxL / 32];
#pragma unroll
  for (int u = 0; u < kMaxL / 32; ++u) mine[u] = 0.0;
  for (int64_t r = r0 + warp; r < r1; r += 8) {
    const double vr = (double)v[r];
#pragma unroll
    for (int u = 0; u < kMaxL / 32; ++u) {
      const int a = lane + 32 * u;
      if (a < na) mine[u] = fma((double)M[r * ldm + a], vr, mine[u]);
    }
  }
#pragma unroll
  for (int u = 0; u < kMaxL / 32; ++u) acc[warp][lane + 32 * u] = mine[u];
  __syncthreads();
  for (int a = tid; a < na; a += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += acc[w][a];
    part[(int64_t)blockIdx.x * kMaxL + a] = s;
  }
}

// z = op(T_k) w with w = the ordered sum of the partials; transpose = 0: z (k) = T(1:k, :) w (w: l),
// transpose = 1: z (l) = T(1:k, :)^T w (w: k)
__global__ void __launch_bounds__(256) resid_coef_kernel(const double* __restrict__ part, int nparts, int nw,
                                                         const double* __restrict__ T, int64_t ldt, int k, int l,
                                                         int transpose, double* __restrict__ z) {
  __shared__ double w[kMaxL];
  for (int a = threadIdx.x; a < nw; a += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += part[(int64_t)b * kMaxL + a];
    w[a] = s;
  }
  __syncthreads();
  const int nz = transpose ? l : k;
  for (int i = threadIdx.x; i < nz; i += blockDim.x) {
    double s = 0.0;
    if (!transpose)
      for (int a = 0; a < l; ++a) s = fma(T[i * ldt + a], w[a], s);
    else
      for (int a = 0; a < k; ++a) s = fma(T[a * ldt + i], w[a], s);
    z[i] = s;
  }
}

// y = A x - U_k z (one warp per row), and the CTA's share of ||y||^2
template <typename TA>
__global__ void __launch_bounds__(kResRows * 32) resid_row_kernel(const TA* __restrict__ A, int64_t lda, int64_t m,
                                                                  int64_t n, const TA* __restrict__ x,
                                                                  const TA* __restrict__ U, int64_t ldu, int k,
                                                                  const double* __restrict__ z, TA* __restrict__ y,
                                                                  double* __restrict__ nparts) {
  __shared__ double red[kResRows];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * kResRows + warp;
  double yi = 0.0;
  if (i < m) {
    RowAcc<TA> acc;
    const TA* Ai = A + i * lda;
    for (int64_t j = lane; j < n; j += 32) acc.add(Ai[j], x[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc.shfl_merge(o);
    double corr = 0.0;
    for (int a = lane; a < k; a += 32) corr = fma((double)U[i * ldu + a], z[a], corr);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) corr += __shfl_xor_sync(0xffffffffu, corr, o);
    const TA yv = (TA)(acc.value() - corr);
    if (lane == 0) y[i] = yv;
    yi = (double)yv;
  }
  if (lane == 0) red[warp] = yi * yi;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kResRows; ++w) s += red[w];
    nparts[blockIdx.x] = s;
  }
}

// column products over row range c: colpart[c][j] = sum over rows i of range c of A[i][j] y[i]
template <typename TA>
__global__ void __launch_bounds__(256) resid_col_kernel(const TA* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                                                        const TA* __restrict__ y, double* __restrict__ colpart) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t chunk = cdiv(m, (int64_t)gridDim.y);
  const int64_t r0 = blockIdx.y * chunk, r1 = r0 + chunk < m ? r0 + chunk : m;
  if (j >= n) return;
  RowAcc<TA> acc;
  for (int64_t i = r0; i < r1; ++i) acc.add(A[i * lda + j], y[i]);
  colpart[(int64_t)blockIdx.y * n + j] = acc.value();
}

// x = sum of the column ranges - V z, and the CTA's share of ||x||^2
template <typename TA>
__global__ void __launch_bounds__(256) resid_colfin_kernel(const double* __restrict__ colpart, int nranges, int64_t n,
                                                           const TA* __restrict__ V, int64_t ldv, int l,
                                                           const double* __restrict__ z, TA* __restrict__ x,
                                                           double* __restrict__ nparts) {
  __shared__ double red[8];
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double xj2 = 0.0;
  if (j < n) {
    double s = 0.0;
    for (int c = 0; c < nranges; ++c) s += colpart[(int64_t)c * n + j];
    double corr = 0.0;
    for (int a = 0; a < l; ++a) corr = fma((double)V[j * ldv + a], z[a], corr);
    const TA xv = (TA)(s - corr);
    x[j] = xv;
    xj2 = (double)xv * (double)xv;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) xj2 += __shfl_xor_sync(0xffffffffu, xj2, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = xj2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    nparts[blockIdx.x] = s;
  }
}

// ||v||^2 of a vector (first use: the caller's start vector), one CTA-partial per block
template <typename TA>
__global__ void __launch_bounds__(256) resid_sq_kernel(const TA* __restrict__ v, int64_t len,
                                                       double* __restrict__ nparts) {
  __shared__ double red[8];
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double s = j < len ? (double)v[j] * (double)v[j] : 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    nparts[blockIdx.x] = t;
  }
}

// scal[0] = sqrt(sum of the partials) in block order; dst = src / scal[0] (dst may be src; zero stays zero)
template <typename TA>
__global__ void __launch_bounds__(256) resid_scale_kernel(const double* __restrict__ nparts, int np,
                                                          const TA* src, TA* dst, int64_t len,
                                                          double* __restrict__ scal) {
  __shared__ double nrm;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < np; ++b) s += nparts[b];
    nrm = sqrt(s);
    if (blockIdx.x == 0) scal[0] = nrm;
  }
  __syncthreads();
  if (!dst) return;
  const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < len; j += (int64_t)gridDim.x * blockDim.x)
    dst[j] = (TA)((double)src[j] * inv);
}

struct ResidWs {
  void *x, *y;
  double *wpart, *z, *colpart, *nparts, *scal;
};

size_t resid_layout(ResidWs& w, void* base, int64_t m, int64_t n, int eb) {
  char* p = static_cast<char*>(base);
  size_t off = 0;
  auto take = [&](size_t b) {
    off = (size_t)round_up((int64_t)off, 256);
    void* r = p ? p + off : nullptr;
    off += b;
    return r;
  };
  w.x = take((size_t)n * eb);
  w.y = take((size_t)m * eb);
  w.wpart = static_cast<double*>(take(sizeof(double) * kResParts * kMaxL));
  w.z = static_cast<double*>(take(sizeof(double) * kMaxL));
  w.colpart = static_cast<double*>(take(sizeof(double) * kResColChunks * n));
  const int64_t nb = std::max(cdiv(m, (int64_t)kResRows), cdiv(n, (int64_t)256));
  w.nparts = static_cast<double*>(take(sizeof(double) * nb));
  w.scal = static_cast<double*>(take(sizeof(double) * 4));
  return (size_t)round_up((int64_t)off, 256);
}

template <typename TA>
cudaError_t resid_run(const ResidWs& w, const TA* A, int64_t lda, int64_t m, int64_t n, const TA* U, int64_t ldu,
                      const double* T, int64_t ldt, const TA* V, int64_t ldv, int l, int k, const TA* x0, int iters,
                      cudaStream_t st, int64_t* launches) {
  TA* x = static_cast<TA*>(w.x);
  TA* y = static_cast<TA*>(w.y);
  const unsigned gn = (unsigned)cdiv(n, (int64_t)256);
  const unsigned gm_rows = (unsigned)cdiv(m, (int64_t)kResRows);
  const int pv = (int)std::min<int64_t>(kResParts, n), pu = (int)std::min<int64_t>(kResParts, m);
  // x = x0 / ||x0||
  resid_sq_kernel<TA><<<gn, 256, 0, st>>>(x0, n, w.nparts);
  resid_scale_kernel<TA><<<gn, 256, 0, st>>>(w.nparts, (int)gn, x0, x, n, w.scal);
  *launches += 2;
  auto apply_r = [&]() {
    // y = A x - U_k (T_k (V^T x))
    resid_mtv_part_kernel<TA><<<pv, 256, 0, st>>>(V, ldv, n, l, x, w.wpart);
    resid_coef_kernel<<<1, 256, 0, st>>>(w.wpart, pv, l, T, ldt, k, l, 0, w.z);
    resid_row_kernel<TA><<<gm_rows, kResRows * 32, 0, st>>>(A, lda, m, n, x, U, ldu, k, w.z, y, w.nparts);
    *launches += 3;
  };
  for (int it = 0; it < iters; ++it) {
    apply_r();
    // x = A^T y - V (T_k^T (U_k^T y)), then x / ||x||
    resid_mtv_part_kernel<TA><<<pu, 256, 0, st>>>(U, ldu, m, k, y, w.wpart);
    resid_coef_kernel<<<1, 256, 0, st>>>(w.wpart, pu, k, T, ldt, k, l, 1, w.z);
    resid_col_kernel<TA><<<dim3(gn, kResColChunks), 256, 0, st>>>(A, lda, m, n, y, w.colpart);
    resid_colfin_kernel<TA><<<gn, 256, 0, st>>>(w.colpart, kResColChunks, n, V, ldv, l, w.z, x, w.nparts);
    resid_scale_kernel<TA><<<gn, 256, 0, st>>>(w.nparts, (int)gn, x, x, n, w.scal);
    *launches += 5;
  }
  apply_r();
  resid_scale_kernel<TA><<<1, 256, 0, st>>>(w.nparts, (int)gm_rows, (const TA*)nullptr, (TA*)nullptr, 0, w.scal);
  *launches += 1;
  return cudaGetLastError();
}

}  // namespace

void resid_free(corutv_handle* h) {
  if (h->resid_ws) {
    cudaStreamSynchronize(h->stream);
    cudaFree(h->resid_ws);
  }
  h->resid_ws = nullptr;
  h->resid_ws_bytes = 0;
}

}  // namespace corutv

using namespace corutv;

extern "C" int corutv_residual_norm2(corutv_handle* h, int a_dtype, const void* A, int64_t lda, int64_t m, int64_t n,
                                     const void* U, int64_t ldu, const double* T, int64_t ldt, const void* V,
                                     int64_t ldv, int l, int k, const void* x0, int iters, double* out) {
  if (!h || !A || !U || !T || !V || !x0 || !out) return CORUTV_ERR_INVALID_ARG;
  if (a_dtype != CORUTV_F32 && a_dtype != CORUTV_F64) return CORUTV_ERR_UNSUPPORTED;
  if (m <= 0 || n <= 0 || l < 1 || l > kMaxL || k < 1 || k > l || iters < 0) return CORUTV_ERR_SHAPE;
  if (lda < n || ldu < l || ldv < l || ldt < l) return CORUTV_ERR_SHAPE;
  const int eb = a_dtype == CORUTV_F64 ? 8 : 4;
  ResidWs w{};
  const size_t need = resid_layout(w, nullptr, m, n, eb);
  if (!h->resid_ws || h->resid_ws_bytes < need) {
    resid_free(h);
    if (cudaMalloc(&h->resid_ws, need) != cudaSuccess) {
      cudaGetLastError();
      h->resid_ws = nullptr;
      return CORUTV_ERR_OOM;
    }
    h->resid_ws_bytes = need;
  }
  resid_layout(w, h->resid_ws, m, n, eb);
  int64_t nl = 0;
  cudaError_t e;
  if (a_dtype == CORUTV_F64)
    e = resid_run<double>(w, static_cast<const double*>(A), lda, m, n, static_cast<const double*>(U), ldu, T, ldt,
                          static_cast<const double*>(V), ldv, l, k, static_cast<const double*>(x0), iters, h->stream,
                          &nl);
  else
    e = resid_run<float>(w, static_cast<const float*>(A), lda, m, n, static_cast<const float*>(U), ldu, T, ldt,
                         static_cast<const float*>(V), ldv, l, k, static_cast<const float*>(x0), iters, h->stream,
                         &nl);
  launch_counter() += nl;
  h->launches += nl;
  if (e != cudaSuccess) return CORUTV_ERR_CUDA;
  if (cudaMemcpyAsync(out, w.scal, sizeof(double), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return CORUTV_ERR_CUDA;
  return CORUTV_OK;
}
