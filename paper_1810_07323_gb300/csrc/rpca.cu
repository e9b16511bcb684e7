// Robust PCA by ALM-CoRUTV (Sec. V, Alg. 5 of the paper): M = L + S with L of
// low rank and S sparse.  Every iteration runs one CoR-UTV solve of
// B = M - S + Y / mu through the library's own solve, then
//   - a small kernel counts r = #{T_jj > 1/mu} and forms W^T = V T(1:r,:)^T
//     (n x l, columns p >= r zero), so that C_{1/mu}(B) = U W;
//   - one fused kernel forms each 64 x 64 tile of L = U W (FP32, K = r), and
//     with it the shrinkage S = S_{lambda/mu}(M - L + Y/mu), the multiplier
//     Y += mu (M - L - S) and the tile's share of ||M - L - S||_F^2;
// the host reads the residual back once per iteration for the stopping rule
// of Sec. VI-C.  B lives in L's memory until the fused kernel overwrites it.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <algorithm>

#include "../../include/corutv.h"
#include "common.cuh"
#include "handle.h"
#include "internal.h"

namespace corutv {
namespace {

constexpr int kRT = 64;        // output tile (rows and columns) of the fused update
constexpr int kRK = 32;        // K chunk
constexpr int kRP = kRT + 1;   // shared-memory pitch

// B = M - S + Y / mu (rows by CTA, columns by thread)
__global__ void __launch_bounds__(256) rpca_form_b_kernel(const float* __restrict__ M, int64_t ldm,
                                                          const float* __restrict__ S, int64_t lds,
                                                          const float* __restrict__ Y, int64_t ldy,
                                                          float* __restrict__ B, int64_t ldb, int64_t m, int64_t n,
                                                          float inv_mu) {
  for (int64_t i = blockIdx.x; i < m; i += gridDim.x)
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x)
      B[i * ldb + j] = fmaf(Y[i * ldy + j], inv_mu, M[i * ldm + j] - S[i * lds + j]);
}

// r = #{T_jj > delta} (every CTA counts; CTA 0 stores it) and
// Wt[j][p] = sum_c V[j][c] T[p][c] for p < r, 0 for r <= p < l (rows j of this CTA).
__global__ void __launch_bounds__(128) rpca_rank_w_kernel(const double* __restrict__ T, int64_t ldt,
                                                          const float* __restrict__ V, int64_t ldv, int64_t n,
                                                          int l, float delta, float* __restrict__ Wt, int64_t ldw,
                                                          int* __restrict__ r_out) {
  extern __shared__ float rw_smem[];
  const int LP1 = l + 1;
  float* Ts = rw_smem;                 // l x (l + 1)
  float* Vs = rw_smem + l * LP1;       // 32 x (l + 1)
  const int p = threadIdx.x;
  for (int e = p; e < l * l; e += blockDim.x) Ts[(e / l) * LP1 + e % l] = (float)T[(e / l) * ldt + e % l];
  const int above = __syncthreads_count(p < l && T[p * ldt + p] > (double)delta);
  if (blockIdx.x == 0 && p == 0) *r_out = above;
  const int64_t j0 = (int64_t)blockIdx.x * 32;
  for (int e = p; e < 32 * l; e += blockDim.x) {
    const int jj = e / l, c = e % l;
    Vs[jj * LP1 + c] = (j0 + jj < n) ? V[(j0 + jj) * ldv + c] : 0.f;
  }
  __syncthreads();
  if (p >= l) return;
  for (int jj = 0; jj < 32 && j0 + jj < n; ++jj) {
    float s = 0.f;
    if (p < above)
      for (int c = 0; c < l; ++c) s = fmaf(Vs[jj * LP1 + c], Ts[p * LP1 + c], s);
    Wt[(j0 + jj) * ldw + p] = s;
  }
}

// One 64 x 64 tile: L = U(:, 0:r) Wt(:, 0:r)^T, then the shrinkage, the multiplier
// update and the residual (Alg. 5 steps 2-4); parts[tile] = sum of squared residuals.
__global__ void __launch_bounds__(256) rpca_update_kernel(const float* __restrict__ M, int64_t ldm,
                                                          float* __restrict__ L, int64_t ldl, float* __restrict__ S,
                                                          int64_t lds, float* __restrict__ Y, int64_t ldy,
                                                          const float* __restrict__ U, int64_t ldu,
                                                          const float* __restrict__ Wt, int64_t ldw,
                                                          const int* __restrict__ r_dev, int64_t m, int64_t n,
                                                          float mu, float inv_mu, float thr,
                                                          double* __restrict__ parts) {
  __shared__ float Us[kRK][kRP], Ws[kRK][kRP];
  __shared__ float red[8];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = (int64_t)blockIdx.y * kRT, j0 = (int64_t)blockIdx.x * kRT;
  const int r = *r_dev;
  float acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
  for (int p0 = 0; p0 < r; p0 += kRK) {
#pragma unroll
    for (int q = 0; q < kRT * kRK / 256; ++q) {
      const int e = tid + 256 * q, rr = e / kRK, pp = e % kRK;
      const bool pk = p0 + pp < r;
      Us[pp][rr] = (pk && i0 + rr < m) ? U[(i0 + rr) * ldu + p0 + pp] : 0.f;
      Ws[pp][rr] = (pk && j0 + rr < n) ? Wt[(j0 + rr) * ldw + p0 + pp] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int pp = 0; pp < kRK; ++pp) {
      float a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = Us[pp][4 * ty + u];
#pragma unroll
      for (int v = 0; v < 4; ++v) b[v] = Ws[pp][4 * tx + v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
  float rs = 0.f;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t i = i0 + 4 * ty + u;
    if (i >= m) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int64_t j = j0 + 4 * tx + v;
      if (j >= n) continue;
      const float lv = acc[u][v], mv = M[i * ldm + j], yv = Y[i * ldy + j];
      const float x = fmaf(yv, inv_mu, mv - lv);
      const float ax = fabsf(x) - thr;
      const float sv = ax > 0.f ? copysignf(ax, x) : 0.f;        // S_thr(x)
      const float res = (mv - lv) - sv;
      L[i * ldl + j] = lv;
      S[i * lds + j] = sv;
      Y[i * ldy + j] = fmaf(mu, res, yv);
      rs = fmaf(res, res, rs);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
  if ((tid & 31) == 0) red[tid >> 5] = rs;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += (double)red[w];
    parts[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

// ordered sum of n doubles (one warp)
__global__ void rpca_sum_kernel(const double* __restrict__ parts, int64_t n, double* __restrict__ out) {
  double s = 0.0;
  for (int64_t e = threadIdx.x; e < n; e += 32) s += parts[e];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) *out = s;
}

}  // namespace
}  // namespace corutv

using namespace corutv;

namespace {

struct RpcaBufs {
  float *U, *V, *Wt;
  double *T, *parts, *scal;   // scal[0] = ||M||_F^2, scal[1] = residual^2
  int32_t* perm;
  int* r;
  int64_t ldu, ldv, ldw;
  int64_t nparts;
};

inline size_t al256(size_t x) { return (x + 255) / 256 * 256; }

int rpca_buffers(corutv_handle* h, int64_t m, int64_t n, int l, RpcaBufs& b) {
  b.ldu = b.ldv = b.ldw = round_up(l, 4);
  b.nparts = cdiv(m, kRT) * cdiv(n, kRT);
  const int64_t fparts = fro2_parts(h->sms);
  const size_t need = al256(sizeof(float) * m * b.ldu) + al256(sizeof(float) * n * b.ldv) +
                      al256(sizeof(float) * n * b.ldw) + al256(sizeof(double) * l * l) +
                      al256(sizeof(double) * std::max<int64_t>(b.nparts, fparts)) + al256(sizeof(double) * 4) +
                      al256(sizeof(int32_t) * l) + al256(sizeof(int) * 4);
  if (!h->rpca_ws || h->rpca_ws_bytes < need) {
    if (h->rpca_ws) {
      cudaStreamSynchronize(h->stream);
      cudaFree(h->rpca_ws);
      h->rpca_ws = nullptr;
      h->rpca_ws_bytes = 0;
    }
    if (cudaMalloc(&h->rpca_ws, need) != cudaSuccess) {
      cudaGetLastError();
      h->rpca_ws = nullptr;
      return CORUTV_ERR_OOM;
    }
    h->rpca_ws_bytes = need;
  }
  char* c = static_cast<char*>(h->rpca_ws);
  auto take = [&](size_t bytes) { char* p = c; c += al256(bytes); return p; };
  b.U = reinterpret_cast<float*>(take(sizeof(float) * m * b.ldu));
  b.V = reinterpret_cast<float*>(take(sizeof(float) * n * b.ldv));
  b.Wt = reinterpret_cast<float*>(take(sizeof(float) * n * b.ldw));
  b.T = reinterpret_cast<double*>(take(sizeof(double) * l * l));
  b.parts = reinterpret_cast<double*>(take(sizeof(double) * std::max<int64_t>(b.nparts, fparts)));
  b.scal = reinterpret_cast<double*>(take(sizeof(double) * 4));
  b.perm = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * l));
  b.r = reinterpret_cast<int*>(take(sizeof(int) * 4));
  return CORUTV_OK;
}

#define RCU(x)                                                                               \
  do {                                                                                       \
    cudaError_t e_ = (x);                                                                    \
    if (e_ != cudaSuccess) {                                                                 \
      fprintf(stderr, "corutv_rpca: %s (%s:%d)\n", cudaGetErrorString(e_), __FILE__, __LINE__); \
      return CORUTV_ERR_CUDA;                                                                \
    }                                                                                        \
  } while (0)

}  // namespace

void rpca_free(corutv_handle* h) {
  if (h && h->rpca_ws) {
    cudaFree(h->rpca_ws);
    h->rpca_ws = nullptr;
    h->rpca_ws_bytes = 0;
  }
}

extern "C" int corutv_rpca(corutv_handle* h, const corutv_rpca_params* p, const float* M, int64_t ldm,
                           const float* Phi, int64_t ldphi, float* L, int64_t ldl, float* S, int64_t lds, float* Y,
                           int64_t ldy, corutv_rpca_info* info) {
  if (!h || !p || !M || !Phi || !L || !S || !Y) return CORUTV_ERR_INVALID_ARG;
  for (int r : p->reserved)
    if (r != 0) return CORUTV_ERR_INVALID_ARG;
  if (p->max_iter < 1 || !(p->mu0 > 0.0) || !(p->rho >= 1.0) || !(p->mu_bar >= p->mu0) || !(p->lambda >= 0.0) ||
      !(p->tol >= 0.0))
    return CORUTV_ERR_INVALID_ARG;
  if (p->mma != CORUTV_MMA_AUTO && p->mma != CORUTV_MMA_SIMT && p->mma != CORUTV_MMA_TF32)
    return CORUTV_ERR_UNSUPPORTED;
  const int64_t m = p->m, n = p->n;
  const int l = p->l;
  if (m <= 0 || n <= 0 || ldm < n || ldl < n || lds < n || ldy < n) return CORUTV_ERR_SHAPE;
  if (cdiv(m, kRT) > 65535) return CORUTV_ERR_SHAPE;
  if ((ldl & 3) || ((uintptr_t)L & 15)) return CORUTV_ERR_ALIGN;   // L's memory is the solve's A
  corutv_params cp{};
  cp.m = m;
  cp.n = n;
  cp.k = p->k;
  cp.l = l;
  cp.q = p->q;
  cp.side = p->side;
  cp.core = CORUTV_CORE_EXACT;
  cp.orth = CORUTV_ORTH_STABILISED;
  cp.a_dtype = CORUTV_F32;
  // AUTO: FP32 products.  The thresholds 1/mu fall geometrically, and the TF32 passes' ~2^-11
  // relative product errors surface as extra diagonals of T above them in the late iterations;
  // TF32 stays available on request.
  cp.mma = p->mma == CORUTV_MMA_TF32 ? CORUTV_MMA_TF32 : CORUTV_MMA_SIMT;
  cp.want_fro2 = 0;
  if (p->k < 1 || p->k > l || l >= std::min(m, n) || l > kMaxL || p->q < 0) return CORUTV_ERR_SHAPE;
  if (p->side != CORUTV_SIDE_RIGHT && p->side != CORUTV_SIDE_LEFT) return CORUTV_ERR_INVALID_ARG;
  if (ldphi < l) return CORUTV_ERR_SHAPE;
  RpcaBufs b{};
  int rc = rpca_buffers(h, m, n, l, b);
  if (rc) return rc;
  cudaStream_t st = h->stream;
  corutv_rpca_info out{};
  const int64_t l0 = launch_counter();
  // S_0 = Y_0 = 0 and ||M||_F
  RCU(cudaMemset2DAsync(S, lds * sizeof(float), 0, n * sizeof(float), m, st));
  RCU(cudaMemset2DAsync(Y, ldy * sizeof(float), 0, n * sizeof(float), m, st));
  RCU(launch_fro2(CORUTV_F32, M, ldm, m, n, nullptr, 0, b.parts, fro2_parts(h->sms), b.scal, st));
  double fro2m = 0.0;
  RCU(cudaMemcpyAsync(&fro2m, b.scal, sizeof(double), cudaMemcpyDeviceToHost, st));
  RCU(cudaStreamSynchronize(st));
  const double normM = sqrt(fro2m);
  double mu = p->mu0;
  out.zeta = INFINITY;
  const unsigned rows_grid = (unsigned)std::min<int64_t>(m, (int64_t)h->sms * 8);
  const size_t rw_smem = sizeof(float) * (size_t)(l + 32) * (l + 1);
  RCU(cudaFuncSetAttribute(rpca_rank_w_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rw_smem));
  const dim3 ugrid((unsigned)cdiv(n, kRT), (unsigned)cdiv(m, kRT));
  for (int it = 1; it <= p->max_iter; ++it) {
    const float inv_mu = (float)(1.0 / mu);
    rpca_form_b_kernel<<<rows_grid, 256, 0, st>>>(M, ldm, S, lds, Y, ldy, L, ldl, m, n, inv_mu);   // step 2: B
    CORUTV_COUNT_LAUNCH();
    RCU(cudaGetLastError());
    rc = corutv_solve(h, &cp, L, ldl, nullptr, Phi, ldphi, b.U, b.ldu, b.T, l, b.V, b.ldv, b.perm);
    if (rc) return rc;
    rpca_rank_w_kernel<<<(unsigned)cdiv(n, 32), 128, rw_smem, st>>>(b.T, l, b.V, b.ldv, n, l, inv_mu, b.Wt, b.ldw,
                                                                     b.r);
    CORUTV_COUNT_LAUNCH();
    RCU(cudaGetLastError());
    rpca_update_kernel<<<ugrid, 256, 0, st>>>(M, ldm, L, ldl, S, lds, Y, ldy, b.U, b.ldu, b.Wt, b.ldw, b.r, m, n,
                                               (float)mu, inv_mu, (float)(p->lambda / mu), b.parts);
    CORUTV_COUNT_LAUNCH();
    RCU(cudaGetLastError());
    rpca_sum_kernel<<<1, 32, 0, st>>>(b.parts, b.nparts, b.scal + 1);
    CORUTV_COUNT_LAUNCH();
    RCU(cudaGetLastError());
    double res2 = 0.0;
    int r = 0;
    RCU(cudaMemcpyAsync(&res2, b.scal + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    RCU(cudaMemcpyAsync(&r, b.r, sizeof(int), cudaMemcpyDeviceToHost, st));
    RCU(cudaStreamSynchronize(st));
    mu = std::min(p->rho * mu, p->mu_bar);                                                       // step 5
    out.iters = it;
    out.rank = r;
    out.mu = mu;
    out.zeta = normM > 0.0 ? sqrt(res2) / normM : 0.0;
    if (out.zeta < p->tol) {
      out.converged = 1;
      break;
    }
  }
  corutv_info si{};
  rc = corutv_info_wait(h, &si);
  out.status = rc ? rc : si.status;
  h->launches += launch_counter() - l0;
  if (info) *info = out;
  return CORUTV_OK;
}
