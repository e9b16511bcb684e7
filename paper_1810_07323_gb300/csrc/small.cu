// The l x l and tall-skinny steps of CoR-UTV (Sec. III):
//   - Gram / cross products X Y^T of skinny blocks (FP32 partials per CTA,
//     ordered FP64 reduction): C^T C for CholeskyQR and Q1^T (A Q2) for the core;
//   - one-CTA Cholesky of the (shifted) Gram matrix with the inverse of its
//     factor built alongside, and breakdown detection (dependent columns);
//   - Q = C R^-1 and U = Q1 Q~ as a small-times-skinny product;
//   - one-CTA Householder QRCP of the core (Eq. (D = Q~ R~ P~^T));
//   - staging of Psi, the V = Q2 P~ gather, and ||A||_F^2.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "elem.cuh"
#include "internal.h"

namespace corutv {

constexpr int kCholTPR = 8;   // threads per row of the register Cholesky (1024 threads)
constexpr int kQrcpTPC = 4;   // threads per column of the register QRCP (512 threads)

// =============================================================================== Gram
// parts[c] = X[:, cols_c] Y[:, cols_c]^T over the c-th contiguous column range.
// 512 threads, thread (tx, ty) (32 x 16) owns rows a = R ty + (0..R-1) and
// columns b = C tx + (0..C-1) (R = LP/16, C = LP/32).  Stages of BK columns
// are kept k-major in shared memory (rows padded by 4); the next stage's
// global loads are issued into registers before the current stage is used.
template <typename TC, int LP>
__global__ void __launch_bounds__(512) gram_partial_kernel(const TC* __restrict__ Xt, int64_t ldx,
                                                           const TC* __restrict__ Yt, int64_t ldy, int64_t len,
                                                           int l, TC* __restrict__ parts) {
  constexpr int R = LP / 16, CC = LP / 32;
  constexpr int BK = 32;
  constexpr int LPP = LP + 4;
  constexpr int PER = LP * BK / 512;        // elements of X (and of Y) staged per thread
  __shared__ __align__(16) TC Xs[BK][LPP];
  __shared__ __align__(16) TC Ys[BK][LPP];
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int64_t chunk = cdiv(cdiv(len, BK), gridDim.x) * BK;
  const int64_t c0 = blockIdx.x * chunk;
  int64_t c1 = c0 + chunk;
  if (c1 > len) c1 = len;
  TC acc[R][CC];
#pragma unroll
  for (int v = 0; v < R; ++v)
#pragma unroll
    for (int u = 0; u < CC; ++u) acc[v][u] = TC(0);
  TC px[PER], py[PER];
  auto fetch = [&](int64_t k0) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int x = tid + 512 * q;
      const int r = x / BK, kk = x % BK;
      const int64_t g = k0 + kk;
      const bool ok = r < l && g < c1;
      px[q] = ok ? Xt[r * ldx + g] : TC(0);
      py[q] = ok ? Yt[r * ldy + g] : TC(0);
    }
  };
  if (c0 < c1) fetch(c0);
  for (int64_t k0 = c0; k0 < c1; k0 += BK) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int x = tid + 512 * q;
      const int r = x / BK, kk = x % BK;
      Xs[kk][r] = px[q];
      Ys[kk][r] = py[q];
    }
    __syncthreads();
    if (k0 + BK < c1) fetch(k0 + BK);
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      TC xa[R], yb[CC];
#pragma unroll
      for (int v = 0; v < R; ++v) xa[v] = Xs[kk][R * ty + v];
#pragma unroll
      for (int u = 0; u < CC; ++u) yb[u] = Ys[kk][CC * tx + u];
#pragma unroll
      for (int v = 0; v < R; ++v)
#pragma unroll
        for (int u = 0; u < CC; ++u) acc[v][u] = fma(xa[v], yb[u], acc[v][u]);
    }
    __syncthreads();
  }
  TC* out = parts + (int64_t)blockIdx.x * LP * LP;
#pragma unroll
  for (int v = 0; v < R; ++v)
#pragma unroll
    for (int u = 0; u < CC; ++u) out[(R * ty + v) * LP + CC * tx + u] = acc[v][u];
}

// G[a][b] = sum over parts in a fixed order, in FP64: four threads per element
// each sum every fourth part, then (s0 + s1) + (s2 + s3).
template <typename TC>
__global__ void gram_reduce_kernel(const TC* __restrict__ parts, int nparts, int LP, int l, double* __restrict__ G,
                                   int64_t ldg) {
  const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 2;
  const int q = threadIdx.x & 3;
  const bool ok = e < l * l;
  const int a = ok ? e / l : 0, b = ok ? e % l : 0;
  double s = 0.0;
  if (ok) {
    const TC* src = parts + (int64_t)a * LP + b;
    const int64_t stride = (int64_t)LP * LP;
    int p = q;
    for (; p + 12 < nparts; p += 16) {
      const double v0 = (double)src[p * stride], v1 = (double)src[(p + 4) * stride];
      const double v2 = (double)src[(p + 8) * stride], v3 = (double)src[(p + 12) * stride];
      s += v0; s += v1; s += v2; s += v3;
    }
    for (; p < nparts; p += 4) s += (double)src[p * stride];
  }
  const double s1 = __shfl_xor_sync(0xffffffffu, s, 1);
  const double t = (q & 1) ? s1 + s : s + s1;                 // (s0 + s1), (s2 + s3)
  const double t2 = __shfl_xor_sync(0xffffffffu, t, 2);
  if (ok && q == 0) G[a * ldg + b] = t + t2;
}

int gram_parts(int64_t len, int sms) {
  int64_t p = cdiv(len, 32);
  if (p > sms) p = sms;
  return (int)(p < 1 ? 1 : p);
}

template <typename TC>
cudaError_t launch_gram(const TC* Xt, int64_t ldx, const TC* Yt, int64_t ldy, int64_t len, int l, TC* parts,
                        int gparts, double* G, int64_t ldg, cudaStream_t st) {
  int LP;
  if (l <= 32) {
    LP = 32;
    gram_partial_kernel<TC, 32><<<gparts, 512, 0, st>>>(Xt, ldx, Yt, ldy, len, l, parts); CORUTV_COUNT_LAUNCH();
  } else if (l <= 64) {
    LP = 64;
    gram_partial_kernel<TC, 64><<<gparts, 512, 0, st>>>(Xt, ldx, Yt, ldy, len, l, parts); CORUTV_COUNT_LAUNCH();
  } else {
    LP = 128;
    gram_partial_kernel<TC, 128><<<gparts, 512, 0, st>>>(Xt, ldx, Yt, ldy, len, l, parts); CORUTV_COUNT_LAUNCH();
  }
  gram_reduce_kernel<TC><<<(unsigned)cdiv((int64_t)l * l * 4, 256), 256, 0, st>>>(parts, gparts, LP, l, G, ldg); CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

// =============================================================================== Cholesky
// G + s I = R^T R (R upper, s = shift_rel * trace(G)) and R^-1, by symmetric
// elimination of [G | I]: step j subtracts m_a = G[j][a] / G[j][j] times row j
// from every row a > j (upper triangle of G only, by symmetry; the right block
// receives the same row operations).  Afterwards G = L D L^T with the pivots
// d_j = G[j][j] (as of step j), the upper triangle holding D L^T and the right
// block holding L^-1, so R = D^(1/2) L^T and R^-1[p][j] = L^-1[j][p] / sqrt(d_j).
// Every update of a step is independent: one block barrier per step, no long
// dependent chains.  A pivot d <= tol_rel * (G_jj + s) marks column j
// dependent: it eliminates nothing, R[j][j] = 1, R[j][>j] = 0, defic[j] = 1
// (the caller replaces that column of Q).
template <typename TC>
__global__ void __launch_bounds__(512) cholinv_kernel(const double* __restrict__ G, int64_t ldg, int l,
                                                      double shift_rel, double tol_rel, TC* __restrict__ Rg,
                                                      TC* __restrict__ Rinvg, int* __restrict__ defic,
                                                      DevStatus* status, double* __restrict__ Rout) {
  extern __shared__ unsigned char smem_raw[];
  const int LD = l + 1;
  TC* Gs = reinterpret_cast<TC*>(smem_raw);     // l x LD, upper triangle used
  TC* Li = Gs + l * LD;                          // l x LD, L^-1 (lower, unit diagonal)
  __shared__ double diag0[kMaxL];
  __shared__ TC piv[kMaxL];
  __shared__ int dep_s[kMaxL];
  __shared__ double red[32];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;

  double tr = 0.0;
  for (int e = tid; e < l * l; e += nt) {
    const int a = e / l, b = e % l;
    const double g = G[a * ldg + b];
    if (b >= a) Gs[a * LD + b] = (TC)g;
    Li[a * LD + b] = (a == b) ? TC(1) : TC(0);
    if (a == b) tr += g;
  }
  for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
  if (lane == 0) red[warp] = tr;
  __syncthreads();
  double trace = 0.0;
  for (int w = 0; w < nw; ++w) trace += red[w];
  const double shift = shift_rel * trace;
  for (int a = tid; a < l; a += nt) {
    const double d = (double)Gs[a * LD + a] + shift;
    Gs[a * LD + a] = (TC)d;
    diag0[a] = d;
  }
  __syncthreads();

  for (int j = 0; j < l; ++j) {
    const TC d = Gs[j * LD + j];
    const bool dep = !((double)d > tol_rel * diag0[j]) || !(diag0[j] > 0.0);
    const TC inv_d = dep ? TC(0) : TC(1) / d;
    if (tid == 0) {
      piv[j] = dep ? TC(1) : d;
      dep_s[j] = dep ? 1 : 0;
    }
    // rows a > j, one warp per row: upper triangle b >= a of G, and L^-1 columns b <= j
    for (int a = j + 1 + warp; a < l; a += nw) {
      const TC m = Gs[j * LD + a] * inv_d;
      for (int b = a + lane; b < l; b += 32) Gs[a * LD + b] -= m * Gs[j * LD + b];
      for (int b = lane; b <= j; b += 32) Li[a * LD + b] -= m * Li[j * LD + b];
    }
    __syncthreads();
  }
  int nfall = 0;
  for (int e = tid; e < l * l; e += nt) {
    const int a = e / l, b = e % l;
    const TC ra = sqrt(piv[a]);
    TC r = TC(0);
    if (b == a) r = ra;
    else if (b > a && !dep_s[a]) r = Gs[a * LD + b] / ra;
    Rg[a * kMaxL + b] = r;
    // R^-1[a][b] = L^-1[b][a] / sqrt(d_b)  (upper: a <= b)
    Rinvg[a * kMaxL + b] = (b >= a) ? Li[b * LD + a] / sqrt(piv[b]) : TC(0);
    if (Rout) Rout[a * l + b] = (double)r;
  }
  for (int a = tid; a < l; a += nt) {
    defic[a] = dep_s[a];
    nfall += dep_s[a];
  }
  for (int o = 16; o > 0; o >>= 1) nfall += __shfl_xor_sync(0xffffffffu, nfall, o);
  if (lane == 0 && nfall && status) atomicAdd(&status->chol_fallbacks, nfall);
}

// FP32 variant with rows in registers: thread (a, h) holds columns
// b = 64 h .. 64 h + 63 of row a of both blocks.  Step j: the two threads of
// row j publish it (double-buffered, one barrier per step) with the entries
// that must not act zeroed -- G part only for b > j, L^-1 part only for b <= j
// -- so every row a > j subtracts m_a = G[j][a] / d_j times it with
// unpredicated vector loads.  Same algebra as cholinv_kernel.
template <int TPR>
__global__ void __launch_bounds__(kMaxL * TPR) cholinv_reg_kernel(const double* __restrict__ G, int64_t ldg, int l,
                                                          double shift_rel, double tol_rel, float* __restrict__ Rg,
                                                          float* __restrict__ Rinvg, int* __restrict__ defic,
                                                          DevStatus* status, double* __restrict__ Rout) {
  constexpr int CPT = kMaxL / TPR, NWARP = kMaxL * TPR / 32;
  __shared__ __align__(16) float prow[2][kMaxL];
  __shared__ __align__(16) float plrow[2][kMaxL];
  __shared__ float pivm[2];             // [buf]: 1 / d_j (0 if dependent)
  __shared__ double red[NWARP];
  const int tid = threadIdx.x, a = tid / TPR, h = tid % TPR, lane = tid & 31, warp = tid >> 5;
  const int b0 = h * CPT;
  const unsigned grp = ((TPR == 32) ? 0xffffffffu : ((1u << TPR) - 1u)) << (lane & ~(TPR - 1));
  float g[CPT], li[CPT];
  double tr = 0.0;
#pragma unroll
  for (int s = 0; s < CPT; ++s) {
    const int b = b0 + s;
    const bool ok = a < l && b < l;
    const double v = ok ? G[a * ldg + b] : 0.0;
    g[s] = (float)v;
    li[s] = (ok && a == b) ? 1.f : 0.f;
    if (ok && a == b) tr += v;
  }
  for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
  if (lane == 0) red[warp] = tr;
  __syncthreads();
  double trace = 0.0;
  for (int w = 0; w < NWARP; ++w) trace += red[w];
  const double shift = shift_rel * trace;
  double diag0 = 0.0;
#pragma unroll
  for (int s = 0; s < CPT; ++s)
    if (b0 + s == a && a < l) {
      diag0 = (double)g[s] + shift;
      g[s] = (float)diag0;
    }
#pragma unroll
  for (int o = 1; o < TPR; o <<= 1) diag0 = fmax(diag0, __shfl_xor_sync(0xffffffffu, diag0, o));
  float piv_mine = 1.f;
  bool dep_mine = false;
  for (int j = 0; j < l; ++j) {
    const int buf = j & 1;
    if (a == j) {
      float dj = 0.f;
#pragma unroll
      for (int s = 0; s < CPT; ++s)
        if (b0 + s == j) dj = g[s];
#pragma unroll
      for (int o = 1; o < TPR; o <<= 1) dj += __shfl_xor_sync(grp, dj, o);
      const bool dep = !((double)dj > tol_rel * diag0) || !(diag0 > 0.0);
      piv_mine = dep ? 1.f : dj;
      dep_mine = dep;
      float4* pr = reinterpret_cast<float4*>(&prow[buf][b0]);
      float4* pl = reinterpret_cast<float4*>(&plrow[buf][b0]);
#pragma unroll
      for (int q = 0; q < CPT / 4; ++q) {
        float4 vg, vl;
        float* pg = &vg.x;
        float* plv = &vl.x;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int s = 4 * q + e, b = b0 + s;
          pg[e] = (b > j) ? g[s] : 0.f;
          plv[e] = (b <= j) ? li[s] : 0.f;
        }
        pr[q] = vg;
        pl[q] = vl;
      }
      if (h == 0) pivm[buf] = dep ? 0.f : 1.f / dj;
    }
    __syncthreads();
    if (a > j && a < l) {
      const float m = prow[buf][a] * pivm[buf];
      const float4* pr = reinterpret_cast<const float4*>(&prow[buf][b0]);
      const float4* pl = reinterpret_cast<const float4*>(&plrow[buf][b0]);
#pragma unroll
      for (int q = 0; q < CPT / 4; ++q) {
        const float4 vg = pr[q], vl = pl[q];
        g[4 * q + 0] -= m * vg.x; g[4 * q + 1] -= m * vg.y; g[4 * q + 2] -= m * vg.z; g[4 * q + 3] -= m * vg.w;
        li[4 * q + 0] -= m * vl.x; li[4 * q + 1] -= m * vl.y; li[4 * q + 2] -= m * vl.z; li[4 * q + 3] -= m * vl.w;
      }
    }
  }
  __syncthreads();
  if (a < l) {
    const float ra = sqrtf(piv_mine);
#pragma unroll
    for (int s = 0; s < CPT; ++s) {
      const int b = b0 + s;
      if (b >= l) continue;
      float r = 0.f;
      if (b == a) r = ra;
      else if (b > a && !dep_mine) r = g[s] / ra;
      Rg[a * kMaxL + b] = r;
      if (Rout) Rout[a * l + b] = (double)r;
      // R^-1[b][a] = L^-1[a][b] / sqrt(d_a) for b <= a
      Rinvg[b * kMaxL + a] = (b <= a) ? li[s] / ra : 0.f;
    }
  }
  int nfall = (h == 0 && a < l && dep_mine) ? 1 : 0;
  for (int o = 16; o > 0; o >>= 1) nfall += __shfl_xor_sync(0xffffffffu, nfall, o);
  if (h == 0 && a < l) defic[a] = dep_mine ? 1 : 0;
  if (lane == 0 && nfall && status) atomicAdd(&status->chol_fallbacks, nfall);
}

// C (M x N) = op(A) B over K in shared memory, 4 x 4 register tiles spread
// over the block's threads.  op(A)[r][k] = A[k][r] (TRANS_A) or A[r][k].
// MODE 0: C = result, 1: C -= result, 2: C = -result.  upper_only skips
// tiles strictly below the diagonal.  M, N multiples of 4; rows 16-byte aligned.
template <bool TRANS_A, int MODE>
__device__ __forceinline__ void smem_gemm44(const float* __restrict__ Ap, int lda, const float* __restrict__ Bp,
                                            int ldb, float* __restrict__ Cp, int ldc, int M, int N, int K,
                                            bool upper_only) {
  const int tn = N >> 2, tiles = (M >> 2) * tn;
  for (int t = threadIdx.x; t < tiles; t += blockDim.x) {
    const int r0 = (t / tn) << 2, c0 = (t % tn) << 2;
    if (upper_only && c0 + 3 < r0) continue;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
      float a[4];
      if (TRANS_A) {
        const float4 v = *reinterpret_cast<const float4*>(Ap + k * lda + r0);
        a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w;
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = Ap[(r0 + i) * lda + k];
      }
      const float4 b = *reinterpret_cast<const float4*>(Bp + k * ldb + c0);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        acc[i][0] = fmaf(a[i], b.x, acc[i][0]);
        acc[i][1] = fmaf(a[i], b.y, acc[i][1]);
        acc[i][2] = fmaf(a[i], b.z, acc[i][2]);
        acc[i][3] = fmaf(a[i], b.w, acc[i][3]);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float4* c4 = reinterpret_cast<float4*>(Cp + (r0 + i) * ldc + c0);
      float4 v;
      if (MODE == 1) {
        v = *c4;
        v.x -= acc[i][0]; v.y -= acc[i][1]; v.z -= acc[i][2]; v.w -= acc[i][3];
      } else if (MODE == 2) {
        v = make_float4(-acc[i][0], -acc[i][1], -acc[i][2], -acc[i][3]);
      } else {
        v = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      }
      *c4 = v;
    }
  }
}

// FP32 blocked variant (l <= 128, padded with an identity block to 128 = 4
// blocks of 32).  For each diagonal block o = 32 kb:
//   1. one warp factors the 32 x 32 block by the same symmetric elimination
//      (lane i holds column i of the block and of its L^-1 block; multipliers
//      are broadcast with shuffles, no block barrier) and writes R11, R11^-1;
//   2. panel: R12 = R11^-T A12 (rows of dependent columns zeroed);
//   3. trailing update A22 -= R12^T R12.
// Then R^-1 is completed block column by block column:
//   X_kk = R_kk^-1,  X_ik = -(sum_{p=i}^{k-1} X_ip R_pk) X_kk.
// About twenty block barriers in all; the same algebra and dependent-column
// rule as cholinv_kernel.
__global__ void __launch_bounds__(512) cholinv_blk_kernel(const double* __restrict__ G, int64_t ldg, int l,
                                                          double shift_rel, double tol_rel, float* __restrict__ Rg,
                                                          float* __restrict__ Rinvg, int* __restrict__ defic,
                                                          DevStatus* status, double* __restrict__ Rout) {
  constexpr int N = kMaxL, NB = 32, LD = N + 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* A = reinterpret_cast<float*>(smem_raw);      // N x LD: G, becomes R (upper)
  float* X = A + N * LD;                             // N x LD: R^-1 (upper)
  float* T = X + N * LD;                             // NB x LD scratch (panel / products)
  __shared__ float diag0[N];
  __shared__ int dep[N];
  __shared__ double red[16];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;

  // 32 independent loads per thread, issued before any use (no accumulation in the loop)
  {
    float v[N * N / 512];
#pragma unroll
    for (int q = 0; q < N * N / 512; ++q) {
      const int e = tid + 512 * q, a = e >> 7, b = e & (N - 1);
      v[q] = (a < l && b < l) ? (float)G[a * ldg + b] : ((a == b) ? 1.f : 0.f);
    }
#pragma unroll
    for (int q = 0; q < N * N / 512; ++q) {
      const int e = tid + 512 * q, a = e >> 7, b = e & (N - 1);
      A[a * LD + b] = v[q];
      X[a * LD + b] = 0.f;
    }
  }
  __syncthreads();
  double tr = (tid < l) ? (double)A[tid * LD + tid] : 0.0;
  for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
  if (lane == 0) red[warp] = tr;
  __syncthreads();
  double trace = 0.0;
  for (int w = 0; w < nt / 32; ++w) trace += red[w];
  const float shift = (float)(shift_rel * trace);
  const float tolf = (float)tol_rel;
  for (int a = tid; a < N; a += nt) {
    if (a < l) A[a * LD + a] += shift;
    diag0[a] = A[a * LD + a];
  }
  __syncthreads();

  for (int kb = 0; kb < N / NB; ++kb) {
    const int o = NB * kb, rest = N - o - NB;
    // ---- 1. diagonal block by one warp
    if (warp == 0) {
      float a[NB], w[NB];     // column `lane` of the block and of its L^-1
#pragma unroll
      for (int r = 0; r < NB; ++r) {
        a[r] = A[(o + r) * LD + o + lane];
        w[r] = (r == lane) ? 1.f : 0.f;
      }
      const float dg0 = diag0[o + lane];
      float* prow = T;        // staging of the multipliers of step j (T is free here)
      float dv = 1.f;          // pivot of row `lane`
      bool dp = false;
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        // lane j owns the pivot: publish m_k = A[j][k] / d for every k (A[j][k] = lane k's a[j])
        const float d = __shfl_sync(0xffffffffu, a[j], j);
        const float d0 = __shfl_sync(0xffffffffu, dg0, j);
        const bool depj = !(d > tolf * d0) || !(d0 > 0.f);
        const float inv_d = depj ? 0.f : __frcp_rn(d);
        if (lane == j) { dv = depj ? 1.f : d; dp = depj; }
        prow[lane] = a[j] * inv_d;            // m_lane (used for k > j)
        __syncwarp();
        const float rowj_a = a[j];            // A[j][lane]
        const float rowj_w = w[j];            // L^-1[j][lane]
#pragma unroll
        for (int k = j + 1; k < NB; ++k) {
          const float m = prow[k];
          a[k] = fmaf(-m, rowj_a, a[k]);
          w[k] = fmaf(-m, rowj_w, w[k]);
        }
        __syncwarp();
      }
      // lane holds column `lane` of U = D L^T and of L^-1; its pivot is dv
      const float sq = sqrtf(dv);
      const float rsq = 1.f / sq;
      dep[o + lane] = dp ? 1 : 0;
      // R11[k][lane] = U[k][lane] / sqrt(d_k) for k <= lane (0 above for dependent rows)
#pragma unroll
      for (int k = 0; k < NB; ++k) {
        const float rk = __shfl_sync(0xffffffffu, rsq, k);     // 1 / sqrt(d_k)
        const int depk = __shfl_sync(0xffffffffu, dp ? 1 : 0, k);
        float r = 0.f;
        if (k == lane) r = sq;
        else if (k < lane && !depk) r = a[k] * rk;
        A[(o + k) * LD + o + lane] = r;
        // R11^-1[lane][k] = L^-1[k][lane] / sqrt(d_k), k >= lane
        X[(o + lane) * LD + o + k] = (k >= lane) ? w[k] * rk : 0.f;
      }
    }
    __syncthreads();
    if (rest > 0) {
      const int c0 = o + NB;
      // ---- 2. panel R12 = R11^-T A12 (R11^-1 upper, zero below) into T, rows of dependent columns zeroed
      smem_gemm44<true, 0>(X + o * LD + o, LD, A + o * LD + c0, LD, T + c0, LD, NB, rest, NB, false);
      __syncthreads();
      for (int e = threadIdx.x; e < NB * rest; e += blockDim.x) {
        const int k = e / rest, c = c0 + e % rest;
        if (dep[o + k]) T[k * LD + c] = 0.f;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < NB * rest; e += blockDim.x) {
        const int k = e / rest, c = c0 + e % rest;
        A[(o + k) * LD + c] = T[k * LD + c];
      }
      // ---- 3. trailing update (upper tiles): A22 -= R12^T R12
      smem_gemm44<true, 1>(T + c0, LD, T + c0, LD, A + c0 * LD + c0, LD, rest, rest, NB, true);
      __syncthreads();
    }
  }
  // ---- R^-1 off-diagonal blocks: X_ik = -(sum_{p=i}^{k-1} X_ip R_pk) X_kk.
  // For block column k (columns ok .. ok+31) and every row r < ok:
  //   S[r][c] = sum_{p=r}^{ok-1} X[r][p] R[p][c]   (kept in X's own (r, c) slots),
  //   X[r][c] = -sum_{q=ok}^{c} S[r][q] X[q][c]    (staged in A's unused lower triangle).
  for (int kb = 1; kb < N / NB; ++kb) {
    const int ok = NB * kb;
    // S = X[0:ok, 0:ok] R[0:ok, ok:ok+NB] into T-sized staging (rows of X are zero left of the diagonal)
    // staged in X's own (r, ok..ok+NB) slots, which are still zero and not read here
    smem_gemm44<false, 0>(X, LD, A + ok, LD, X + ok, LD, ok, NB, ok, false);
    __syncthreads();
    // X[r, ok:ok+NB] = -S[r, :] X_kk, one row per thread (read the row, then overwrite it)
    for (int r = tid; r < ok; r += nt) {
      float sv[NB], out[NB];
#pragma unroll
      for (int q = 0; q < NB; q += 4) {
        const float4 v = *reinterpret_cast<const float4*>(X + r * LD + ok + q);
        sv[q] = v.x; sv[q + 1] = v.y; sv[q + 2] = v.z; sv[q + 3] = v.w;
      }
#pragma unroll
      for (int c = 0; c < NB; ++c) out[c] = 0.f;
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        const float* xk = X + (ok + q) * LD + ok;
#pragma unroll
        for (int c = 0; c < NB; c += 4) {
          const float4 v = *reinterpret_cast<const float4*>(xk + c);
          out[c] = fmaf(sv[q], v.x, out[c]);
          out[c + 1] = fmaf(sv[q], v.y, out[c + 1]);
          out[c + 2] = fmaf(sv[q], v.z, out[c + 2]);
          out[c + 3] = fmaf(sv[q], v.w, out[c + 3]);
        }
      }
#pragma unroll
      for (int c = 0; c < NB; c += 4)
        *reinterpret_cast<float4*>(X + r * LD + ok + c) = make_float4(-out[c], -out[c + 1], -out[c + 2], -out[c + 3]);
    }
    __syncthreads();
  }
  // ---- outputs
  int nfall = 0;
  for (int e = tid; e < l * l; e += nt) {
    const int a = e / l, b = e % l;
    const float r = (b >= a) ? A[a * LD + b] : 0.f;
    Rg[a * kMaxL + b] = r;
    Rinvg[a * kMaxL + b] = (b >= a) ? X[a * LD + b] : 0.f;
    if (Rout) Rout[a * l + b] = (double)r;
  }
  for (int a = tid; a < l; a += nt) {
    defic[a] = dep[a];
    nfall += dep[a];
  }
  for (int o2 = 16; o2 > 0; o2 >>= 1) nfall += __shfl_xor_sync(0xffffffffu, nfall, o2);
  if (lane == 0 && nfall && status) atomicAdd(&status->chol_fallbacks, nfall);
}

template <typename TC>
cudaError_t launch_cholinv(const double* G, int64_t ldg, int l, double shift_rel, double tol_rel, TC* R, TC* Rinv,
                           int* defic, DevStatus* status, double* Rout, cudaStream_t st) {
  if constexpr (sizeof(TC) == 4) {
    const size_t smem_blk = (size_t)(2 * kMaxL + 32) * (kMaxL + 4) * sizeof(float);
    cudaError_t e0 = cudaFuncSetAttribute(cholinv_blk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem_blk);
    if (e0 != cudaSuccess) return e0;
    cholinv_blk_kernel<<<1, 512, smem_blk, st>>>(G, ldg, l, shift_rel, tol_rel, R, Rinv, defic, status, Rout);
    CORUTV_COUNT_LAUNCH();
    return cudaGetLastError();
  }
  const size_t smem = (size_t)2 * l * (l + 1) * sizeof(TC);
  cudaError_t e = cudaFuncSetAttribute(cholinv_kernel<TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cholinv_kernel<TC><<<1, 512, smem, st>>>(G, ldg, l, shift_rel, tol_rel, R, Rinv, defic, status, Rout); CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

// =============================================================================== lmul
// Out[j][i] = sum_{p<l} S[p][j] In[p][i]   (Out = S^T In on ST blocks, i.e. C S in
// the untransposed view).  A CTA computes a BI-column tile; thread (tx, ty)
// owns j = R ty + (0..R-1) and i = BI/16 tx + (0..BI/16-1).  upper: S is upper
// triangular (S[p][j] = 0 for p > j), so the p loop stops at the thread's last j.
// out_rowmajor: write Out^T into a row-major len x l matrix (staged through
// shared memory so the row writes coalesce).
template <typename TC, typename TS, int LP, int BI>
__global__ void __launch_bounds__(256) lmul_kernel(const TC* __restrict__ In, int64_t ldi, int64_t len, int l,
                                                   const TS* __restrict__ S, int64_t lds, TC* __restrict__ Out,
                                                   int64_t ldo, int out_rowmajor, int upper) {
  constexpr int R = LP / 16, RI = BI / 16;
  constexpr int SP = LP + 4, IP = BI + 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC* Ss = reinterpret_cast<TC*>(smem_raw);      // LP x SP   (row p, column j)
  TC* Is = Ss + LP * SP;                         // LP x IP   (row p, column i)
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = (int64_t)blockIdx.x * BI;
  for (int e = tid; e < LP * LP; e += 256) {
    const int p = e / LP, j = e % LP;
    Ss[p * SP + j] = (p < l && j < l) ? (TC)S[p * lds + j] : TC(0);
  }
  // (S rows p >= l and columns j >= l are zero: the p loop below can stop at l)
  for (int e = tid; e < LP * BI; e += 256) {
    const int p = e / BI, ii = e % BI;
    const int64_t g = i0 + ii;
    Is[p * IP + ii] = (p < l && g < len) ? In[p * ldi + g] : TC(0);
  }
  __syncthreads();
  TC acc[R][RI];
#pragma unroll
  for (int v = 0; v < R; ++v)
#pragma unroll
    for (int u = 0; u < RI; ++u) acc[v][u] = TC(0);
  int pend = l;
  if (upper) {
    // the warp's rows: ty and ty ^ 1 (both halves of the warp); the larger bounds the loop
    const int jmax = R * ((ty | 1) + 1);
    pend = jmax < l ? jmax : l;
  }
#pragma unroll 2
  for (int p = 0; p < pend; ++p) {
    TC sv[R], xv[RI];
#pragma unroll
    for (int v = 0; v < R; ++v) sv[v] = Ss[p * SP + R * ty + v];
#pragma unroll
    for (int u = 0; u < RI; ++u) xv[u] = Is[p * IP + RI * tx + u];
#pragma unroll
    for (int v = 0; v < R; ++v)
#pragma unroll
      for (int u = 0; u < RI; ++u) acc[v][u] = fma(sv[v], xv[u], acc[v][u]);
  }
  if (!out_rowmajor) {
#pragma unroll
    for (int v = 0; v < R; ++v) {
      const int j = R * ty + v;
      if (j >= l) continue;
#pragma unroll
      for (int u = 0; u < RI; ++u) {
        const int64_t g = i0 + RI * tx + u;
        if (g < len) Out[j * ldo + g] = acc[v][u];
      }
    }
  } else {
    __syncthreads();
    TC* Os = Is;                                  // BI x (LP + 1)
#pragma unroll
    for (int v = 0; v < R; ++v)
#pragma unroll
      for (int u = 0; u < RI; ++u) Os[(RI * tx + u) * (LP + 1) + R * ty + v] = acc[v][u];
    __syncthreads();
    for (int e = tid; e < BI * l; e += 256) {
      const int ii = e / l, j = e % l;
      const int64_t g = i0 + ii;
      if (g < len) Out[g * ldo + j] = Os[ii * (LP + 1) + j];
    }
  }
}

template <typename TC, typename TS, int LP, int BI>
static cudaError_t lmul_variant(const TC* In, int64_t ldi, int64_t len, int l, const TS* S, int64_t lds, TC* Out,
                                int64_t ldo, bool rowmajor, bool upper, cudaStream_t st) {
  const unsigned grid = (unsigned)cdiv(len, BI);
  if (grid == 0) return cudaSuccess;
  const size_t a = (size_t)LP * (LP + 4) + (size_t)LP * (BI + 4);
  const size_t b = (size_t)LP * (LP + 4) + (size_t)BI * (LP + 1);
  const size_t sm = (a > b ? a : b) * sizeof(TC);
  cudaError_t e = cudaFuncSetAttribute(lmul_kernel<TC, TS, LP, BI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  lmul_kernel<TC, TS, LP, BI><<<grid, 256, sm, st>>>(In, ldi, len, l, S, lds, Out, ldo, rowmajor ? 1 : 0,
                                                     upper ? 1 : 0);
  CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

template <typename TC, typename TS>
static cudaError_t lmul_dispatch(const TC* In, int64_t ldi, int64_t len, int l, const TS* S, int64_t lds, TC* Out,
                                 int64_t ldo, bool rowmajor, bool upper, cudaStream_t st) {
  constexpr int BI = 64;
  if (l <= 32) return lmul_variant<TC, TS, 32, BI>(In, ldi, len, l, S, lds, Out, ldo, rowmajor, upper, st);
  if (l <= 64) return lmul_variant<TC, TS, 64, BI>(In, ldi, len, l, S, lds, Out, ldo, rowmajor, upper, st);
  return lmul_variant<TC, TS, 128, BI>(In, ldi, len, l, S, lds, Out, ldo, rowmajor, upper, st);
}

template <typename TC>
cudaError_t launch_lmul(const TC* In, int64_t ldi, int64_t len, int l, const TC* S, int64_t lds, TC* Out,
                        int64_t ldo, bool out_rowmajor, cudaStream_t st) {
  // the CholeskyQR factor R^-1 is upper triangular
  return lmul_dispatch<TC, TC>(In, ldi, len, l, S, lds, Out, ldo, out_rowmajor, true, st);
}
template <typename TC>
cudaError_t launch_lmul_f64s(const TC* In, int64_t ldi, int64_t len, int l, const double* S, int64_t lds, TC* Out,
                             int64_t ldo, bool out_rowmajor, cudaStream_t st) {
  return lmul_dispatch<TC, double>(In, ldi, len, l, S, lds, Out, ldo, out_rowmajor, false, st);
}

// =============================================================================== deficient columns
// Replace row j of an ST block (column j of Q) flagged dependent by a
// deterministic pseudo-random vector (SplitMix64 of (pass, j, i), uniform in
// [-1, 1)); the next CholeskyQR pass orthonormalises it against the others.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename TC>
__global__ void fill_deficient_kernel(TC* __restrict__ Ct, int64_t ldc, int64_t len, int l,
                                      const int* __restrict__ defic, int pass) {
  const int j = blockIdx.y;
  if (j >= l || !defic[j]) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t h = mix64(0x5EEDull + ((uint64_t)pass << 48) + ((uint64_t)j << 32) + (uint64_t)i * 0x9E3779B97F4A7C15ull);
    const double u = (double)(h >> 11) * (1.0 / 9007199254740992.0);
    Ct[j * ldc + i] = (TC)(2.0 * u - 1.0);
  }
}

template <typename TC>
cudaError_t launch_fill_deficient(TC* Ct, int64_t ldc, int64_t len, int l, const int* defic, int pass,
                                  cudaStream_t st) {
  dim3 grid(32, l);
  fill_deficient_kernel<TC><<<grid, 256, 0, st>>>(Ct, ldc, len, l, defic, pass); CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

// =============================================================================== gather / stage
// Out[i][j] = St[perm[j]][i]  (row-major len x l output from an ST block).
template <typename TC>
__global__ void gather_cols_kernel(const TC* __restrict__ St, int64_t lds, int64_t len, int l,
                                   const int32_t* __restrict__ perm, TC* __restrict__ Out, int64_t ldo) {
  __shared__ TC tile[kMaxL][33];
  __shared__ int pm[kMaxL];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  for (int j = threadIdx.x; j < l; j += blockDim.x) pm[j] = perm ? perm[j] : j;
  for (int e = threadIdx.x; e < l * 32; e += blockDim.x) {
    const int r = e / 32, ii = e % 32;
    const int64_t g = i0 + ii;
    tile[r][ii] = g < len ? St[r * lds + g] : TC(0);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * l; e += blockDim.x) {
    const int ii = e / l, j = e % l;
    const int64_t g = i0 + ii;
    if (g < len) Out[g * ldo + j] = tile[pm[j]][ii];
  }
}

template <typename TC>
cudaError_t launch_gather_cols(const TC* St, int64_t lds, int64_t len, int l, const int32_t* perm, TC* Out,
                               int64_t ldo, cudaStream_t st) {
  const unsigned grid = (unsigned)cdiv(len, 32);
  if (grid) { gather_cols_kernel<TC><<<grid, 256, 0, st>>>(St, lds, len, l, perm, Out, ldo); CORUTV_COUNT_LAUNCH(); }
  return cudaGetLastError();
}

// Xt[j][i] = Phi[i][j] (ST staging of the caller's row-major Psi).
template <typename TC>
__global__ void stage_transpose_kernel(const TC* __restrict__ Phi, int64_t ldphi, int64_t len, int l,
                                       TC* __restrict__ Xt, int64_t ldx) {
  __shared__ TC tile[32][kMaxL + 1];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  for (int e = threadIdx.x; e < 32 * l; e += blockDim.x) {
    const int ii = e / l, j = e % l;
    const int64_t g = i0 + ii;
    tile[ii][j] = g < len ? Phi[g * ldphi + j] : TC(0);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < l * 32; e += blockDim.x) {
    const int j = e / 32, ii = e % 32;
    const int64_t g = i0 + ii;
    if (g < len) Xt[j * ldx + g] = tile[ii][j];
  }
}

template <typename TC>
cudaError_t launch_stage_transpose(const TC* Phi, int64_t ldphi, int64_t len, int l, TC* Xt, int64_t ldx,
                                   cudaStream_t st) {
  const unsigned grid = (unsigned)cdiv(len, 32);
  if (grid) { stage_transpose_kernel<TC><<<grid, 256, 0, st>>>(Phi, ldphi, len, l, Xt, ldx); CORUTV_COUNT_LAUNCH(); }
  return cudaGetLastError();
}

// =============================================================================== QRCP
// One CTA of 16 warps.  Warp w keeps columns c = w, w + 16, ... of D in
// registers (lane holds rows lane + 32 r).  Columns never move: every warp
// keeps the same position -> column map (4 entries per lane) and applies the
// same swaps, so "first maximum by current position" matches the textbook
// algorithm with physical column exchanges.  Step j: all warps pick the pivot
// from the trailing norms (shared memory); its owner builds the Householder
// vector and publishes it; every warp applies it to its trailing columns and
// recomputes their trailing norms exactly.  Two block barriers per step; the
// reductions of a warp's columns are interleaved.  Q~ = H_0 ... H_{l-1} is then
// formed column by column in registers without barriers.
template <typename TC>
__device__ __forceinline__ TC warp_sum(TC v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int sel4(const int (&m)[4], int r) {
  int v = m[0];
  v = (r == 1) ? m[1] : v;
  v = (r == 2) ? m[2] : v;
  v = (r == 3) ? m[3] : v;
  return v;
}

template <typename TC>
__global__ void __launch_bounds__(512) qrcp_kernel(const double* __restrict__ Dg, int64_t ldd, int l, int k,
                                                   double* __restrict__ Qg, int64_t ldq, double* __restrict__ Rg,
                                                   int64_t ldr, int r_transposed, int32_t* __restrict__ perm,
                                                   double* __restrict__ fro2, DevStatus* status) {
  constexpr int NW = 16, U = kMaxL / NW;    // 8 columns per warp
  extern __shared__ unsigned char smem_raw[];
  TC* Vs = reinterpret_cast<TC*>(smem_raw);  // Vs[j * kMaxL + i]: reflector j (rows i >= j)
  __shared__ TC norms[kMaxL];
  __shared__ TC betas[kMaxL];
  __shared__ TC rdiag[kMaxL];
  __shared__ int pcol[kMaxL];
  __shared__ double red[NW][2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  TC d[U][4];
  bool trailing[U];
  int posof[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int c = warp + NW * u;
    trailing[u] = c < l;
    posof[u] = -1;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = lane + 32 * r;
      d[u][r] = (c < l && i < l) ? (TC)Dg[i * ldd + c] : TC(0);
    }
  }
  {
    TC nv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) nv[u] = d[u][0] * d[u][0] + d[u][1] * d[u][1] + d[u][2] * d[u][2] + d[u][3] * d[u][3];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int u = 0; u < U; ++u) nv[u] += __shfl_xor_sync(0xffffffffu, nv[u], o);
    if (lane == 0)
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (warp + NW * u < l) norms[warp + NW * u] = nv[u];
  }
  int map[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) map[r] = lane + 32 * r;
  __syncthreads();

  for (int j = 0; j < l; ++j) {
    // pivot: first maximum of the trailing norms by current position
    TC best = TC(-1);
    int bpos = l;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int pos = lane + 32 * r;
      if (pos >= j && pos < l) {
        const TC nv = norms[map[r]];
        if (nv > best) { best = nv; bpos = pos; }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const TC ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int op = __shfl_xor_sync(0xffffffffu, bpos, o);
      if (ob > best || (ob == best && op < bpos)) { best = ob; bpos = op; }
    }
    const int cj = __shfl_sync(0xffffffffu, sel4(map, j >> 5), j & 31);
    const int cp = __shfl_sync(0xffffffffu, sel4(map, (bpos >> 5) & 3), bpos & 31);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int pos = lane + 32 * r;
      if (pos == j) map[r] = cp;
      else if (pos == bpos) map[r] = cj;
    }
    // owner of the pivot column builds and publishes the reflector (rows j..l-1)
    if (warp == cp % NW) {
      const int up = cp / NW;
      TC x[4];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (u == up)
#pragma unroll
          for (int r = 0; r < 4; ++r) x[r] = d[u][r];
      TC ss = 0;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int i = lane + 32 * r;
        if (i >= j && i < l) ss += x[r] * x[r];
      }
      ss = warp_sum(ss);
      const TC x0 = __shfl_sync(0xffffffffu, (j >> 5) == 0 ? x[0] : ((j >> 5) == 1 ? x[1] : ((j >> 5) == 2 ? x[2] : x[3])), j & 31);
      const TC nrm = sqrt(ss);
      TC alpha, v0, beta;
      if (nrm == TC(0)) {
        alpha = 0; v0 = 1; beta = 0;
      } else {
        alpha = (x0 >= TC(0)) ? -nrm : nrm;
        v0 = x0 - alpha;
        beta = TC(1) / (nrm * (nrm + fabs(x0)));
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int i = lane + 32 * r;
        if (i >= j && i < l) Vs[j * kMaxL + i] = (i == j) ? v0 : x[r];
      }
      if (lane == 0) { betas[j] = beta; rdiag[j] = alpha; pcol[j] = cp; }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (u == up) { trailing[u] = false; posof[u] = j; }
    }
    __syncthreads();
    // apply the reflector to this warp's trailing columns and recompute their norms
    const TC beta = betas[j];
    TC v[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = lane + 32 * r;
      v[r] = (i >= j && i < l) ? Vs[j * kMaxL + i] : TC(0);
    }
    TC w[U];
#pragma unroll
    for (int u = 0; u < U; ++u) w[u] = v[0] * d[u][0] + v[1] * d[u][1] + v[2] * d[u][2] + v[3] * d[u][3];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int u = 0; u < U; ++u) w[u] += __shfl_xor_sync(0xffffffffu, w[u], o);
    TC nv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      nv[u] = 0;
      if (trailing[u]) {
        const TC f = beta * w[u];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          d[u][r] -= f * v[r];
          const int i = lane + 32 * r;
          if (i > j && i < l) nv[u] += d[u][r] * d[u][r];
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int u = 0; u < U; ++u) nv[u] += __shfl_xor_sync(0xffffffffu, nv[u], o);
    if (lane == 0)
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (trailing[u]) norms[warp + NW * u] = nv[u];
    __syncthreads();
  }

  // R (diag(R) >= 0 by flipping rows with a negative pivot) from each pivot column's owner
  double fa = 0.0, fb = 0.0;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int jp = posof[u];
    if (jp < 0) continue;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = lane + 32 * r;
      if (i >= l) continue;
      TC val;
      if (i < jp) val = (rdiag[i] < TC(0) ? TC(-1) : TC(1)) * d[u][r];
      else if (i == jp) val = fabs(rdiag[i]);
      else val = 0;
      if (r_transposed) Rg[jp * ldr + i] = (double)val;
      else Rg[i * ldr + jp] = (double)val;
      fa += (double)val * (double)val;
      if (i < k) fb += (double)val * (double)val;
    }
  }
  fa = warp_sum(fa);
  fb = warp_sum(fb);
  if (lane == 0) { red[warp][0] = fa; red[warp][1] = fb; }
  // Q~: column q = H_0 ... H_q e_q (registers reuse the warp's column slots)
  TC qv[U][4];
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int r = 0; r < 4; ++r) qv[u][r] = (warp + NW * u == lane + 32 * r) ? TC(1) : TC(0);
  for (int j = l - 1; j >= 0; --j) {
    const TC beta = betas[j];
    TC v[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = lane + 32 * r;
      v[r] = (i >= j && i < l) ? Vs[j * kMaxL + i] : TC(0);
    }
    TC w[U];
#pragma unroll
    for (int u = 0; u < U; ++u) w[u] = v[0] * qv[u][0] + v[1] * qv[u][1] + v[2] * qv[u][2] + v[3] * qv[u][3];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int u = 0; u < U; ++u) w[u] += __shfl_xor_sync(0xffffffffu, w[u], o);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (warp + NW * u < j) continue;       // H_j leaves e_q untouched for q < j
      const TC f = beta * w[u];
#pragma unroll
      for (int r = 0; r < 4; ++r) qv[u][r] -= f * v[r];
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int q = warp + NW * u;
    if (q >= l) continue;
    const TC sg = rdiag[q] < TC(0) ? TC(-1) : TC(1);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = lane + 32 * r;
      if (i < l) Qg[i * ldq + q] = (double)(sg * qv[u][r]);
    }
  }
  for (int j = tid; j < l; j += blockDim.x) perm[j] = pcol[j];
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, b = 0.0;
    for (int w2 = 0; w2 < NW; ++w2) { a += red[w2][0]; b += red[w2][1]; }
    if (fro2) { fro2[0] = a; fro2[1] = b; }
    if (status) { status->fro2_T = a; status->fro2_Tk = b; }
  }
}

// FP32 variant with columns in registers: thread (c, h) holds rows
// i = 64 h .. 64 h + 63 of column c, so every column reduction is a per-thread
// sum (four independent partial sums) plus one shuffle.  The published
// reflector is zero outside rows j..l-1, so it is applied with unpredicated
// vector loads.  Step j: trailing norms are published by position; after a
// barrier every warp evaluates the same argmax and applies the same swap to
// its copy of the position map; the two threads of the pivot column publish
// the reflector; after a second barrier every trailing column is updated and
// its trailing norm recomputed exactly.  Same choices as the warp-per-column
// kernel (first maximum by current position).
template <int N>
__device__ __forceinline__ float dotN(const float* __restrict__ v, const float (&x)[N]) {
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  const float4* v4 = reinterpret_cast<const float4*>(v);
#pragma unroll
  for (int q = 0; q < N / 4; ++q) {
    const float4 t = v4[q];
    s0 = fmaf(t.x, x[4 * q + 0], s0);
    s1 = fmaf(t.y, x[4 * q + 1], s1);
    s2 = fmaf(t.z, x[4 * q + 2], s2);
    s3 = fmaf(t.w, x[4 * q + 3], s3);
  }
  return (s0 + s1) + (s2 + s3);
}

template <int N>
__device__ __forceinline__ void axpyN(const float* __restrict__ v, float f, float (&x)[N]) {
  const float4* v4 = reinterpret_cast<const float4*>(v);
#pragma unroll
  for (int q = 0; q < N / 4; ++q) {
    const float4 t = v4[q];
    x[4 * q + 0] = fmaf(-f, t.x, x[4 * q + 0]);
    x[4 * q + 1] = fmaf(-f, t.y, x[4 * q + 1]);
    x[4 * q + 2] = fmaf(-f, t.z, x[4 * q + 2]);
    x[4 * q + 3] = fmaf(-f, t.w, x[4 * q + 3]);
  }
}

template <int TPC>
__global__ void __launch_bounds__(kMaxL * TPC) qrcp_reg_kernel(const double* __restrict__ Dg, int64_t ldd, int l, int k,
                                                       double* __restrict__ Qg, int64_t ldq, double* __restrict__ Rg,
                                                       int64_t ldr, int r_transposed, int32_t* __restrict__ perm,
                                                       double* __restrict__ fro2, DevStatus* status) {
  constexpr int RPT = kMaxL / TPC, NWARP = kMaxL * TPC / 32, CPW = 32 / TPC;   // columns per warp
  __shared__ __align__(16) float vbuf[kMaxL];       // reflector of the current step (zero outside j..l-1)
  __shared__ __align__(16) float pcolv[kMaxL];      // raw pivot column
  __shared__ float npos[kMaxL];                      // trailing norms by current position
  __shared__ float sc[2];                            // beta, alpha of the current step
  __shared__ int piv[3];                             // pivot column, column previously at position j, its new position
  __shared__ float rdiag[kMaxL];
  __shared__ int pcol[kMaxL];
  __shared__ double red[NWARP][2];
  const int tid = threadIdx.x, c = tid / TPC, h = tid % TPC, lane = tid & 31, warp = tid >> 5;
  const int i0 = RPT * h;
  const unsigned grp = ((TPC == 32) ? 0xffffffffu : ((1u << TPC) - 1u)) << (lane & ~(TPC - 1));
  float d[RPT], m[RPT];       // column c of D (rows i0..) and column c of M = H_j ... H_0 (rows i0..)
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int i = i0 + r;
    d[r] = (c < l && i < l) ? (float)Dg[i * ldd + c] : 0.f;
    m[r] = (i == c) ? 1.f : 0.f;
  }
  int map[4];                 // position -> column (kept by warp 0)
#pragma unroll
  for (int r = 0; r < 4; ++r) map[r] = lane + 32 * r;
  int mypos = c;
  bool trailing = c < l;
  int posof = -1;
  {
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int r = 0; r < RPT; r += 2) { s0 = fmaf(d[r], d[r], s0); s1 = fmaf(d[r + 1], d[r + 1], s1); }
    float ss = s0 + s1;
#pragma unroll
    for (int o = 1; o < TPC; o <<= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (h == 0 && c < l) npos[c] = ss;
  }
  __syncthreads();
  for (int j = 0; j < l; ++j) {
    // ---- phase 1: warp 0 picks the pivot (first maximum by current position) and swaps the map
    if (warp == 0) {
      float best = -1.f;
      int bpos = l;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int pos = lane + 32 * r;
        if (pos >= j && pos < l) {
          const float nv = npos[pos];
          if (nv > best) { best = nv; bpos = pos; }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int op = __shfl_xor_sync(0xffffffffu, bpos, o);
        if (ob > best || (ob == best && op < bpos)) { best = ob; bpos = op; }
      }
      const int cj = __shfl_sync(0xffffffffu, sel4(map, j >> 5), j & 31);
      const int cp = __shfl_sync(0xffffffffu, sel4(map, (bpos >> 5) & 3), bpos & 31);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int pos = lane + 32 * r;
        if (pos == j) map[r] = cp;
        else if (pos == bpos) map[r] = cj;
      }
      if (lane == 0) { piv[0] = cp; piv[1] = cj; piv[2] = bpos; }
    }
    __syncthreads();
    const int cp = piv[0];
    if (c == piv[1]) mypos = piv[2];
    if (c == cp) mypos = j;
    // ---- phase 2: the pivot column's warp builds the reflector from a shared copy of the column
    if (warp == cp / CPW) {
      if (c == cp) {
        float4* p4 = reinterpret_cast<float4*>(pcolv + i0);
#pragma unroll
        for (int q = 0; q < RPT / 4; ++q) p4[q] = make_float4(d[4 * q], d[4 * q + 1], d[4 * q + 2], d[4 * q + 3]);
        trailing = false;
        posof = j;
      }
      __syncwarp();
      const float4 x4 = reinterpret_cast<const float4*>(pcolv)[lane];   // rows 4 lane .. 4 lane + 3
      float xv[4] = {x4.x, x4.y, x4.z, x4.w};
      float ss = 0.f;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = 4 * lane + e;
        if (i >= j && i < l) ss = fmaf(xv[e], xv[e], ss);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      const float x0 = pcolv[j];
      const float nrm = sqrtf(ss);
      float alpha, v0, beta;
      if (nrm == 0.f) {
        alpha = 0.f; v0 = 1.f; beta = 0.f;
      } else {
        alpha = (x0 >= 0.f) ? -nrm : nrm;
        v0 = x0 - alpha;
        beta = 1.f / (nrm * (nrm + fabsf(x0)));
      }
      float4 vo;
      float* vp = &vo.x;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = 4 * lane + e;
        vp[e] = (i == j) ? v0 : ((i > j && i < l) ? xv[e] : 0.f);
      }
      reinterpret_cast<float4*>(vbuf)[lane] = vo;
      if (lane == 0) { sc[0] = beta; sc[1] = alpha; rdiag[j] = alpha; pcol[j] = cp; }
    }
    __syncthreads();
    // ---- phase 3: every column of M and every trailing column of D takes the reflector
    {
      float v[RPT];
      const float4* v4 = reinterpret_cast<const float4*>(vbuf + i0);
#pragma unroll
      for (int q = 0; q < RPT / 4; ++q) {
        const float4 t = v4[q];
        v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
      }
      const float beta = sc[0];
      float wm0 = 0.f, wm1 = 0.f, wd0 = 0.f, wd1 = 0.f;
#pragma unroll
      for (int r = 0; r < RPT; r += 2) {
        wm0 = fmaf(v[r], m[r], wm0);
        wm1 = fmaf(v[r + 1], m[r + 1], wm1);
        wd0 = fmaf(v[r], d[r], wd0);
        wd1 = fmaf(v[r + 1], d[r + 1], wd1);
      }
      float wm = wm0 + wm1, wd = trailing ? wd0 + wd1 : 0.f;
#pragma unroll
      for (int o = 1; o < TPC; o <<= 1) {
        wm += __shfl_xor_sync(grp, wm, o);
        wd += __shfl_xor_sync(grp, wd, o);
      }
      const float fm = beta * wm, fd = beta * wd;
      float s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        m[r] = fmaf(-fm, v[r], m[r]);
        d[r] = fmaf(-fd, v[r], d[r]);          // fd = 0 for columns that are not trailing
        const float x = (i0 + r > j) ? d[r] : 0.f;
        if (r & 1) s1 = fmaf(x, x, s1); else s0 = fmaf(x, x, s0);
      }
      if (trailing) {
        float ns = s0 + s1;
#pragma unroll
        for (int o = 1; o < TPC; o <<= 1) ns += __shfl_xor_sync(grp, ns, o);
        if (h == 0) npos[mypos] = ns;
      }
    }
    __syncthreads();
  }
  // R from each pivot column (rows above its position), diag(R) >= 0
  double fa = 0.0, fb = 0.0;
  if (posof >= 0) {
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int i = i0 + r;
      if (i >= l) continue;
      float val;
      if (i < posof) val = (rdiag[i] < 0.f ? -1.f : 1.f) * d[r];
      else if (i == posof) val = fabsf(rdiag[i]);
      else val = 0.f;
      if (r_transposed) Rg[posof * ldr + i] = (double)val;
      else Rg[i * ldr + posof] = (double)val;
      fa += (double)val * (double)val;
      if (i < k) fb += (double)val * (double)val;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    fa += __shfl_xor_sync(0xffffffffu, fa, o);
    fb += __shfl_xor_sync(0xffffffffu, fb, o);
  }
  if (lane == 0) { red[warp][0] = fa; red[warp][1] = fb; }
  // Q~ = H_0 ... H_{l-1} = M^T: Q~[c][q] = M[q][c] (thread holds M[i0.., c]), column sign from diag(R)
  if (c < l) {
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int q = i0 + r;
      if (q < l) Qg[c * ldq + q] = (double)((rdiag[q] < 0.f ? -1.f : 1.f) * m[r]);
    }
  }
  for (int j = tid; j < l; j += blockDim.x) perm[j] = pcol[j];
  __syncthreads();
  if (tid == 0) {
    double a2 = 0.0, b2 = 0.0;
    for (int w2 = 0; w2 < NWARP; ++w2) { a2 += red[w2][0]; b2 += red[w2][1]; }
    if (fro2) { fro2[0] = a2; fro2[1] = b2; }
    if (status) { status->fro2_T = a2; status->fro2_Tk = b2; }
  }
}

template <typename TC>
cudaError_t launch_qrcp(const double* D, int64_t ldd, int l, int k, double* Q, int64_t ldq, double* R, int64_t ldr,
                        bool r_transposed, int32_t* perm, double* fro2, DevStatus* status, cudaStream_t st) {
  const size_t smem = (size_t)l * kMaxL * sizeof(TC);
  if constexpr (sizeof(TC) == 4) {
    qrcp_reg_kernel<kQrcpTPC><<<1, kMaxL * kQrcpTPC, 0, st>>>(D, ldd, l, k, Q, ldq, R, ldr, r_transposed ? 1 : 0,
                                                                 perm, fro2, status);
    CORUTV_COUNT_LAUNCH();
    return cudaGetLastError();
  }
  cudaError_t e = cudaFuncSetAttribute(qrcp_kernel<TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  qrcp_kernel<TC><<<1, 512, smem, st>>>(D, ldd, l, k, Q, ldq, R, ldr, r_transposed ? 1 : 0, perm, fro2, status); CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

// =============================================================================== ||A||_F^2
// FP32 squares folded into FP64 every 64 elements (FP64 throughout for FP64 A);
// per-block partials then an ordered FP64 sum.
template <typename TA>
__global__ void __launch_bounds__(256) fro2_kernel(const TA* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                                                   const float* __restrict__ scales, int64_t sld,
                                                   double* __restrict__ parts) {
  using TC = typename Elem<TA>::acc;
  __shared__ double red[8];
  double acc = 0.0;
  TC run = 0;
  int cnt = 0;
  const int64_t total = m * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e - i * n;
    const TC a = Elem<TA>::load(A, i, j, lda, scales, sld);
    run = fma(a, a, run);
    if (++cnt == 64) { acc += (double)run; run = 0; cnt = 0; }
  }
  acc += (double)run;
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    parts[blockIdx.x] = s;
  }
}

__global__ void sum_parts_kernel(const double* __restrict__ parts, int n, double* out, DevStatus* status) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += parts[i];
    if (out) *out = s;
    if (status) status->fro2_A = s;
  }
}

int fro2_parts(int sms) { return sms * 4; }

cudaError_t launch_fro2(int a_dtype, const void* A, int64_t lda, int64_t m, int64_t n, const float* scales,
                        int64_t sld, double* parts, int nparts, double* out, cudaStream_t st) {
  switch (a_dtype) {
    case 0: fro2_kernel<double><<<nparts, 256, 0, st>>>((const double*)A, lda, m, n, scales, sld, parts); CORUTV_COUNT_LAUNCH(); break;
    case 1: fro2_kernel<float><<<nparts, 256, 0, st>>>((const float*)A, lda, m, n, scales, sld, parts); CORUTV_COUNT_LAUNCH(); break;
    case 2:
      fro2_kernel<__nv_bfloat16><<<nparts, 256, 0, st>>>((const __nv_bfloat16*)A, lda, m, n, scales, sld, parts); CORUTV_COUNT_LAUNCH();
      break;
    case 3:
      fro2_kernel<__nv_fp8_e4m3><<<nparts, 256, 0, st>>>((const __nv_fp8_e4m3*)A, lda, m, n, scales, sld, parts); CORUTV_COUNT_LAUNCH();
      break;
    default: return cudaErrorInvalidValue;
  }
  sum_parts_kernel<<<1, 32, 0, st>>>(parts, nparts, out, nullptr); CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ instantiations
#define INST(TC)                                                                                                   \
  template cudaError_t launch_gram<TC>(const TC*, int64_t, const TC*, int64_t, int64_t, int, TC*, int, double*,   \
                                       int64_t, cudaStream_t);                                                     \
  template cudaError_t launch_cholinv<TC>(const double*, int64_t, int, double, double, TC*, TC*, int*, DevStatus*, \
                                          double*, cudaStream_t);                                                  \
  template cudaError_t launch_lmul<TC>(const TC*, int64_t, int64_t, int, const TC*, int64_t, TC*, int64_t, bool,  \
                                       cudaStream_t);                                                              \
  template cudaError_t launch_lmul_f64s<TC>(const TC*, int64_t, int64_t, int, const double*, int64_t, TC*,        \
                                            int64_t, bool, cudaStream_t);                                          \
  template cudaError_t launch_fill_deficient<TC>(TC*, int64_t, int64_t, int, const int*, int, cudaStream_t);      \
  template cudaError_t launch_gather_cols<TC>(const TC*, int64_t, int64_t, int, const int32_t*, TC*, int64_t,     \
                                              cudaStream_t);                                                       \
  template cudaError_t launch_stage_transpose<TC>(const TC*, int64_t, int64_t, int, TC*, int64_t, cudaStream_t);  \
  template cudaError_t launch_qrcp<TC>(const double*, int64_t, int, int, double*, int64_t, double*, int64_t, bool, \
                                       int32_t*, double*, DevStatus*, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace corutv
