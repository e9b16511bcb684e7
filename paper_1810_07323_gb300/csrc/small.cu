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

// =============================================================================== Gram
// parts[c] = X[:, cols_c] Y[:, cols_c]^T over the c-th contiguous column range.
template <typename TC, int JPT>
__global__ void __launch_bounds__(256) gram_partial_kernel(const TC* __restrict__ Xt, int64_t ldx,
                                                           const TC* __restrict__ Yt, int64_t ldy, int64_t len,
                                                           int l, TC* __restrict__ parts) {
  constexpr int LP = 16 * JPT;
  constexpr int BK = 32;
  __shared__ TC Xs[LP][BK + 1];
  __shared__ TC Ys[LP][BK + 1];
  const int tid = threadIdx.x, ti = tid & 15, tj = tid >> 4;
  const int64_t chunk = cdiv(cdiv(len, BK), gridDim.x) * BK;
  const int64_t c0 = blockIdx.x * chunk;
  int64_t c1 = c0 + chunk;
  if (c1 > len) c1 = len;
  TC acc[JPT][JPT];
#pragma unroll
  for (int v = 0; v < JPT; ++v)
#pragma unroll
    for (int u = 0; u < JPT; ++u) acc[v][u] = TC(0);
  for (int64_t k0 = c0; k0 < c1; k0 += BK) {
    for (int x = tid; x < LP * BK; x += 256) {
      const int r = x / BK, kk = x % BK;
      const int64_t g = k0 + kk;
      const bool ok = r < l && g < c1;
      Xs[r][kk] = ok ? Xt[r * ldx + g] : TC(0);
      Ys[r][kk] = ok ? Yt[r * ldy + g] : TC(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < BK; ++kk) {
      TC xa[JPT], yb[JPT];
#pragma unroll
      for (int v = 0; v < JPT; ++v) xa[v] = Xs[tj + 16 * v][kk];
#pragma unroll
      for (int u = 0; u < JPT; ++u) yb[u] = Ys[ti + 16 * u][kk];
#pragma unroll
      for (int v = 0; v < JPT; ++v)
#pragma unroll
        for (int u = 0; u < JPT; ++u) acc[v][u] = fma(xa[v], yb[u], acc[v][u]);
    }
    __syncthreads();
  }
  TC* out = parts + (int64_t)blockIdx.x * LP * LP;
#pragma unroll
  for (int v = 0; v < JPT; ++v)
#pragma unroll
    for (int u = 0; u < JPT; ++u) out[(tj + 16 * v) * LP + ti + 16 * u] = acc[v][u];
}

// G[a][b] = sum over parts in order, in FP64.
template <typename TC>
__global__ void gram_reduce_kernel(const TC* __restrict__ parts, int nparts, int LP, int l, double* __restrict__ G,
                                   int64_t ldg) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= l * l) return;
  const int a = e / l, b = e % l;
  double s = 0.0;
  for (int p = 0; p < nparts; ++p) s += (double)parts[((int64_t)p * LP + a) * LP + b];
  G[a * ldg + b] = s;
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
    gram_partial_kernel<TC, 2><<<gparts, 256, 0, st>>>(Xt, ldx, Yt, ldy, len, l, parts); CORUTV_COUNT_LAUNCH();
  } else if (l <= 64) {
    LP = 64;
    gram_partial_kernel<TC, 4><<<gparts, 256, 0, st>>>(Xt, ldx, Yt, ldy, len, l, parts); CORUTV_COUNT_LAUNCH();
  } else {
    LP = 128;
    gram_partial_kernel<TC, 8><<<gparts, 256, 0, st>>>(Xt, ldx, Yt, ldy, len, l, parts); CORUTV_COUNT_LAUNCH();
  }
  gram_reduce_kernel<TC><<<(unsigned)cdiv((int64_t)l * l, 256), 256, 0, st>>>(parts, gparts, LP, l, G, ldg); CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

// =============================================================================== Cholesky
// G + s I = R^T R (R upper, s = shift_rel * trace(G)), right-looking, with
// R^-1 built column by column in the same sweep:
//   Rinv[i][j] = (delta_ij - sum_{p=i}^{j-1} Rinv[i][p] R[p][j]) / R[j][j].
// Storage: the active trailing matrix lives in the upper triangle of Gs, the
// finished rows of R are stored transposed in its lower triangle
// (R[p][b] at Gs[b][p]), so one barrier per column suffices.
// A pivot d <= tol_rel * (G_jj + s) marks column j dependent: R[j][j] = 1,
// R[j][>j] = 0, and defic[j] = 1 (the caller replaces that column of Q).
template <typename TC>
__global__ void __launch_bounds__(512) cholinv_kernel(const double* __restrict__ G, int64_t ldg, int l,
                                                      double shift_rel, double tol_rel, TC* __restrict__ Rg,
                                                      TC* __restrict__ Rinvg, int* __restrict__ defic,
                                                      DevStatus* status, double* __restrict__ Rout) {
  extern __shared__ unsigned char smem_raw[];
  const int LD = l + 1;
  TC* Gs = reinterpret_cast<TC*>(smem_raw);     // l x LD
  TC* Ri = Gs + l * LD;                          // l x LD, R^-1 (upper)
  __shared__ double diag0[kMaxL];
  __shared__ TC rdiag[kMaxL];
  __shared__ double red[32];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;

  double tr = 0.0;
  for (int e = tid; e < l * l; e += nt) {
    const int a = e / l, b = e % l;
    const double g = G[a * ldg + b];
    if (b >= a) Gs[a * LD + b] = (TC)g;
    Ri[a * LD + b] = TC(0);
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

  int nfall = 0;
  for (int j = 0; j < l; ++j) {
    // every thread evaluates the pivot of column j (final since the last barrier)
    const TC d = Gs[j * LD + j];
    const bool dep = !((double)d > tol_rel * diag0[j]) || !(diag0[j] > 0.0);
    const TC piv = dep ? TC(1) : (TC)sqrt(d);
    const TC rs = dep ? TC(0) : TC(1) / piv;
    if (tid == 0) {
      defic[j] = dep ? 1 : 0;
      rdiag[j] = piv;
      nfall += dep ? 1 : 0;
    }
    // (a) column j of R^-1, rows i <= j (R[p][j] = Gs[j][p] for p < j)
    for (int i = tid; i <= j; i += nt) {
      TC s0 = (i == j) ? TC(1) : TC(0), s1 = TC(0);
      int p = i;
      for (; p + 1 < j; p += 2) {
        s0 -= Ri[i * LD + p] * Gs[j * LD + p];
        s1 -= Ri[i * LD + p + 1] * Gs[j * LD + p + 1];
      }
      if (p < j) s0 -= Ri[i * LD + p] * Gs[j * LD + p];
      Ri[i * LD + j] = (s0 + s1) / piv;
    }
    // (b) trailing update, upper triangle: G[a][b] -= R[j][a] R[j][b], j < a <= b
    for (int a = j + 1 + warp; a < l; a += nw) {
      const TC rja = Gs[j * LD + a] * rs;
      for (int b = a + lane; b < l; b += 32) Gs[a * LD + b] -= rja * (Gs[j * LD + b] * rs);
    }
    // (c) finished row j of R, stored transposed in the lower triangle
    for (int b = j + 1 + tid; b < l; b += nt) Gs[b * LD + j] = Gs[j * LD + b] * rs;
    __syncthreads();
  }
  for (int e = tid; e < l * l; e += nt) {
    const int a = e / l, b = e % l;
    const TC r = (b > a) ? Gs[b * LD + a] : (b == a ? rdiag[a] : TC(0));
    Rg[a * kMaxL + b] = r;
    Rinvg[a * kMaxL + b] = (b >= a) ? Ri[a * LD + b] : TC(0);
    if (Rout) Rout[a * l + b] = (double)r;
  }
  if (tid == 0 && nfall && status) atomicAdd(&status->chol_fallbacks, nfall);
}

template <typename TC>
cudaError_t launch_cholinv(const double* G, int64_t ldg, int l, double shift_rel, double tol_rel, TC* R, TC* Rinv,
                           int* defic, DevStatus* status, double* Rout, cudaStream_t st) {
  const size_t smem = (size_t)2 * l * (l + 1) * sizeof(TC);
  cudaError_t e = cudaFuncSetAttribute(cholinv_kernel<TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cholinv_kernel<TC><<<1, 512, smem, st>>>(G, ldg, l, shift_rel, tol_rel, R, Rinv, defic, status, Rout); CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

// =============================================================================== lmul
// Out[j][i] = sum_{p<l} S[p][j] In[p][i]   (Out = S^T In on ST blocks, i.e. C S in
// the untransposed view).  out_rowmajor: write Out^T into a row-major len x l matrix.
template <typename TC, typename TS, int JPT>
__global__ void __launch_bounds__(256) lmul_kernel(const TC* __restrict__ In, int64_t ldi, int64_t len, int l,
                                                   const TS* __restrict__ S, int64_t lds, TC* __restrict__ Out,
                                                   int64_t ldo, int out_rowmajor) {
  constexpr int LP = 16 * JPT;
  constexpr int BI = 64;
  extern __shared__ unsigned char smem_raw[];
  TC* Ss = reinterpret_cast<TC*>(smem_raw);      // LP x (LP+1)
  TC* Is = Ss + LP * (LP + 1);                   // LP x (BI+1)
  const int tid = threadIdx.x, ti = tid & 15, tj = tid >> 4;
  const int64_t i0 = (int64_t)blockIdx.x * BI;
  for (int e = tid; e < LP * LP; e += 256) {
    const int p = e / LP, j = e % LP;
    Ss[p * (LP + 1) + j] = (p < l && j < l) ? (TC)S[p * lds + j] : TC(0);
  }
  for (int e = tid; e < LP * BI; e += 256) {
    const int p = e / BI, ii = e % BI;
    const int64_t g = i0 + ii;
    Is[p * (BI + 1) + ii] = (p < l && g < len) ? In[p * ldi + g] : TC(0);
  }
  __syncthreads();
  TC acc[JPT][4];
#pragma unroll
  for (int v = 0; v < JPT; ++v)
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[v][u] = TC(0);
  for (int p = 0; p < l; ++p) {
    TC sv[JPT], xv[4];
#pragma unroll
    for (int v = 0; v < JPT; ++v) sv[v] = Ss[p * (LP + 1) + tj + 16 * v];
#pragma unroll
    for (int u = 0; u < 4; ++u) xv[u] = Is[p * (BI + 1) + ti + 16 * u];
#pragma unroll
    for (int v = 0; v < JPT; ++v)
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[v][u] = fma(sv[v], xv[u], acc[v][u]);
  }
  __syncthreads();
  if (!out_rowmajor) {
#pragma unroll
    for (int v = 0; v < JPT; ++v) {
      const int j = tj + 16 * v;
      if (j >= l) continue;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t g = i0 + ti + 16 * u;
        if (g < len) Out[j * ldo + g] = acc[v][u];
      }
    }
  } else {
    // stage through shared memory (reuse Is as [BI][LP+1]) so row-major writes coalesce
    TC* Os = Is;
#pragma unroll
    for (int v = 0; v < JPT; ++v)
#pragma unroll
      for (int u = 0; u < 4; ++u) Os[(ti + 16 * u) * (LP + 1) + tj + 16 * v] = acc[v][u];
    __syncthreads();
    for (int e = tid; e < BI * l; e += 256) {
      const int ii = e / l, j = e % l;
      const int64_t g = i0 + ii;
      if (g < len) Out[g * ldo + j] = Os[ii * (LP + 1) + j];
    }
  }
}

template <typename TC, typename TS>
static cudaError_t lmul_dispatch(const TC* In, int64_t ldi, int64_t len, int l, const TS* S, int64_t lds, TC* Out,
                                 int64_t ldo, bool rowmajor, cudaStream_t st) {
  const unsigned grid = (unsigned)cdiv(len, 64);
  if (grid == 0) return cudaSuccess;
  int LP = l <= 32 ? 32 : (l <= 64 ? 64 : 128);
  const size_t smem = (size_t)(LP * (LP + 1) + LP * 65) * sizeof(TC);
  const size_t smem_out = (size_t)(LP * (LP + 1) + 64 * (LP + 1)) * sizeof(TC);
  const size_t sm = smem > smem_out ? smem : smem_out;
  cudaError_t e;
  if (LP == 32) {
    e = cudaFuncSetAttribute(lmul_kernel<TC, TS, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    lmul_kernel<TC, TS, 2><<<grid, 256, sm, st>>>(In, ldi, len, l, S, lds, Out, ldo, rowmajor); CORUTV_COUNT_LAUNCH();
  } else if (LP == 64) {
    e = cudaFuncSetAttribute(lmul_kernel<TC, TS, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    lmul_kernel<TC, TS, 4><<<grid, 256, sm, st>>>(In, ldi, len, l, S, lds, Out, ldo, rowmajor); CORUTV_COUNT_LAUNCH();
  } else {
    e = cudaFuncSetAttribute(lmul_kernel<TC, TS, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    lmul_kernel<TC, TS, 8><<<grid, 256, sm, st>>>(In, ldi, len, l, S, lds, Out, ldo, rowmajor); CORUTV_COUNT_LAUNCH();
  }
  return cudaGetLastError();
}

template <typename TC>
cudaError_t launch_lmul(const TC* In, int64_t ldi, int64_t len, int l, const TC* S, int64_t lds, TC* Out,
                        int64_t ldo, bool out_rowmajor, cudaStream_t st) {
  return lmul_dispatch<TC, TC>(In, ldi, len, l, S, lds, Out, ldo, out_rowmajor, st);
}
template <typename TC>
cudaError_t launch_lmul_f64s(const TC* In, int64_t ldi, int64_t len, int l, const double* S, int64_t lds, TC* Out,
                             int64_t ldo, bool out_rowmajor, cudaStream_t st) {
  return lmul_dispatch<TC, double>(In, ldi, len, l, S, lds, Out, ldo, out_rowmajor, st);
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
// One CTA, 16 warps.  Columns are never moved in shared memory: every warp
// keeps the same position -> column map (4 entries per lane) and applies the
// same swaps, so "first maximum by current position" matches the textbook
// algorithm with physical column exchanges.  Warp w owns physical columns
// c = w, w + 16, ...; each step it updates its trailing columns with the
// reflector and recomputes their trailing norms exactly.  One block barrier
// per step.  Q~ is then formed column by column (H_0 ... H_{l-1} e_c) without
// barriers.
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
  extern __shared__ unsigned char smem_raw[];
  const int LD = l + 1;
  TC* Ds = reinterpret_cast<TC*>(smem_raw);   // column-major: Ds[c*LD + i] = D[i][c]
  TC* Qs = Ds + l * LD;                        // column-major Q~
  __shared__ TC norms[kMaxL];
  __shared__ TC vdiag[kMaxL];
  __shared__ TC betas[kMaxL];
  __shared__ TC rdiag[kMaxL];
  __shared__ int pcol[kMaxL];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;

  for (int e = tid; e < l * l; e += blockDim.x) {
    const int i = e / l, c = e % l;
    Ds[c * LD + i] = (TC)Dg[i * ldd + c];
  }
  __syncthreads();
  for (int c = warp; c < l; c += nw) {
    TC s = 0;
    for (int i = lane; i < l; i += 32) s += Ds[c * LD + i] * Ds[c * LD + i];
    s = warp_sum(s);
    if (lane == 0) norms[c] = s;
  }
  // position -> column map, lane holds positions lane + 32*r
  int map[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) map[r] = lane + 32 * r;
  __syncthreads();

  for (int j = 0; j < l; ++j) {
    // argmax of trailing norms over positions j..l-1, first maximum wins
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
    // swap positions j and bpos in the map
    const int cj = __shfl_sync(0xffffffffu, sel4(map, j >> 5), j & 31);
    const int cp = __shfl_sync(0xffffffffu, sel4(map, (bpos >> 5) & 3), bpos & 31);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int pos = lane + 32 * r;
      if (pos == j) map[r] = cp;
      else if (pos == bpos) map[r] = cj;
    }
    const int c = cp;   // physical pivot column
    // Householder vector of column c, rows j..l-1 (computed by every warp)
    TC x0 = Ds[c * LD + j];
    TC s = 0;
    for (int i = j + lane; i < l; i += 32) s += Ds[c * LD + i] * Ds[c * LD + i];
    s = warp_sum(s);
    const TC nrm = sqrt(s);
    TC alpha, v0, beta;
    if (nrm == TC(0)) {
      alpha = 0; v0 = 1; beta = 0;
    } else {
      alpha = (x0 >= TC(0)) ? -nrm : nrm;
      v0 = x0 - alpha;
      beta = TC(1) / (nrm * (nrm + fabs(x0)));
    }
    if (tid == 0) {
      vdiag[j] = v0; betas[j] = beta; rdiag[j] = alpha; pcol[j] = c;
    }
    // update owned trailing columns (not yet pivoted: position > j)
    for (int cc = warp; cc < l; cc += nw) {
      // is column cc still trailing (at a position > j)?  every lane checks its 4 entries
      bool mine = false;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int pos = lane + 32 * r;
        if (pos > j && pos < l && map[r] == cc) mine = true;
      }
      if (!__any_sync(0xffffffffu, mine)) continue;
      TC w = 0;
      for (int i = j + lane; i < l; i += 32) {
        const TC vi = (i == j) ? v0 : Ds[c * LD + i];
        w += vi * Ds[cc * LD + i];
      }
      w = warp_sum(w) * beta;
      TC ns = 0;
      for (int i = j + lane; i < l; i += 32) {
        const TC vi = (i == j) ? v0 : Ds[c * LD + i];
        const TC nv = Ds[cc * LD + i] - w * vi;
        Ds[cc * LD + i] = nv;
        if (i > j) ns += nv * nv;
      }
      ns = warp_sum(ns);
      if (lane == 0) norms[cc] = ns;
    }
    __syncthreads();
  }

  // Q~ = H_0 H_1 ... H_{l-1}: column q of Q~ is H_0 ... H_q e_q
  for (int q = warp; q < l; q += nw) {
    for (int i = lane; i < l; i += 32) Qs[q * LD + i] = (i == q) ? TC(1) : TC(0);
    __syncwarp();
    for (int j = q; j >= 0; --j) {
      const int c = pcol[j];
      const TC beta = betas[j], v0 = vdiag[j];
      TC w = 0;
      for (int i = j + lane; i < l; i += 32) w += ((i == j) ? v0 : Ds[c * LD + i]) * Qs[q * LD + i];
      w = warp_sum(w) * beta;
      for (int i = j + lane; i < l; i += 32) Qs[q * LD + i] -= w * ((i == j) ? v0 : Ds[c * LD + i]);
      __syncwarp();
    }
  }
  __syncthreads();
  // signs so that diag(R) >= 0; write R (or R^T), Q~, perm
  for (int e = tid; e < l * l; e += blockDim.x) {
    const int i = e / l, jj = e % l;   // R[i][jj]
    const TC sg = rdiag[i] < TC(0) ? TC(-1) : TC(1);
    TC r;
    if (jj < i) r = 0;
    else if (jj == i) r = fabs(rdiag[i]);
    else r = sg * Ds[pcol[jj] * LD + i];
    if (r_transposed) Rg[jj * ldr + i] = (double)r;
    else Rg[i * ldr + jj] = (double)r;
    const TC sq = rdiag[jj] < TC(0) ? TC(-1) : TC(1);
    Qg[i * ldq + jj] = (double)(sq * Qs[jj * LD + i]);
  }
  for (int j = tid; j < l; j += blockDim.x) perm[j] = pcol[j];
  // ||R||_F^2 and ||R(1:k,:)||_F^2 in FP64
  __syncthreads();
  if (warp == 0) {
    double a = 0.0, b = 0.0;
    for (int e = lane; e < l * l; e += 32) {
      const int i = e / l, jj = e % l;
      if (jj < i) continue;
      const double r = (jj == i) ? (double)rdiag[i] : (double)Ds[pcol[jj] * LD + i];
      a += r * r;
      if (i < k) b += r * r;
    }
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) {
      if (fro2) { fro2[0] = a; fro2[1] = b; }
      if (status) { status->fro2_T = a; status->fro2_Tk = b; }
    }
  }
}

template <typename TC>
cudaError_t launch_qrcp(const double* D, int64_t ldd, int l, int k, double* Q, int64_t ldq, double* R, int64_t ldr,
                        bool r_transposed, int32_t* perm, double* fro2, DevStatus* status, cudaStream_t st) {
  const size_t smem = (size_t)2 * l * (l + 1) * sizeof(TC);
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
