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
#include "tc_common.cuh"

namespace corutv {

constexpr int kQrcpTPC = 4;   // threads per column of the register QRCP (512 threads)
// its dynamic shared memory: the l reflectors (rows skewed by 4 per RPT-row piece), later
// the l x (l + 1) staging tile of the outputs
constexpr size_t kQrcpSmem = (size_t)kMaxL * (kMaxL + 4 * kQrcpTPC) * sizeof(float);

// =============================================================================== Gram
// parts[c] = X[:, cols_c] Y[:, cols_c]^T over the c-th contiguous column range.
// 512 threads, thread (tx, ty) (32 x 16) owns rows a = R ty + (0..R-1) and
// columns b = C tx + (0..C-1) (R = LP/16, C = LP/32).  Stages of BK columns
// are kept k-major in shared memory (rows padded by 4); the next stage's
// global loads (16-byte vectors where the rows allow) are issued into
// registers before the current stage is used.
template <typename TC, int LP>
__device__ __forceinline__ void gram_partial_body(const TC* __restrict__ Xt, int64_t ldx, const TC* __restrict__ Yt,
                                                  int64_t ldy, int64_t len, int l, TC* __restrict__ parts, int cta,
                                                  int ncta) {
  constexpr int R = LP / 16, CC = LP / 32;
  constexpr int BK = 32;
  constexpr int LPP = LP + 4;
  constexpr int VW = (sizeof(TC) == 4 && LP * BK / 4 >= 512) ? 4 : 1;   // elements per load
  constexpr int PER = LP * BK / VW / 512;                              // loads of X (and of Y) per thread
  __shared__ __align__(16) TC Xs[BK][LPP];
  __shared__ __align__(16) TC Ys[BK][LPP];
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int64_t chunk = cdiv(cdiv(len, BK), ncta) * BK;
  const int64_t c0 = cta * chunk;
  int64_t c1 = c0 + chunk;
  if (c1 > len) c1 = len;
  const bool vec = VW == 4 && (ldx & 3) == 0 && (ldy & 3) == 0 && ((uintptr_t)Xt & 15) == 0 &&
                   ((uintptr_t)Yt & 15) == 0;
  TC acc[R][CC];
#pragma unroll
  for (int v = 0; v < R; ++v)
#pragma unroll
    for (int u = 0; u < CC; ++u) acc[v][u] = TC(0);
  TC px[PER][VW], py[PER][VW];
  auto fetch = [&](int64_t k0) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int x = tid + 512 * q;
      const int r = x / (BK / VW), kk = VW * (x % (BK / VW));
      const int64_t g = k0 + kk;
      const TC* xs = Xt + r * ldx + g;
      const TC* ys = Yt + r * ldy + g;
      if constexpr (VW == 4) {
        if (vec && r < l && g + 3 < c1) {
          const float4 a4 = *reinterpret_cast<const float4*>(xs);
          const float4 b4 = *reinterpret_cast<const float4*>(ys);
          px[q][0] = a4.x; px[q][1] = a4.y; px[q][2] = a4.z; px[q][3] = a4.w;
          py[q][0] = b4.x; py[q][1] = b4.y; py[q][2] = b4.z; py[q][3] = b4.w;
          continue;
        }
      }
#pragma unroll
      for (int u = 0; u < VW; ++u) {
        const bool ok = r < l && g + u < c1;
        px[q][u] = ok ? xs[u] : TC(0);
        py[q][u] = ok ? ys[u] : TC(0);
      }
    }
  };
  if (c0 < c1) fetch(c0);
  for (int64_t k0 = c0; k0 < c1; k0 += BK) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int x = tid + 512 * q;
      const int r = x / (BK / VW), kk = VW * (x % (BK / VW));
#pragma unroll
      for (int u = 0; u < VW; ++u) {
        Xs[kk + u][r] = px[q][u];
        Ys[kk + u][r] = py[q][u];
      }
    }
    __syncthreads();
    if (k0 + BK < c1) fetch(k0 + BK);
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      TC xa[R], yb[CC];
      if constexpr (sizeof(TC) == 4 && R % 4 == 0 && CC % 4 == 0) {
#pragma unroll
        for (int v = 0; v < R; v += 4) {
          const float4 t = *reinterpret_cast<const float4*>(&Xs[kk][R * ty + v]);
          xa[v] = t.x; xa[v + 1] = t.y; xa[v + 2] = t.z; xa[v + 3] = t.w;
        }
#pragma unroll
        for (int u = 0; u < CC; u += 4) {
          const float4 t = *reinterpret_cast<const float4*>(&Ys[kk][CC * tx + u]);
          yb[u] = t.x; yb[u + 1] = t.y; yb[u + 2] = t.z; yb[u + 3] = t.w;
        }
      } else {
#pragma unroll
        for (int v = 0; v < R; ++v) xa[v] = Xs[kk][R * ty + v];
#pragma unroll
        for (int u = 0; u < CC; ++u) yb[u] = Ys[kk][CC * tx + u];
      }
#pragma unroll
      for (int v = 0; v < R; ++v)
#pragma unroll
        for (int u = 0; u < CC; ++u) acc[v][u] = fma(xa[v], yb[u], acc[v][u]);
    }
    __syncthreads();
  }
  TC* out = parts + (int64_t)cta * LP * LP;
#pragma unroll
  for (int v = 0; v < R; ++v)
#pragma unroll
    for (int u = 0; u < CC; ++u) out[(R * ty + v) * LP + CC * tx + u] = acc[v][u];
}

template <typename TC, int LP>
__global__ void __launch_bounds__(512) gram_partial_kernel(const TC* __restrict__ Xt, int64_t ldx,
                                                           const TC* __restrict__ Yt, int64_t ldy, int64_t len,
                                                           int l, TC* __restrict__ parts) {
  pdl_enter();
  gram_partial_body<TC, LP>(Xt, ldx, Yt, ldy, len, l, parts, blockIdx.x, gridDim.x);
}

// Error-free sum of two FP32 numbers (Knuth's TwoSum): s = fl(a + b), a + b = s + e exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}

// G[a][b] = sum over parts in a fixed order.  A CTA of 256 threads takes 32
// consecutive elements e = a l + b (one per lane, so every load of a warp is one
// coalesced row segment); warp w sums parts w, w + 8, w + 16, ... with all its
// loads issued before the first add, and lane 0..31 of warp 0 then adds the
// eight warp sums in warp order.  FP64 sketches: FP64 sums.  FP32 sketches:
// compensated FP32 sums (TwoSum, the rounding errors carried in a second word),
// as accurate as an FP64 sum of these few hundred terms at the FP32 rate
// (GB300's FP64 pipe is ~1/64 of it); the output is the rounded pair, in TG.
template <typename TC, typename TG>
__device__ __forceinline__ void gram_reduce_body(const TC* __restrict__ parts, int nparts, int LP, int l,
                                                 TG* __restrict__ G, int64_t ldg, int blk) {
  __shared__ TC red_s[kRedWarps][32], red_c[kRedWarps][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int e = blk * 32 + lane;
  const bool ok = e < l * l;
  const int a = ok ? e / l : 0, b = ok ? e % l : 0;
  const TC* src = parts + (int64_t)a * LP + b;
  const int64_t stride = (int64_t)LP * LP;
  constexpr int U = 8;                       // loads in flight per thread
  TC s = TC(0), c = TC(0);
  for (int p0 = w; p0 < nparts; p0 += kRedWarps * U) {
    TC v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int p = p0 + kRedWarps * u;
      v[u] = (ok && p < nparts) ? src[p * stride] : TC(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if constexpr (sizeof(TC) == 8) {
        s += v[u];
      } else {
        float t, er;
        two_sum(s, v[u], t, er);
        s = t;
        c += er;
      }
    }
  }
  red_s[w][lane] = s;
  red_c[w][lane] = c;
  __syncthreads();
  if (w == 0 && ok) {
    if constexpr (sizeof(TC) == 8) {
      double t = red_s[0][lane];
      for (int k = 1; k < kRedWarps; ++k) t += red_s[k][lane];
      G[a * ldg + b] = (TG)t;
    } else {
      float t = red_s[0][lane], tc = red_c[0][lane];
      for (int k = 1; k < kRedWarps; ++k) {
        float u, er;
        two_sum(t, red_s[k][lane], u, er);
        t = u;
        tc += red_c[k][lane] + er;
      }
      if constexpr (sizeof(TG) == 8) G[a * ldg + b] = (double)t + (double)tc;
      else G[a * ldg + b] = t + tc;
    }
  }
}

template <typename TC, typename TG>
__global__ void __launch_bounds__(kRedWarps * 32) gram_reduce_kernel(const TC* __restrict__ parts, int nparts, int LP,
                                                                      int l, TG* __restrict__ G, int64_t ldg) {
  pdl_enter();
  gram_reduce_body<TC, TG>(parts, nparts, LP, l, G, ldg, blockIdx.x);
}

int gram_parts(int64_t len, int sms) {
  int64_t p = cdiv(len, 32);
  if (p > sms) p = sms;
  return (int)(p < 1 ? 1 : p);
}

template <typename TC, typename TG>
cudaError_t launch_gram(const TC* Xt, int64_t ldx, const TC* Yt, int64_t ldy, int64_t len, int l, TC* parts,
                        int gparts, TG* G, int64_t ldg, cudaStream_t st) {
  int LP;
  if (l <= 32) {
    LP = 32;
    CU_RET(launch_pdl(gram_partial_kernel<TC, 32>, gparts, 512, 0, st, Xt, ldx, Yt, ldy, len, l, parts));
    CORUTV_COUNT_LAUNCH();
  } else if (l <= 64) {
    LP = 64;
    CU_RET(launch_pdl(gram_partial_kernel<TC, 64>, gparts, 512, 0, st, Xt, ldx, Yt, ldy, len, l, parts));
    CORUTV_COUNT_LAUNCH();
  } else {
    LP = 128;
    CU_RET(launch_pdl(gram_partial_kernel<TC, 128>, gparts, 512, 0, st, Xt, ldx, Yt, ldy, len, l, parts));
    CORUTV_COUNT_LAUNCH();
  }
  CU_RET(launch_pdl(gram_reduce_kernel<TC, TG>, (unsigned)cdiv((int64_t)l * l, 32), kRedWarps * 32, 0, st, parts,
                    gparts, LP, l, G, ldg));
  CORUTV_COUNT_LAUNCH();
  return cudaSuccess;
}

template <typename TC, typename TG>
cudaError_t launch_gram_auto(const TC* Xt, int64_t ldx, const TC* Yt, int64_t ldy, int64_t len, int l, TC* parts,
                             int sms, DevStatus* status, TG* G, int64_t ldg, cudaStream_t st, bool allow_tc) {
  if constexpr (sizeof(TC) == 4) {
    if (allow_tc && gram_tc_ok(Xt, ldx, Yt, ldy, l)) {
      cudaError_t e = launch_gram_tc_partials(Xt, ldx, Yt, ldy, len, l, parts, sms, status, st);
      if (e != cudaSuccess) return e;
      CU_RET(launch_pdl(gram_reduce_kernel<TC, TG>, (unsigned)cdiv((int64_t)l * l, 32), kRedWarps * 32, 0, st,
                        parts, gram_tc_parts(len, sms), 128, l, G, ldg));
      CORUTV_COUNT_LAUNCH();
      return cudaSuccess;
    }
  }
  return launch_gram<TC, TG>(Xt, ldx, Yt, ldy, len, l, parts, gram_parts(len, sms), G, ldg, st);
}

// =============================================================================== Cholesky
// G + s I = R^T R (R upper, s = shift_rel * trace(G)) and R^-1, by symmetric
// elimination of [G | I] in FP64: step j subtracts m_a = G[j][a] / G[j][j] times
// row j from every row a > j (upper triangle of G only, by symmetry; the right
// block receives the same row operations).  Afterwards G = L D L^T with the
// pivots d_j = G[j][j] (as of step j), the upper triangle holding D L^T and the
// right block holding L^-1, so R = D^(1/2) L^T and R^-1[p][j] = L^-1[j][p] /
// sqrt(d_j).  Every update of a step is independent: one block barrier per step,
// no long dependent chains.  A pivot d <= tol_rel * (G_jj + s) marks column j
// dependent: it eliminates nothing, R[j][j] = 1, R[j][>j] = 0, defic[j] = 1 (the
// caller replaces that column of Q).
// One l x (l + 1) FP64 array in shared memory holds both triangles: G on and above
// the diagonal, L^-1 strictly below it (its unit diagonal implicit), so l = 128
// needs 132 KB.  R and R^-1 are written in TO: FP64 for FP64 sketches, FP32 for
// FP32 sketches whose small factorisations run in FP64.
template <typename TO>
__global__ void __launch_bounds__(512) cholinv_kernel(const double* __restrict__ G, int64_t ldg, int l,
                                                      double shift_rel, double tol_rel, TO* __restrict__ Rg,
                                                      TO* __restrict__ Rinvg, int* __restrict__ defic,
                                                      DevStatus* status, double* __restrict__ Rout) {
  extern __shared__ unsigned char smem_raw[];
  const int LD = l + 1;
  double* S = reinterpret_cast<double*>(smem_raw);   // l x LD: G (b >= a), L^-1 (b < a)
  __shared__ double diag0[kMaxL];
  __shared__ double piv[kMaxL];
  __shared__ int dep_s[kMaxL];
  __shared__ double red[32];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;

  double tr = 0.0;
  for (int e = tid; e < l * l; e += nt) {
    const int a = e / l, b = e % l;
    const double g = G[a * ldg + b];
    S[a * LD + b] = (b >= a) ? g : 0.0;
    if (a == b) tr += g;
  }
  for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
  if (lane == 0) red[warp] = tr;
  __syncthreads();
  double trace = 0.0;
  for (int w = 0; w < nw; ++w) trace += red[w];
  const double shift = shift_rel * trace;
  for (int a = tid; a < l; a += nt) {
    const double d = S[a * LD + a] + shift;
    S[a * LD + a] = d;
    diag0[a] = d;
  }
  __syncthreads();

  for (int j = 0; j < l; ++j) {
    const double d = S[j * LD + j];
    const bool dep = !(d > tol_rel * diag0[j]) || !(diag0[j] > 0.0);
    const double inv_d = dep ? 0.0 : 1.0 / d;
    if (tid == 0) {
      piv[j] = dep ? 1.0 : d;
      dep_s[j] = dep ? 1 : 0;
    }
    // rows a > j, one warp per row: the upper triangle b >= a of G, and L^-1 columns b <= j
    // (L^-1[j][j] = 1 is implicit; L^-1[j][b < j] sits below the diagonal of row j)
    for (int a = j + 1 + warp; a < l; a += nw) {
      const double m = S[j * LD + a] * inv_d;
      for (int b = a + lane; b < l; b += 32) S[a * LD + b] -= m * S[j * LD + b];
      for (int b = lane; b <= j; b += 32) S[a * LD + b] -= m * (b == j ? 1.0 : S[j * LD + b]);
    }
    __syncthreads();
  }
  int nfall = 0;
  for (int e = tid; e < l * l; e += nt) {
    const int a = e / l, b = e % l;
    const double ra = sqrt(piv[a]);
    double r = 0.0;
    if (b == a) r = ra;
    else if (b > a && !dep_s[a]) r = S[a * LD + b] / ra;
    Rg[a * kMaxL + b] = (TO)r;
    // R^-1[a][b] = L^-1[b][a] / sqrt(d_b)  (upper: a <= b)
    const double lib = (b == a) ? 1.0 : (b > a ? S[b * LD + a] : 0.0);
    Rinvg[a * kMaxL + b] = (TO)(lib / sqrt(piv[b]));
    if (Rout) Rout[a * l + b] = r;
  }
  for (int a = tid; a < l; a += nt) {
    defic[a] = dep_s[a];
    nfall += dep_s[a];
  }
  for (int o = 16; o > 0; o >>= 1) nfall += __shfl_xor_sync(0xffffffffu, nfall, o);
  if (lane == 0 && nfall && status) atomicAdd(&status->chol_fallbacks, nfall);
}

// FP32 variant, blocked: G + s I = L L^T by a right-looking Cholesky over
// 32 x 32 diagonal blocks, then R = L^T and R^-1 = L^-T.  Per block column k:
//   (a) one warp factors the diagonal block (lane i holds row i in registers,
//       column j broadcast by shuffles) and forms its inverse X_kk = L_kk^-1;
//   (b) the panel below it becomes L_ik = A_ik X_kk^T;
//   (c) the trailing lower blocks take A_ij -= L_ik L_jk^T.
// The off-diagonal blocks of L^-1 follow by block distance d = i - j:
// X_ij = -X_ii (sum_{p=j}^{i-1} L_ip X_pj).  About 20 block barriers at l = 128
// instead of one per column.  A pivot d <= tol_rel * (G_jj + s) marks column j
// dependent: L[j][j] = 1 and the rest of column j is zero, so it eliminates
// nothing, R[j][j] = 1, R[j][>j] = 0, defic[j] = 1 (the caller replaces that
// column of Q).  The matrix is padded to 32 * ceil(l / 32) with the identity.
// Reciprocal and reciprocal square root for the latency-bound one-CTA kernels:
// the hardware approximation (MUFU) refined by one Newton-Raphson step,
// y <- y (2 - x y) for 1 / x and r <- r (3 - x r^2) / 2 for 1 / sqrt(x), which
// roughly doubles the correct bits (about 1 ulp after the step).  Inputs below
// the smallest normal number take the IEEE path (the approximations flush
// them).  The IEEE operators are not used on the common path: they branch to
// a subroutine that costs hundreds of cycles per call in a large kernel.
__device__ __forceinline__ float rcp_nr(float x) {
  if (!(fabsf(x) >= 1.17549435e-38f)) return 1.f / x;
  const float y = __fdividef(1.f, x);
  return y * fmaf(-x, y, 2.f);
}
__device__ __forceinline__ float rsqrt_nr(float x) {
  if (!(x >= 1.17549435e-38f)) return 1.f / sqrtf(x);
  const float r = rsqrtf(x);
  return r * fmaf(-0.5f * x * r, r, 1.5f);
}
// 1 / pivot in the elimination loop: the MUFU approximation and one Newton step, as rcp_nr but
// without its branch for subnormal inputs (the branch cost ~25% of a step).  A pivot that
// reaches the reciprocal is positive (above tol times a positive diagonal entry); one below the
// smallest normal number is raised to it, so the result stays finite.
__device__ __forceinline__ float rcp_pivot(float x) {
  const float xs = fmaxf(x, 1.17549435e-38f);
  const float y = __fdividef(1.f, xs);
  return y * fmaf(-xs, y, 2.f);
}

// FP32 variant with the matrices in registers: the same elimination of
// [G + s I | I] as cholinv_kernel, with the upper triangle of G and the lower
// triangle of L^-1 split into 4 x 4 blocks.  Thread t owns block (I, J), J >= I,
// of G and block (J, I) of L^-1 (t enumerates the upper block triangle column
// by column).  Step j reads row j of G and of L^-1 from a double-buffered shared
// row (published by the owners of row j), applies its multipliers
// m_a = G[j][a] / d_j to the rows a > j of both blocks; steps go in pairs with
// one block barrier per pair (see the loop).  Reciprocals and
// square roots come from rcp_nr / rsqrt_nr, and the input is the FP32 Gram
// matrix (no FP64 arithmetic: GB300's FP64 pipe would dominate the step).
__device__ __forceinline__ float f4(const float4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

constexpr int kPipeMaxThreads = (kMaxL / 4) * (kMaxL / 4 + 1) / 2 + 16;   // 528 blocks -> 544 threads

// skip_flag (may be null): the kernel first measures max |G - I| over the l x l
// block; at or below skip_tol it writes 1 to *skip_flag, R_out = I (if asked)
// and returns (the caller's Q already has orthonormal columns to that level),
// otherwise it writes 0 and factors as usual.
__device__ __forceinline__ void cholinv_pipe_body(const float* __restrict__ G, int64_t ldg, int l, double shift_rel,
                                                  double tol_rel, float* __restrict__ Rg, float* __restrict__ Rinvg,
                                                  int64_t ldr, int* __restrict__ defic, DevStatus* status,
                                                  double* __restrict__ Rout, int* __restrict__ skip_flag,
                                                  float skip_tol) {
  __shared__ __align__(16) float rowbuf[2][2][kMaxL];   // [pair parity][row j / j + 1]
  __shared__ __align__(16) float libuf[2][2][kMaxL];
  __shared__ float diag0[kMaxL];
  __shared__ float piv[kMaxL];
  __shared__ float pivrs[kMaxL];     // 1 / sqrt(piv)
  __shared__ int dep_s[kMaxL];
  __shared__ float red[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int nb = (l + 3) >> 2;
  const bool own = tid < nb * (nb + 1) / 2;
  // blocks enumerated column by column (t = J (J + 1) / 2 + I): a thread has nothing left
  // to do once j >= 4 J + 3, and the threads of a warp reach that point together
  int I = 0, J = 0;
  if (own) {
    int jj = 0;
    while ((jj + 1) * (jj + 2) / 2 <= tid) ++jj;
    J = jj;
    I = tid - jj * (jj + 1) / 2;
  }
  __shared__ float redmax[32];
  float g[4][4], li[4][4];
  float tr = 0.f, dev = 0.f;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int a = 4 * I + r, b = 4 * J + c;
      const bool in = own && a < l && b < l;
      g[r][c] = in ? G[a * ldg + b] : 0.f;
      if (in) dev = fmaxf(dev, fabsf(g[r][c] - (a == b ? 1.f : 0.f)));
      li[r][c] = (4 * J + r == 4 * I + c) ? 1.f : 0.f;
    }
  if (own && I == J) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (4 * I + r < l) tr += g[r][r];
  }
  for (int e = tid; e < 4 * kMaxL; e += blockDim.x) (&libuf[0][0][0])[e] = 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tr += __shfl_xor_sync(0xffffffffu, tr, o);
    dev = fmaxf(dev, __shfl_xor_sync(0xffffffffu, dev, o));
  }
  if (lane == 0) {
    red[warp] = tr;
    redmax[warp] = dev;
  }
  __syncthreads();
  float trace = 0.f, devmax = 0.f;
  for (int w = 0; w < nw; ++w) {
    trace += red[w];
    devmax = fmaxf(devmax, redmax[w]);
  }
  if (skip_flag) {
    const bool skip = devmax <= skip_tol;
    if (tid == 0) *skip_flag = skip ? 1 : 0;
    if (skip) {
      if (Rout)
        for (int e = tid; e < l * l; e += blockDim.x) Rout[e] = (e / l == e % l) ? 1.0 : 0.0;
      return;
    }
  }
  const float shift = (float)shift_rel * trace;
  const float tolf = (float)tol_rel;
  if (own) {
    if (I == J) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int a = 4 * I + r;
        if (a < l) {
          g[r][r] += shift;
          diag0[a] = g[r][r];
        }
      }
    }
    // rows 0 and 1 of G and of L^-1
    if (I == 0) {
      *reinterpret_cast<float4*>(&rowbuf[0][0][4 * J]) = make_float4(g[0][0], g[0][1], g[0][2], g[0][3]);
      *reinterpret_cast<float4*>(&rowbuf[0][1][4 * J]) = make_float4(g[1][0], g[1][1], g[1][2], g[1][3]);
    }
    if (J == 0) {
      *reinterpret_cast<float4*>(&libuf[0][0][4 * I]) = make_float4(li[0][0], li[0][1], li[0][2], li[0][3]);
      *reinterpret_cast<float4*>(&libuf[0][1][4 * I]) = make_float4(li[1][0], li[1][1], li[1][2], li[1][3]);
    }
  }
  __syncthreads();

  // Two elimination steps per barrier: step pair (j, j + 1) reads rows j and j + 1 as of
  // step j - 1; every thread forms the part of row j + 1 after step j that it needs itself
  // (row_{j+1} - m row_j, m = G[j][j+1] / d_j), so the owners publish rows j + 2 and j + 3
  // once per pair.
  for (int j = 0; j < l; j += 2) {
    const int pb = (j >> 1) & 1;
    const bool two = j + 1 < l;
    const float dj = rowbuf[pb][0][j];
    const float d0j = diag0[j];
    const bool depj = !(dj > tolf * d0j) || !(d0j > 0.f);
    const float invj = depj ? 0.f : rcp_pivot(dj);
    // row j + 1 after step j: its multiplier, pivot and dependence
    const float m1 = two ? rowbuf[pb][0][j + 1] * invj : 0.f;
    const float dk = two ? fmaf(-m1, rowbuf[pb][0][j + 1], rowbuf[pb][1][j + 1]) : 1.f;
    const float d0k = two ? diag0[j + 1] : 1.f;
    const bool depk = !(dk > tolf * d0k) || !(d0k > 0.f);
    const float invk = (depk || !two) ? 0.f : rcp_pivot(dk);
    if (tid == 0) {
      piv[j] = depj ? 1.f : dj;
      pivrs[j] = depj ? 1.f : rsqrt_nr(dj);
      dep_s[j] = depj ? 1 : 0;
      if (two) {
        piv[j + 1] = depk ? 1.f : dk;
        pivrs[j + 1] = depk ? 1.f : rsqrt_nr(dk);
        dep_s[j + 1] = depk ? 1 : 0;
      }
    }
    if (own && 4 * J + 3 > j) {
      const float4 rI0 = *reinterpret_cast<const float4*>(&rowbuf[pb][0][4 * I]);
      const float4 rJ0 = *reinterpret_cast<const float4*>(&rowbuf[pb][0][4 * J]);
      const float4 lI0 = *reinterpret_cast<const float4*>(&libuf[pb][0][4 * I]);
      float4 rI1 = *reinterpret_cast<const float4*>(&rowbuf[pb][1][4 * I]);
      float4 rJ1 = *reinterpret_cast<const float4*>(&rowbuf[pb][1][4 * J]);
      float4 lI1 = *reinterpret_cast<const float4*>(&libuf[pb][1][4 * I]);
      // step j
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float mi = (4 * I + r > j) ? f4(rI0, r) * invj : 0.f;   // rows of the G block
        const float mj = (4 * J + r > j) ? f4(rJ0, r) * invj : 0.f;   // rows of the L^-1 block
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          g[r][c] = fmaf(-mi, f4(rJ0, c), g[r][c]);
          li[r][c] = fmaf(-mj, f4(lI0, c), li[r][c]);
        }
      }
      // step j + 1 with row j + 1 as of step j (invk = 0 when there is no step j + 1)
      rI1 = make_float4(fmaf(-m1, rI0.x, rI1.x), fmaf(-m1, rI0.y, rI1.y), fmaf(-m1, rI0.z, rI1.z),
                        fmaf(-m1, rI0.w, rI1.w));
      rJ1 = make_float4(fmaf(-m1, rJ0.x, rJ1.x), fmaf(-m1, rJ0.y, rJ1.y), fmaf(-m1, rJ0.z, rJ1.z),
                        fmaf(-m1, rJ0.w, rJ1.w));
      lI1 = make_float4(fmaf(-m1, lI0.x, lI1.x), fmaf(-m1, lI0.y, lI1.y), fmaf(-m1, lI0.z, lI1.z),
                        fmaf(-m1, lI0.w, lI1.w));
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float mi = (4 * I + r > j + 1) ? f4(rI1, r) * invk : 0.f;
        const float mj = (4 * J + r > j + 1) ? f4(rJ1, r) * invk : 0.f;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          g[r][c] = fmaf(-mi, f4(rJ1, c), g[r][c]);
          li[r][c] = fmaf(-mj, f4(lI1, c), li[r][c]);
        }
      }
      // publish rows j + 2 and j + 3 (the same block row; register rows 0, 1 or 2, 3)
      const int p = j + 2;
      if (p < l) {
        const int qb = pb ^ 1, hi = (p & 3) >> 1;
        if (I == (p >> 2)) {
          const float4 a0 = hi ? make_float4(g[2][0], g[2][1], g[2][2], g[2][3])
                               : make_float4(g[0][0], g[0][1], g[0][2], g[0][3]);
          const float4 a1 = hi ? make_float4(g[3][0], g[3][1], g[3][2], g[3][3])
                               : make_float4(g[1][0], g[1][1], g[1][2], g[1][3]);
          *reinterpret_cast<float4*>(&rowbuf[qb][0][4 * J]) = a0;
          *reinterpret_cast<float4*>(&rowbuf[qb][1][4 * J]) = a1;
        }
        if (J == (p >> 2)) {
          const float4 b0 = hi ? make_float4(li[2][0], li[2][1], li[2][2], li[2][3])
                               : make_float4(li[0][0], li[0][1], li[0][2], li[0][3]);
          const float4 b1 = hi ? make_float4(li[3][0], li[3][1], li[3][2], li[3][3])
                               : make_float4(li[1][0], li[1][1], li[1][2], li[1][3]);
          *reinterpret_cast<float4*>(&libuf[qb][0][4 * I]) = b0;
          *reinterpret_cast<float4*>(&libuf[qb][1][4 * I]) = b1;
        }
      }
    }
    __syncthreads();
  }
  // outputs: R = D^(1/2) L^T (upper; rows of dependent columns e_j^T), R^-1[a][b] = L^-1[b][a] / sqrt(d_b)
  if (own) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int a = 4 * I + r, b = 4 * J + c;
        if (a >= l || b >= l) continue;
        float rv = 0.f, xv = 0.f;
        if (b == a) rv = piv[a] * pivrs[a];
        else if (b > a && !dep_s[a]) rv = g[r][c] * pivrs[a];
        if (b >= a) xv = li[c][r] * pivrs[b];
        Rg[a * ldr + b] = rv;
        Rinvg[a * ldr + b] = xv;
        if (Rout) Rout[a * l + b] = (double)rv;
        if (b > a) {            // the mirrored lower entries
          Rg[b * ldr + a] = 0.f;
          Rinvg[b * ldr + a] = 0.f;
          if (Rout) Rout[b * l + a] = 0.0;
        }
      }
  }
  int nfall = 0;
  for (int a = tid; a < l; a += blockDim.x) {
    defic[a] = dep_s[a];
    nfall += dep_s[a];
  }
  for (int o = 16; o > 0; o >>= 1) nfall += __shfl_xor_sync(0xffffffffu, nfall, o);
  if (lane == 0 && nfall && status) atomicAdd(&status->chol_fallbacks, nfall);
}

__global__ void __launch_bounds__(kPipeMaxThreads, 1) cholinv_pipe_kernel(
    const float* __restrict__ G, int64_t ldg, int l, double shift_rel, double tol_rel, float* __restrict__ Rg,
    float* __restrict__ Rinvg, int* __restrict__ defic, DevStatus* status, double* __restrict__ Rout,
    int* __restrict__ skip_flag, float skip_tol) {
  pdl_enter();
  cholinv_pipe_body(G, ldg, l, shift_rel, tol_rel, Rg, Rinvg, kMaxL, defic, status, Rout, skip_flag, skip_tol);
}

// Shared-memory limits are raised once per kernel and device (before any stream
// capture records the launches).
constexpr int kAttrDevices = 64;
static bool* attr_flag(bool (&flags)[kAttrDevices]) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kAttrDevices) return nullptr;
  return &flags[dev];
}

template <typename K>
static cudaError_t raise_smem_once(K kernel, size_t bytes, bool (&flags)[kAttrDevices]) {
  bool* flag = attr_flag(flags);
  if (flag && *flag) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && flag) *flag = true;
  return e;
}

template <typename TC>
cudaError_t launch_cholinv(const TC* G, int64_t ldg, int l, double shift_rel, double tol_rel, TC* R, TC* Rinv,
                           int* defic, DevStatus* status, double* Rout, int* skip_flag, float skip_tol,
                           cudaStream_t st) {
  if constexpr (sizeof(TC) == 4) {
    const int nb = (l + 3) / 4;
    const int threads = (nb * (nb + 1) / 2 + 31) / 32 * 32;
    CU_RET(launch_pdl(cholinv_pipe_kernel, 1, threads, 0, st, G, ldg, l, shift_rel, tol_rel, R, Rinv, defic, status,
                      Rout, skip_flag, skip_tol));
    CORUTV_COUNT_LAUNCH();
    return cudaSuccess;
  } else {
    return launch_cholinv_f64<double>(G, ldg, l, shift_rel, tol_rel, R, Rinv, defic, status, Rout, st);
  }
}

template <typename TO>
cudaError_t launch_cholinv_f64(const double* G, int64_t ldg, int l, double shift_rel, double tol_rel, TO* R,
                               TO* Rinv, int* defic, DevStatus* status, double* Rout, cudaStream_t st) {
  const size_t smem = (size_t)l * (l + 1) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(cholinv_kernel<TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cholinv_kernel<TO><<<1, 512, smem, st>>>(G, ldg, l, shift_rel, tol_rel, R, Rinv, defic, status, Rout);
  CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}
template cudaError_t launch_cholinv_f64<float>(const double*, int64_t, int, double, double, float*, float*, int*,
                                               DevStatus*, double*, cudaStream_t);
template cudaError_t launch_cholinv_f64<double>(const double*, int64_t, int, double, double, double*, double*, int*,
                                                DevStatus*, double*, cudaStream_t);

// Dependent columns: row j of an ST block (column j of Q) flagged dependent is
// replaced by a deterministic pseudo-random vector (SplitMix64 of (pass, j, i),
// uniform in [-1, 1)); the next CholeskyQR pass orthonormalises it against the
// others.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double replacement_value(int pass, int j, int64_t i) {
  const uint64_t h =
      mix64(0x5EEDull + ((uint64_t)pass << 48) + ((uint64_t)j << 32) + (uint64_t)i * 0x9E3779B97F4A7C15ull);
  return 2.0 * ((double)(h >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

// =============================================================================== lmul
// Out[j][i] = sum_{p<l} S[p][j] In[p][i]   (Out = S^T In on ST blocks, i.e. C S in
// the untransposed view).  S (LP x LP) is staged in shared memory once per CTA;
// the CTA then takes BI-column tiles of In in turn (a persistent loop over
// tiles: the grid is sized to the resident CTAs, so no partial second wave).
// Thread (tx, ty) owns rows j = R ty + (0..R-1) and columns i = BI/16 tx +
// (0..BI/16-1) of the tile.  upper: S is upper triangular (S[p][j] = 0 for
// p > j), so the p loop stops at the last row of the thread's warp.  The tile
// is read completely before it is written, so In == Out (in place) is allowed.
// defic (may be null): rows j with defic[j] != 0 receive the replacement vector
// of `pass` instead of the product.  out_rowmajor: write Out^T into a
// row-major len x l matrix (staged through shared memory so the row writes
// coalesce).  round_out (FP32, may be null): also write the rows rounded to TF32.
template <typename TC, int LP, int BI>
__host__ __device__ constexpr size_t lmul_smem_bytes() {
  return ((size_t)LP * (LP + 4) + (size_t)(LP * (BI + 4) > BI * (LP + 1) ? LP * (BI + 4) : BI * (LP + 1))) *
         sizeof(TC);
}

// S (l x l, ld lds, type TS) -> Ss (LP x (LP + 4), zero outside l x l)
template <typename TC, typename TS, int LP>
__device__ __forceinline__ void lmul_stage_S(const TS* __restrict__ S, int64_t lds, int l, TC* __restrict__ Ss) {
  constexpr int SP = LP + 4;
  const int tid = threadIdx.x;
  if constexpr (sizeof(TS) == 4 && sizeof(TC) == 4) {
    constexpr int N4 = LP * LP / 4 / 256;
    float4 v[N4];
    const bool s_vec = (lds & 3) == 0 && ((uintptr_t)S & 15) == 0;
#pragma unroll
    for (int q = 0; q < N4; ++q) {
      const int e = tid + 256 * q, p = e / (LP / 4), j = 4 * (e % (LP / 4));
      float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
      if (p < l) {
        const TS* src = S + p * lds + j;
        if (j + 3 < l && s_vec) {
          t = *reinterpret_cast<const float4*>(src);
        } else {
          if (j < l) t.x = src[0];
          if (j + 1 < l) t.y = src[1];
          if (j + 2 < l) t.z = src[2];
          if (j + 3 < l) t.w = src[3];
        }
      }
      v[q] = t;
    }
#pragma unroll
    for (int q = 0; q < N4; ++q) {
      const int e = tid + 256 * q, p = e / (LP / 4), j = 4 * (e % (LP / 4));
      *reinterpret_cast<float4*>(reinterpret_cast<float*>(Ss) + p * SP + j) = v[q];
    }
  } else {
    for (int e = tid; e < LP * LP; e += 256) {
      const int p = e / LP, j = e % LP;
      Ss[p * SP + j] = (p < l && j < l) ? (TC)S[p * lds + j] : TC(0);
    }
  }
}

// one BI-column tile (index bx) with S already staged in Ss; Is: LP x (BI + 4).  SKIP_PAD: warps
// whose rows are all at or beyond l skip the product (the grouped launches, where LP is a class
// width above the problem's l)
template <typename TC, int LP, int BI, bool SKIP_PAD = false>
__device__ __forceinline__ void lmul_tile(const TC* __restrict__ In, int64_t ldi, int64_t len, int l,
                                          const TC* __restrict__ Ss, TC* __restrict__ Is, TC* __restrict__ Out,
                                          int64_t ldo, int out_rowmajor, int upper, const int* __restrict__ defic,
                                          int pass, int64_t bx, float* __restrict__ round_out, int64_t ldr) {
  constexpr int R = LP / 16, RI = BI / 16;
  constexpr int SP = LP + 4, IP = BI + 4;
  constexpr bool kVecIn = sizeof(TC) == 4 && (LP * BI / 4) % 256 == 0;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = bx * BI;
  if constexpr (kVecIn) {
    constexpr int N4 = LP * BI / 4 / 256;
    float4 v[N4];
    const bool vec_ok = (ldi & 3) == 0 && ((uintptr_t)In & 15) == 0;
#pragma unroll
    for (int q = 0; q < N4; ++q) {
      const int e = tid + 256 * q, p = e / (BI / 4), ii = 4 * (e % (BI / 4));
      const int64_t g = i0 + ii;
      float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
      if (p < l) {
        const TC* src = In + p * ldi + g;
        if (vec_ok && g + 3 < len) {
          t = *reinterpret_cast<const float4*>(src);
        } else {
          if (g < len) t.x = src[0];
          if (g + 1 < len) t.y = src[1];
          if (g + 2 < len) t.z = src[2];
          if (g + 3 < len) t.w = src[3];
        }
      }
      v[q] = t;
    }
#pragma unroll
    for (int q = 0; q < N4; ++q) {
      const int e = tid + 256 * q, p = e / (BI / 4), ii = 4 * (e % (BI / 4));
      *reinterpret_cast<float4*>(reinterpret_cast<float*>(Is) + p * IP + ii) = v[q];
    }
  } else {
    for (int e = tid; e < LP * BI; e += 256) {
      const int p = e / BI, ii = e % BI;
      const int64_t g = i0 + ii;
      Is[p * IP + ii] = (p < l && g < len) ? In[p * ldi + g] : TC(0);
    }
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
  if (SKIP_PAD && R * (ty & ~1) >= l) pend = 0;   // all rows of the warp are padding (j >= l)
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
      const bool repl = defic && defic[j];
#pragma unroll
      for (int u = 0; u < RI; ++u) {
        const int64_t g = i0 + RI * tx + u;
        if (g < len) {
          const TC val = repl ? (TC)replacement_value(pass, j, g) : acc[v][u];
          Out[j * ldo + g] = val;
          if constexpr (sizeof(TC) == 4)
            if (round_out) round_out[j * ldr + g] = to_tf32(val);   // the next pass's TF32 operand
        }
      }
    }
    __syncthreads();                              // Is is refilled by the next tile
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
    __syncthreads();
  }
}

// one CTA per block index bx (the grouped launches: one tile each)
template <typename TC, typename TS, int LP, int BI>
__device__ __forceinline__ void lmul_body(const TC* __restrict__ In, int64_t ldi, int64_t len, int l,
                                          const TS* __restrict__ S, int64_t lds, TC* __restrict__ Out, int64_t ldo,
                                          int out_rowmajor, int upper, const int* __restrict__ defic, int pass,
                                          int bx, float* __restrict__ round_out = nullptr, int64_t ldr = 0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC* Ss = reinterpret_cast<TC*>(smem_raw);
  TC* Is = Ss + LP * (LP + 4);
  lmul_stage_S<TC, TS, LP>(S, lds, l, Ss);
  lmul_tile<TC, LP, BI, true>(In, ldi, len, l, Ss, Is, Out, ldo, out_rowmajor, upper, defic, pass, bx, round_out,
                              ldr);
}

template <typename TC, typename TS, int LP, int BI>
__global__ void __launch_bounds__(256, 2) lmul_kernel(const TC* __restrict__ In, int64_t ldi, int64_t len, int l,
                                                      const TS* __restrict__ S, int64_t lds, TC* __restrict__ Out,
                                                      int64_t ldo, int out_rowmajor, int upper,
                                                      const int* __restrict__ defic, int pass,
                                                      const int* __restrict__ skip_flag, float* __restrict__ round_out,
                                                      int64_t ldr) {
  pdl_enter();
  const int64_t tiles = cdiv(len, BI);
  if (skip_flag && *skip_flag) {           // the factor was found to be the identity: Out = In
    if constexpr (sizeof(TC) == 4) {
      if (round_out) {
        for (int64_t bx = blockIdx.x; bx < tiles; bx += gridDim.x) {
          const int64_t i0 = bx * BI;
          for (int e = threadIdx.x; e < l * BI; e += blockDim.x) {
            const int j = e / BI;
            const int64_t g = i0 + e % BI;
            if (g < len) round_out[j * ldr + g] = to_tf32(In[j * ldi + g]);
          }
        }
      }
    }
    return;
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC* Ss = reinterpret_cast<TC*>(smem_raw);
  TC* Is = Ss + LP * (LP + 4);
  lmul_stage_S<TC, TS, LP>(S, lds, l, Ss);
  for (int64_t bx = blockIdx.x; bx < tiles; bx += gridDim.x)
    lmul_tile<TC, LP, BI>(In, ldi, len, l, Ss, Is, Out, ldo, out_rowmajor, upper, defic, pass, bx, round_out, ldr);
}

template <typename TC, typename TS, int LP, int BI>
static cudaError_t lmul_variant(const TC* In, int64_t ldi, int64_t len, int l, const TS* S, int64_t lds, TC* Out,
                                int64_t ldo, bool rowmajor, bool upper, const int* defic, int pass,
                                const int* skip_flag, float* round_out, int64_t ldr, cudaStream_t st) {
  const int64_t tiles = cdiv(len, BI);
  if (tiles == 0) return cudaSuccess;
  constexpr size_t sm = lmul_smem_bytes<TC, LP, BI>();
  static bool attr_set[kAttrDevices] = {};
  static int resident[kAttrDevices] = {};
  bool* flag = attr_flag(attr_set);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (!flag || !*flag) {
    e = cudaFuncSetAttribute(lmul_kernel<TC, TS, LP, BI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lmul_kernel<TC, TS, LP, BI>, 256, sm);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (dev < kAttrDevices) resident[dev] = (per_sm < 1 ? 1 : per_sm) * sms;
    if (flag) *flag = true;
  }
  const int cap = (dev < kAttrDevices && resident[dev] > 0) ? resident[dev] : 148;
  const unsigned grid = (unsigned)(tiles < cap ? tiles : cap);
  CU_RET(launch_pdl(lmul_kernel<TC, TS, LP, BI>, grid, 256, sm, st, In, ldi, len, l, S, lds, Out, ldo,
                    rowmajor ? 1 : 0, upper ? 1 : 0, defic, pass, skip_flag, round_out, ldr));
  CORUTV_COUNT_LAUNCH();
  return cudaSuccess;
}

template <typename TC, typename TS>
static cudaError_t lmul_dispatch(const TC* In, int64_t ldi, int64_t len, int l, const TS* S, int64_t lds, TC* Out,
                                 int64_t ldo, bool rowmajor, bool upper, const int* defic, int pass,
                                 const int* skip_flag, float* round_out, int64_t ldr, cudaStream_t st) {
  // FP32: 32-column tiles (S and the tile in ~86 KB of shared memory: two CTAs per SM, and fine
  // enough that the last round of tiles leaves few SMs idle); FP64: 32 columns
  constexpr int BI = 32;
  if (l <= 32)
    return lmul_variant<TC, TS, 32, BI>(In, ldi, len, l, S, lds, Out, ldo, rowmajor, upper, defic, pass, skip_flag,
                                        round_out, ldr, st);
  if (l <= 64)
    return lmul_variant<TC, TS, 64, BI>(In, ldi, len, l, S, lds, Out, ldo, rowmajor, upper, defic, pass, skip_flag,
                                        round_out, ldr, st);
  return lmul_variant<TC, TS, 128, BI>(In, ldi, len, l, S, lds, Out, ldo, rowmajor, upper, defic, pass, skip_flag,
                                       round_out, ldr, st);
}

template <typename TC>
cudaError_t launch_lmul(const TC* In, int64_t ldi, int64_t len, int l, const TC* S, int64_t lds, TC* Out,
                        int64_t ldo, bool out_rowmajor, const int* defic, int pass, const int* skip_flag,
                        float* round_out, int64_t ldr, cudaStream_t st) {
  // the CholeskyQR factor R^-1 is upper triangular
  return lmul_dispatch<TC, TC>(In, ldi, len, l, S, lds, Out, ldo, out_rowmajor, true, defic, pass, skip_flag,
                               round_out, ldr, st);
}
template <typename TC>
cudaError_t launch_lmul_full(const TC* In, int64_t ldi, int64_t len, int l, const TC* S, int64_t lds, TC* Out,
                             int64_t ldo, bool out_rowmajor, cudaStream_t st) {
  return lmul_dispatch<TC, TC>(In, ldi, len, l, S, lds, Out, ldo, out_rowmajor, false, nullptr, 0, nullptr, nullptr,
                               0, st);
}

cudaError_t launch_lmul_full_f64s(const float* In, int64_t ldi, int64_t len, int l, const double* S, int64_t lds,
                                  float* Out, int64_t ldo, bool out_rowmajor, cudaStream_t st) {
  return lmul_dispatch<float, double>(In, ldi, len, l, S, lds, Out, ldo, out_rowmajor, false, nullptr, 0, nullptr,
                                      nullptr, 0, st);
}

// =============================================================================== R composition
// C = A B for upper-triangular A, B (l x l, FP64, ld l): C[i][j] = sum_{k=i..j} A[i][k] B[k][j].
__global__ void upper_mul_kernel(const double* __restrict__ A, const double* __restrict__ B,
                                 double* __restrict__ C, int l) {
  const int i = blockIdx.x;
  for (int j = threadIdx.x; j < l; j += blockDim.x) {
    double s = 0.0;
    for (int k = i; k <= j; ++k) s = fma(A[i * l + k], B[k * l + j], s);
    C[i * l + j] = s;
  }
}

cudaError_t launch_upper_mul(const double* A, const double* B, double* C, int l, cudaStream_t st) {
  upper_mul_kernel<<<l, 128, 0, st>>>(A, B, C, l);
  CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

// =============================================================================== gather / stage
// Out[i][j] = St[perm[j]][i]  (row-major len x l output from an ST block).
template <typename TC>
__device__ __forceinline__ void gather_cols_body(const TC* __restrict__ St, int64_t lds, int64_t len, int l,
                                                 const int32_t* __restrict__ perm, TC* __restrict__ Out, int64_t ldo,
                                                 int bx) {
  __shared__ TC tile[kMaxL][33];
  __shared__ int pm[kMaxL];
  const int64_t i0 = (int64_t)bx * 32;
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
__global__ void gather_cols_kernel(const TC* __restrict__ St, int64_t lds, int64_t len, int l,
                                   const int32_t* __restrict__ perm, TC* __restrict__ Out, int64_t ldo) {
  gather_cols_body<TC>(St, lds, len, l, perm, Out, ldo, blockIdx.x);
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
__device__ __forceinline__ void stage_transpose_body(const TC* __restrict__ Phi, int64_t ldphi, int64_t len, int l,
                                                     TC* __restrict__ Xt, int64_t ldx, int bx,
                                                     float* __restrict__ round_out = nullptr, int64_t ldr = 0) {
  __shared__ TC tile[32][kMaxL + 1];
  const int64_t i0 = (int64_t)bx * 32;
  for (int e = threadIdx.x; e < 32 * l; e += blockDim.x) {
    const int ii = e / l, j = e % l;
    const int64_t g = i0 + ii;
    tile[ii][j] = g < len ? Phi[g * ldphi + j] : TC(0);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < l * 32; e += blockDim.x) {
    const int j = e / 32, ii = e % 32;
    const int64_t g = i0 + ii;
    if (g < len) {
      Xt[j * ldx + g] = tile[ii][j];
      if constexpr (sizeof(TC) == 4)
        if (round_out) round_out[j * ldr + g] = to_tf32(tile[ii][j]);
    }
  }
}

template <typename TC>
__global__ void stage_transpose_kernel(const TC* __restrict__ Phi, int64_t ldphi, int64_t len, int l,
                                       TC* __restrict__ Xt, int64_t ldx, float* __restrict__ round_out, int64_t ldr) {
  stage_transpose_body<TC>(Phi, ldphi, len, l, Xt, ldx, blockIdx.x, round_out, ldr);
}

template <typename TC>
cudaError_t launch_stage_transpose(const TC* Phi, int64_t ldphi, int64_t len, int l, TC* Xt, int64_t ldx,
                                   float* round_out, int64_t ldr, cudaStream_t st) {
  const unsigned grid = (unsigned)cdiv(len, 32);
  if (grid) {
    stage_transpose_kernel<TC><<<grid, 256, 0, st>>>(Phi, ldphi, len, l, Xt, ldx, round_out, ldr);
    CORUTV_COUNT_LAUNCH();
  }
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
// i = RPT h .. RPT h + RPT - 1 of column c of D and of M = H_j ... H_0 (TPC
// threads per column), so every column reduction is a per-thread sum plus
// TPC - 1 shuffles.  Step j: warp 0 reduces the sixteen warp candidates (each
// warp's trailing column of largest exact trailing norm, lowest current
// position on ties) to the pivot; the pivot column's warp builds the reflector
// and publishes it; every trailing column (and every column of M) takes it,
// recomputes its trailing norm exactly and its warp forms the next candidate.
// Three block barriers per step: the pivot choice and the reflector are each
// formed once, which costs less than forming them in every warp.  Every column
// tracks its own position (the pivot moves to j, the column at j to the
// pivot's old place), so the choices are those of the textbook algorithm with
// physical column exchanges.  The reflector and pivot column are stored with a
// skew (row i at i + 4 (i / RPT)) so the TPC threads of a column read them
// without shared-memory bank conflicts.
// LQ: the capacity (rows and columns, l <= LQ); the grouped launches size it by l's class.
// PIVOT = false: the unpivoted Householder QR (step j takes the column at position j), the
// second factorisation of the QLP.  d_transposed: the input is D^T (Dg read column-wise).
// tk_by_col: the rank-k readout sums the squares of the first k columns of R (the first k
// rows of the output R^T) instead of its first k rows.
template <int TPC, typename TD, typename TQ, bool PIVOT = true, int LQ = kMaxL>
__device__ __forceinline__ void qrcp_reg_body(const TD* __restrict__ Dg, int64_t ldd, int l, int k,
                                              TQ* __restrict__ Qg, int64_t ldq, double* __restrict__ Rg,
                                              int64_t ldr, int r_transposed, int32_t* __restrict__ perm,
                                              double* __restrict__ fro2, DevStatus* status, int d_transposed = 0,
                                              int tk_by_col = 0) {
  constexpr int RPT = LQ / TPC, NWARP = LQ * TPC / 32, CPW = 32 / TPC;   // columns per warp
  static_assert(RPT % 4 == 0 && NWARP <= 32 && LQ <= kMaxL, "qrcp capacity");
  // row i of the reflector and of the pivot column lives at i + 4 (i / RPT): the RPT-row
  // pieces that the TPC threads of a column read start in different banks
  constexpr int SKW = LQ + 4 * TPC;
  extern __shared__ __align__(16) unsigned char qrcp_smem[];
  float* Vs = reinterpret_cast<float*>(qrcp_smem);   // reflector of step j in row j (zero outside j..l-1)
  __shared__ __align__(16) float pcolv[SKW];         // raw pivot column
  __shared__ float betas[LQ];
  auto sk = [](int i) { return i + 4 * (i / RPT); };
  __shared__ float cnrm[NWARP];                      // each warp's candidate: trailing norm^2 (-1: none),
  __shared__ int cpos[NWARP], ccol[NWARP];           // its current position and its column
  __shared__ int piv[3];                             // pivot column, -, its position before the swap
  __shared__ float rdiag[LQ];
  __shared__ int pcol[LQ];
  __shared__ double red[NWARP][2];
  const int tid = threadIdx.x, c = tid / TPC, h = tid % TPC, lane = tid & 31, warp = tid >> 5;
  const int i0 = RPT * h;
  float d[RPT];               // column c of D (rows i0..)
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int i = i0 + r;
    d[r] = (c < l && i < l) ? (float)Dg[d_transposed ? c * ldd + i : i * ldd + c] : 0.f;
  }
  int mypos = c;
  bool trailing = c < l;
  int posof = -1;
  // the warp's candidate for the next pivot: its trailing column of largest norm, lowest position on ties
  auto publish = [&](float nrm2) {
    float bn = trailing ? nrm2 : -1.f;
    int bp = trailing ? mypos : 0x7fffffff, bc = c;
#pragma unroll
    for (int o = TPC; o < 32; o <<= 1) {
      const float on = __shfl_xor_sync(0xffffffffu, bn, o);
      const int op = __shfl_xor_sync(0xffffffffu, bp, o);
      const int oc = __shfl_xor_sync(0xffffffffu, bc, o);
      if (on > bn || (on == bn && op < bp)) { bn = on; bp = op; bc = oc; }
    }
    if (lane == 0) { cnrm[warp] = bn; cpos[warp] = bp; ccol[warp] = bc; }
  };
  {
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int r = 0; r < RPT; r += 2) { s0 = fmaf(d[r], d[r], s0); s1 = fmaf(d[r + 1], d[r + 1], s1); }
    float ss = s0 + s1;
#pragma unroll
    for (int o = 1; o < TPC; o <<= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if constexpr (PIVOT) publish(ss);
  }
  __syncthreads();
  for (int j = 0; j < l; ++j) {
    // ---- phase 1: warp 0 reduces the warps' candidates to the pivot (first maximum by current
    // position); the column at position j takes the pivot's old position
    if (PIVOT && warp == 0) {
      float bn = (lane < NWARP) ? cnrm[lane] : -1.f;
      int bp = (lane < NWARP) ? cpos[lane] : 0x7fffffff;
      int bc = (lane < NWARP) ? ccol[lane] : 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float on = __shfl_xor_sync(0xffffffffu, bn, o);
        const int op = __shfl_xor_sync(0xffffffffu, bp, o);
        const int oc = __shfl_xor_sync(0xffffffffu, bc, o);
        if (on > bn || (on == bn && op < bp)) { bn = on; bp = op; bc = oc; }
      }
      if (lane == 0) { piv[0] = bc; piv[2] = bp; }
    }
    if constexpr (PIVOT) __syncthreads();
    const int cp = PIVOT ? piv[0] : j;
    if (c == cp) mypos = j;
    else if (mypos == j) mypos = piv[2];
    // ---- phase 2: the pivot column's warp builds the reflector from a shared copy of the column
    if (warp == cp / CPW) {
      if (c == cp) {
        float4* p4 = reinterpret_cast<float4*>(pcolv + sk(i0));
#pragma unroll
        for (int q = 0; q < RPT / 4; ++q) p4[q] = make_float4(d[4 * q], d[4 * q + 1], d[4 * q + 2], d[4 * q + 3]);
        trailing = false;
        posof = j;
      }
      __syncwarp();
      const bool rl = 4 * lane < LQ;               // the lane's rows 4 lane .. 4 lane + 3 exist
      const float4 x4 = rl ? *reinterpret_cast<const float4*>(pcolv + sk(4 * lane)) : make_float4(0.f, 0.f, 0.f, 0.f);
      float xv[4] = {x4.x, x4.y, x4.z, x4.w};
      float ss = 0.f;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = 4 * lane + e;
        if (i >= j && i < l) ss = fmaf(xv[e], xv[e], ss);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      const float x0 = pcolv[sk(j)];
      const float nrm = (ss > 0.f) ? ss * rsqrt_nr(ss) : 0.f;
      float alpha, v0, beta;
      if (nrm == 0.f) {
        alpha = 0.f; v0 = 1.f; beta = 0.f;
      } else {
        alpha = (x0 >= 0.f) ? -nrm : nrm;
        v0 = x0 - alpha;
        beta = rcp_nr(nrm * (nrm + fabsf(x0)));
      }
      float4 vo;
      float* vp = &vo.x;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = 4 * lane + e;
        vp[e] = (i == j) ? v0 : ((i > j && i < l) ? xv[e] : 0.f);
      }
      if (rl) *reinterpret_cast<float4*>(Vs + j * SKW + sk(4 * lane)) = vo;
      if (lane == 0) { betas[j] = beta; rdiag[j] = alpha; pcol[j] = cp; }
    }
    __syncthreads();
    // ---- phase 3: every trailing column of D takes the reflector
    {
      float v[RPT];
      const float4* v4 = reinterpret_cast<const float4*>(Vs + j * SKW + sk(i0));
#pragma unroll
      for (int q = 0; q < RPT / 4; ++q) {
        const float4 t = v4[q];
        v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
      }
      const float beta = betas[j];
      float wd0 = 0.f, wd1 = 0.f;
#pragma unroll
      for (int r = 0; r < RPT; r += 2) {
        wd0 = fmaf(v[r], d[r], wd0);
        wd1 = fmaf(v[r + 1], d[r + 1], wd1);
      }
      float wd = trailing ? wd0 + wd1 : 0.f;
#pragma unroll
      for (int o = 1; o < TPC; o <<= 1) wd += __shfl_xor_sync(0xffffffffu, wd, o);   // within the column's group
      const float fd = beta * wd;
      float s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        d[r] = fmaf(-fd, v[r], d[r]);          // fd = 0 for columns that are not trailing
        const float x = (i0 + r > j) ? d[r] : 0.f;
        if (r & 1) s1 = fmaf(x, x, s1); else s0 = fmaf(x, x, s0);
      }
      float ns = s0 + s1;
#pragma unroll
      for (int o = 1; o < TPC; o <<= 1) ns += __shfl_xor_sync(0xffffffffu, ns, o);   // within the column's group
      publish(ns);
    }
    __syncthreads();
  }
  // Q~ = H_0 H_1 ... H_{l-1}, column by column: column c is H_0 (... (H_c e_c)) (the reflectors
  // H_i with i > c leave e_c unchanged: v_i is zero above row i).  Every thread runs the same
  // count (its warp's last column), so the shuffles stay warp-wide; for i > c the product
  // v_i^T q is exactly zero.  No barriers: the reflectors are read-only now.
  float q[RPT];
#pragma unroll
  for (int r = 0; r < RPT; ++r) q[r] = (i0 + r == c) ? 1.f : 0.f;
  {
    int imax = (warp + 1) * (32 / TPC) - 1;
    if (imax > l - 1) imax = l - 1;
    for (int i = imax; i >= 0; --i) {
      float v[RPT];
      const float4* v4 = reinterpret_cast<const float4*>(Vs + i * SKW + sk(i0));
#pragma unroll
      for (int qq = 0; qq < RPT / 4; ++qq) {
        const float4 t = v4[qq];
        v[4 * qq] = t.x; v[4 * qq + 1] = t.y; v[4 * qq + 2] = t.z; v[4 * qq + 3] = t.w;
      }
      float w0 = 0.f, w1 = 0.f;
#pragma unroll
      for (int r = 0; r < RPT; r += 2) {
        w0 = fmaf(v[r], q[r], w0);
        w1 = fmaf(v[r + 1], q[r + 1], w1);
      }
      float w = w0 + w1;
#pragma unroll
      for (int o = 1; o < TPC; o <<= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
      const float f = betas[i] * w;
#pragma unroll
      for (int r = 0; r < RPT; ++r) q[r] = fmaf(-f, v[r], q[r]);
    }
  }
  __syncthreads();                             // the reflectors' memory becomes the staging tile
  // ||R||_F^2 and ||R(1:k, :)||_F^2 as compensated FP32 sums (exact squares, TwoSum), in FP64
  // across warps; R and Q~ go through a shared tile so that their rows are written whole
  float* St = Vs;                              // l x (l + 1)
  const int SL = l + 1;
  float fa = 0.f, fae = 0.f, fb = 0.f, fbe = 0.f;
  auto acc_sq = [](float v, float& sum, float& err) {
    const float p = v * v;
    float t, e;
    two_sum(sum, p, t, e);
    sum = t;
    err += e + fmaf(v, v, -p);
  };
  // Q~[a][c] with the column sign of diag(R) (diag(R) >= 0)
  if (c < l) {
    const float sgn = rdiag[c] < 0.f ? -1.f : 1.f;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int a = i0 + r;
      if (a < l) St[a * SL + c] = sgn * q[r];
    }
  }
  __syncthreads();
  for (int e = tid; e < l * l; e += blockDim.x) {
    const int a = e / l, b = e - a * l;
    Qg[a * ldq + b] = (TQ)St[a * SL + b];
  }
  __syncthreads();
  // R from each pivot column (rows above its position), diag(R) >= 0
  if (posof >= 0) {
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int i = i0 + r;
      if (i >= l) continue;
      float val;
      if (i < posof) val = (rdiag[i] < 0.f ? -1.f : 1.f) * d[r];
      else if (i == posof) val = fabsf(rdiag[i]);
      else val = 0.f;
      if (r_transposed) St[posof * SL + i] = val;
      else St[i * SL + posof] = val;
      acc_sq(val, fa, fae);
      if ((tk_by_col ? posof : i) < k) acc_sq(val, fb, fbe);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const float oa = __shfl_xor_sync(0xffffffffu, fa, o), oae = __shfl_xor_sync(0xffffffffu, fae, o);
    const float ob = __shfl_xor_sync(0xffffffffu, fb, o), obe = __shfl_xor_sync(0xffffffffu, fbe, o);
    const bool lo = (lane & o) == 0;      // lower lane first: every lane forms the same sums
    float t, e;
    two_sum(lo ? fa : oa, lo ? oa : fa, t, e);
    fa = t;
    fae = (lo ? fae + oae : oae + fae) + e;
    two_sum(lo ? fb : ob, lo ? ob : fb, t, e);
    fb = t;
    fbe = (lo ? fbe + obe : obe + fbe) + e;
  }
  if (lane == 0) {
    red[warp][0] = (double)fa + (double)fae;
    red[warp][1] = (double)fb + (double)fbe;
  }
  for (int jj = tid; jj < l; jj += blockDim.x) perm[jj] = pcol[jj];
  __syncthreads();
  for (int e = tid; e < l * l; e += blockDim.x) {
    const int a = e / l, b = e - a * l;
    Rg[a * ldr + b] = (double)St[a * SL + b];
  }
  if (tid == 0) {
    double a2 = 0.0, b2 = 0.0;
    for (int w2 = 0; w2 < NWARP; ++w2) { a2 += red[w2][0]; b2 += red[w2][1]; }
    if (fro2) { fro2[0] = a2; fro2[1] = b2; }
    if (status) { status->fro2_T = a2; status->fro2_Tk = b2; }
  }
}

template <int TPC, typename TD, typename TQ, bool PIVOT = true>
__global__ void __launch_bounds__(kMaxL * TPC) qrcp_reg_kernel(const TD* __restrict__ Dg, int64_t ldd, int l, int k,
                                                       TQ* __restrict__ Qg, int64_t ldq, double* __restrict__ Rg,
                                                       int64_t ldr, int r_transposed, int32_t* __restrict__ perm,
                                                       double* __restrict__ fro2, DevStatus* status,
                                                       int d_transposed, int tk_by_col) {
  qrcp_reg_body<TPC, TD, TQ, PIVOT>(Dg, ldd, l, k, Qg, ldq, Rg, ldr, r_transposed, perm, fro2, status, d_transposed,
                                    tk_by_col);
}

template <typename TC>
cudaError_t launch_qrcp(const TC* D, int64_t ldd, int l, int k, TC* Q, int64_t ldq, double* R, int64_t ldr,
                        bool r_transposed, int32_t* perm, double* fro2, DevStatus* status, cudaStream_t st) {
  if constexpr (sizeof(TC) == 4) {
    static bool attr_set[kAttrDevices] = {};
    cudaError_t e = raise_smem_once(qrcp_reg_kernel<kQrcpTPC, float, float>, kQrcpSmem, attr_set);
    if (e != cudaSuccess) return e;
    qrcp_reg_kernel<kQrcpTPC, float, float><<<1, kMaxL * kQrcpTPC, kQrcpSmem, st>>>(D, ldd, l, k, Q, ldq, R, ldr,
                                                                                    r_transposed ? 1 : 0, perm, fro2,
                                                                                    status, 0, 0);
    CORUTV_COUNT_LAUNCH();
    return cudaGetLastError();
  } else {
    const size_t smem = (size_t)l * kMaxL * sizeof(TC);
    cudaError_t e = cudaFuncSetAttribute(qrcp_kernel<TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    qrcp_kernel<TC><<<1, 512, smem, st>>>(D, ldd, l, k, Q, ldq, R, ldr, r_transposed ? 1 : 0, perm, fro2, status);
    CORUTV_COUNT_LAUNCH();
    return cudaGetLastError();
  }
}

// Second half of the QLP of the core: an unpivoted QR of R~^T, R~^T = Qh Rh.  R (FP64,
// l x l, ld ldr) holds R~ on entry and receives L = Rh^T (to_lower, the URV side) or Rh
// (the ULV side); Qh (FP32, l x l, ld l).  status->fro2_T / fro2_Tk are refreshed
// (||L||_F^2 = ||R~||_F^2; the rank-k part is L(1:k, 1:k)).
cudaError_t launch_qlp_second(double* R, int64_t ldr, int l, int k, float* Qh, bool to_lower, int32_t* perm_scratch,
                              DevStatus* status, cudaStream_t st) {
  static bool attr_set[kAttrDevices] = {};
  cudaError_t e = raise_smem_once(qrcp_reg_kernel<kQrcpTPC, double, float, false>, kQrcpSmem, attr_set);
  if (e != cudaSuccess) return e;
  qrcp_reg_kernel<kQrcpTPC, double, float, false><<<1, kMaxL * kQrcpTPC, kQrcpSmem, st>>>(
      R, ldr, l, k, Qh, l, R, ldr, to_lower ? 1 : 0, perm_scratch, nullptr, status, 1, to_lower ? 1 : 0);
  CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

// S = P~ Qh: S[perm[j]][c] = Qh[j][c] (l x l, ld l)
__global__ void perm_rows_kernel(const float* __restrict__ Qh, const int32_t* __restrict__ perm, int l,
                                 float* __restrict__ S) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < l * l; e += gridDim.x * blockDim.x) {
    const int j = e / l, c = e % l;
    S[perm[j] * l + c] = Qh[j * l + c];
  }
}

cudaError_t launch_perm_rows(const float* Qh, const int32_t* perm, int l, float* S, cudaStream_t st) {
  perm_rows_kernel<<<(l * l + 255) / 256, 256, 0, st>>>(Qh, perm, l, S);
  CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

template <typename TC>
cudaError_t launch_qrcp_f64io(const double* D, int64_t ldd, int l, int k, double* Q, int64_t ldq, double* R,
                              int64_t ldr, int32_t* perm, double* fro2, cudaStream_t st) {
  if constexpr (sizeof(TC) == 4) {
    static bool attr_set[kAttrDevices] = {};
    cudaError_t e = raise_smem_once(qrcp_reg_kernel<kQrcpTPC, double, double>, kQrcpSmem, attr_set);
    if (e != cudaSuccess) return e;
    qrcp_reg_kernel<kQrcpTPC, double, double><<<1, kMaxL * kQrcpTPC, kQrcpSmem, st>>>(D, ldd, l, k, Q, ldq, R, ldr, 0,
                                                                                      perm, fro2, nullptr, 0, 0);
    CORUTV_COUNT_LAUNCH();
    return cudaGetLastError();
  } else {
    return launch_qrcp<double>(D, ldd, l, k, Q, ldq, R, ldr, false, perm, fro2, nullptr, st);
  }
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

// dst[a][t] += src[a][t] for a < l, t < len: sums the row-chunk products A_c^T Y_c of a pass
// over a host-streamed A (ST blocks, one CTA row per sketch column)
template <typename TC>
__global__ void add_st_kernel(const TC* __restrict__ src, int64_t lds, int64_t len, TC* __restrict__ dst,
                              int64_t ldd) {
  const int64_t a = blockIdx.y;
  const TC* s = src + a * lds;
  TC* d = dst + a * ldd;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < len; t += (int64_t)gridDim.x * blockDim.x)
    d[t] += s[t];
}

template <typename TC>
cudaError_t launch_add_st(const TC* src, int64_t lds, int l, int64_t len, TC* dst, int64_t ldd, cudaStream_t st) {
  const int64_t bx = cdiv(len, 256) < 32 ? cdiv(len, 256) : 32;
  add_st_kernel<TC><<<dim3((unsigned)bx, (unsigned)l), 256, 0, st>>>(src, lds, len, dst, ldd);
  CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}
template cudaError_t launch_add_st<float>(const float*, int64_t, int, int64_t, float*, int64_t, cudaStream_t);
template cudaError_t launch_add_st<double>(const double*, int64_t, int, int64_t, double*, int64_t, cudaStream_t);

// Sum of n FP64 partials by one warp in a fixed order: lane t adds parts t, t + 32, ... in
// turn, then the 32 lane sums meet in a fixed shuffle tree (the same bits on every run).
__global__ void sum_parts_kernel(const double* __restrict__ parts, int n, double* out, DevStatus* status) {
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  double s = 0.0;
  for (int i = lane; i < n; i += 32) s += parts[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) {
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

// =============================================================================== batched (grouped) launches
// Each grouped kernel runs the single-problem body for the problem a block map
// assigns to its block (FP32 storage of the sketches).  A problem takes part in
// an orthonormalisation pass while it is within its power steps and the pass
// index is below its CholeskyQR pass count (3 for the last step or ORTH_STRICT,
// else 1).
__device__ __forceinline__ bool batch_orth_active(const BatchProb& P, int it, int pass) {
  if (it > P.q) return false;
  const int passes = (it == P.q || P.orth == 1) ? 3 : 1;
  return pass < passes;
}

__global__ void __launch_bounds__(256) stage_grouped_kernel(const BatchProb* __restrict__ probs,
                                                            const int2* __restrict__ map) {
  const int2 pm = map[blockIdx.x];
  const BatchProb& P = probs[pm.x];
  stage_transpose_body<float>(P.Phi, P.ldphi, P.len2, P.l, P.P2, P.ld2, pm.y);
}

// which: kG_ORTH1 (P1 P1^T -> G), kG_ORTH2 (P2 P2^T -> G), kG_CORE_EXACT (P1 P3^T -> D),
// kG_CORE_SKETCH (P3 P2^T -> D: the saved last C2 against Q2)
__device__ __forceinline__ bool batch_gram_sel(const BatchProb& P, int which, int it, int pass, const float** X,
                                               int64_t* ldx, const float** Y, int64_t* ldy, int64_t* len,
                                               float** out) {
  switch (which) {
    case kG_ORTH1:
      if (!batch_orth_active(P, it, pass)) return false;
      *X = P.P1; *ldx = P.ld1; *Y = P.P1; *ldy = P.ld1; *len = P.len1; *out = P.G;
      return true;
    case kG_ORTH2:
      if (!batch_orth_active(P, it, pass)) return false;
      *X = P.P2; *ldx = P.ld2; *Y = P.P2; *ldy = P.ld2; *len = P.len2; *out = P.G;
      return true;
    case kG_CORE_EXACT:
      if (P.core != 0) return false;
      *X = P.P1; *ldx = P.ld1; *Y = P.P3; *ldy = P.ld3; *len = P.len1; *out = P.D;
      return true;
    default:
      if (P.core == 0) return false;
      *X = P.P3; *ldx = P.ld3; *Y = P.P2; *ldy = P.ld2; *len = P.len2; *out = P.D;
      return true;
  }
}

// FP32 Gram partial of one column range for the grouped launches, with register tiles: a
// thread owns a TM x TM tile of the partial (TM = 4 for LP <= 64, 8 for LP = 128), so each k
// costs two or four 16-byte shared loads per 16 or 64 FMAs.  Only the tiles that hold rows and
// columns below the problem's own l are formed (TL = ceil(l / TM) per side), and for X X^T only
// those on or above the diagonal (the rest is their transpose, written as such): the class
// padding of l to LP costs no FMAs.  The active tiles are taken by G groups of threads (G up to
// 8, as many as fit in the block), group g forming the columns k = g mod G of every staged
// block; the group sums are added in group order at the end.  The sums are over this problem's
// own column range only and G depends on l alone, so the result does not depend on the other
// problems of the batch.
template <int LP>
__device__ __forceinline__ void gram_tiles_body(const float* __restrict__ Xt, int64_t ldx,
                                                const float* __restrict__ Yt, int64_t ldy, int64_t len, int l,
                                                float* __restrict__ parts, int cta, int ncta) {
  constexpr int TM = LP == 128 ? 8 : 4;
  constexpr int TS = LP / TM;
  constexpr int kMaxG = 8;
  constexpr int BK = 32, LPP = LP + 4;
  constexpr int PER = LP * BK / 4 / 256;        // 16-byte loads of X (and of Y) per thread per stage
  static_assert(PER >= 1 && PER * 256 * 4 == LP * BK, "gram stage");
  static_assert(2 * BK * LPP >= 128 * TM * TM, "group sums reuse the stage buffers");
  __shared__ __align__(16) float sbuf[2 * BK * LPP];     // X stage, then Y stage
  float (*Xs)[LPP] = reinterpret_cast<float (*)[LPP]>(sbuf);
  float (*Ys)[LPP] = reinterpret_cast<float (*)[LPP]>(sbuf + BK * LPP);
  // stage row kk keeps its 4-float chunks in the order chunk ^ ((kk / 4) mod 8): the transposing
  // stores of a warp (eight k, four rows of A's sketch) then fall in 32 different banks, and a
  // tile's 4 consecutive rows stay one 16-byte vector
  static_assert(LP >= 32 && LPP % 32 == 4, "gram stage swizzle");
  auto sw = [](int kk, int col) { return (((col >> 2) ^ ((kk >> 2) & 7)) << 2) | (col & 3); };
  const int tid = threadIdx.x;
  const int64_t chunk = cdiv(cdiv(len, BK), ncta) * BK;
  const int64_t c0 = cta * chunk;
  int64_t c1 = c0 + chunk;
  if (c1 > len) c1 = len;
  const bool same = Xt == Yt && ldx == ldy;     // X X^T: Y is not staged separately, upper tiles only
  const bool vec = (ldx & 3) == 0 && (ldy & 3) == 0 && ((uintptr_t)Xt & 15) == 0 && ((uintptr_t)Yt & 15) == 0;
  int TL = (l + TM - 1) / TM;
  if (TL > TS) TL = TS;
  const int nact = same ? TL * (TL + 1) / 2 : TL * TL;
  int G = nact > 0 ? 256 / nact : 1;
  if (G > kMaxG) G = kMaxG;
  if (G < 1) G = 1;
  const int g = tid / (nact > 0 ? nact : 1), t = tid - g * (nact > 0 ? nact : 1);
  const bool active = nact > 0 && g < G;
  int ti = 0, tj = 0;
  if (same) {
    int rem = t;
    while (ti < TL && rem >= TL - ti) { rem -= TL - ti; ++ti; }
    tj = ti + rem;
  } else if (TL > 0) {
    ti = t / TL;
    tj = t - ti * TL;
  }
  float acc[TM][TM];
#pragma unroll
  for (int v = 0; v < TM; ++v)
#pragma unroll
    for (int u = 0; u < TM; ++u) acc[v][u] = 0.f;
  float4 px[PER], py[PER];
  auto load4 = [&](const float* base, int64_t ld, int r, int64_t g0) {
    float4 v4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r >= l) return v4;
    const float* src = base + r * ld + g0;
    if (vec && g0 + 3 < c1) return *reinterpret_cast<const float4*>(src);
    if (g0 < c1) v4.x = src[0];
    if (g0 + 1 < c1) v4.y = src[1];
    if (g0 + 2 < c1) v4.z = src[2];
    if (g0 + 3 < c1) v4.w = src[3];
    return v4;
  };
  auto fetch = [&](int64_t k0) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int x = tid + 256 * q, r = x / (BK / 4), kk = 4 * (x % (BK / 4));
      px[q] = load4(Xt, ldx, r, k0 + kk);
      if (!same) py[q] = load4(Yt, ldy, r, k0 + kk);
    }
  };
  if (c0 < c1) fetch(c0);
  for (int64_t k0 = c0; k0 < c1; k0 += BK) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int x = tid + 256 * q, r = x / (BK / 4), kk = 4 * (x % (BK / 4));
      const int rs = sw(kk, r);                  // the same chunk order for rows kk .. kk + 3
      Xs[kk][rs] = px[q].x; Xs[kk + 1][rs] = px[q].y; Xs[kk + 2][rs] = px[q].z; Xs[kk + 3][rs] = px[q].w;
      if (!same) {
        Ys[kk][rs] = py[q].x; Ys[kk + 1][rs] = py[q].y; Ys[kk + 2][rs] = py[q].z; Ys[kk + 3][rs] = py[q].w;
      }
    }
    __syncthreads();
    if (k0 + BK < c1) fetch(k0 + BK);
    const float (*Yv)[LPP] = same ? Xs : Ys;
    if (active) {
#pragma unroll 4
      for (int kk = g; kk < BK; kk += G) {
        float xa[TM], yb[TM];
#pragma unroll
        for (int v = 0; v < TM; v += 4) {
          const float4 a4 = *reinterpret_cast<const float4*>(&Xs[kk][sw(kk, TM * ti + v)]);
          const float4 b4 = *reinterpret_cast<const float4*>(&Yv[kk][sw(kk, TM * tj + v)]);
          xa[v] = a4.x; xa[v + 1] = a4.y; xa[v + 2] = a4.z; xa[v + 3] = a4.w;
          yb[v] = b4.x; yb[v + 1] = b4.y; yb[v + 2] = b4.z; yb[v + 3] = b4.w;
        }
#pragma unroll
        for (int v = 0; v < TM; ++v)
#pragma unroll
          for (int u = 0; u < TM; ++u) acc[v][u] = fmaf(xa[v], yb[u], acc[v][u]);
      }
    }
    __syncthreads();
  }
  if (G > 1) {
    // group sums in group order, through the (now free) stage buffers: nact <= 128 when G > 1
    float* red = sbuf;
#pragma unroll 1
    for (int gg = 1; gg < G; ++gg) {
      if (active && g == gg)
#pragma unroll
        for (int v = 0; v < TM; ++v)
#pragma unroll
          for (int u = 0; u < TM; ++u) red[(t * TM + v) * TM + u] = acc[v][u];
      __syncthreads();
      if (active && g == 0)
#pragma unroll
        for (int v = 0; v < TM; ++v)
#pragma unroll
          for (int u = 0; u < TM; ++u) acc[v][u] += red[(t * TM + v) * TM + u];
      __syncthreads();
    }
  }
  if (active && g == 0) {
    float* out = parts + (int64_t)cta * LP * LP;
#pragma unroll
    for (int v = 0; v < TM; ++v)
#pragma unroll
      for (int u = 0; u < TM; u += 4)
        *reinterpret_cast<float4*>(&out[(TM * ti + v) * LP + TM * tj + u]) =
            make_float4(acc[v][u], acc[v][u + 1], acc[v][u + 2], acc[v][u + 3]);
    if (same && ti != tj)
#pragma unroll
      for (int u = 0; u < TM; ++u)
#pragma unroll
        for (int v = 0; v < TM; v += 4)
          *reinterpret_cast<float4*>(&out[(TM * tj + u) * LP + TM * ti + v]) =
              make_float4(acc[v][u], acc[v + 1][u], acc[v + 2][u], acc[v + 3][u]);
  }
}

template <int LP>
__global__ void __launch_bounds__(256, LP == 128 ? 1 : 3) gram_partial_grouped_kernel(const BatchProb* __restrict__ probs,
                                                                   const int2* __restrict__ map, int which, int it,
                                                                   int pass) {
  const int2 pm = map[blockIdx.x];
  const BatchProb& P = probs[pm.x];
  const float *X, *Y;
  int64_t ldx, ldy, len;
  float* out;
  if (!batch_gram_sel(P, which, it, pass, &X, &ldx, &Y, &ldy, &len, &out)) return;
  const int nparts = (which == kG_ORTH2 || which == kG_CORE_SKETCH) ? P.gp2 : P.gp1;
  gram_tiles_body<LP>(X, ldx, Y, ldy, len, P.l, P.gparts, pm.y, nparts);
}

template <int LP>
__global__ void __launch_bounds__(256) gram_reduce_grouped_kernel(const BatchProb* __restrict__ probs,
                                                                  const int2* __restrict__ map, int which, int it,
                                                                  int pass) {
  const int2 pm = map[blockIdx.x];
  const BatchProb& P = probs[pm.x];
  const float *X, *Y;
  int64_t ldx, ldy, len;
  float* out;
  if (!batch_gram_sel(P, which, it, pass, &X, &ldx, &Y, &ldy, &len, &out)) return;
  const int nparts = (which == kG_ORTH2 || which == kG_CORE_SKETCH) ? P.gp2 : P.gp1;
  gram_reduce_body<float, float>(P.gparts, nparts, LP, P.l, out, P.l, pm.y);
}

__global__ void __launch_bounds__(kPipeMaxThreads, 1) cholinv_grouped_kernel(const BatchProb* __restrict__ probs,
                                                                            int it, int pass, float skip_tol,
                                                                            double shift_rel, double tol_rel) {
  const BatchProb& P = probs[blockIdx.x];
  if (!batch_orth_active(P, it, pass)) return;     // uniform over the block
  int* skip = (pass == 2) ? &P.status->orth_skip : nullptr;
  cholinv_pipe_body(P.G, P.l, P.l, pass == 0 ? shift_rel : 0.0, tol_rel, P.R, P.Rinv, P.l, P.defic, P.status,
                    nullptr, skip, skip_tol);
}

template <int LP>
__global__ void __launch_bounds__(256, LP == 32 ? 8 : (LP == 64 ? 4 : 1)) lmul_orth_grouped_kernel(const BatchProb* __restrict__ probs,
                                                                   const int2* __restrict__ map, int which, int it,
                                                                   int pass) {
  const int2 pm = map[blockIdx.x];
  const BatchProb& P = probs[pm.x];
  if (!batch_orth_active(P, it, pass)) return;
  if (pass == 2 && P.status->orth_skip) return;
  // ORTH1_W: orth(C1)'s factor applied to W in P2 (fused power steps), no column replacement
  const bool w = which == kG_ORTH1_W;
  if (w && !P.fuse) return;
  float* C = which == kG_ORTH1 ? P.P1 : P.P2;
  const int64_t ldc = which == kG_ORTH1 ? P.ld1 : P.ld2;
  const int64_t len = which == kG_ORTH1 ? P.len1 : P.len2;
  lmul_body<float, float, LP, kBatchLmulBI>(C, ldc, len, P.l, P.Rinv, P.l, C, ldc, 0, 1, w ? nullptr : P.defic, pass,
                                            pm.y);
}

// the last C2 of a problem (power step it == q) is kept in P3 for the sketch core
__global__ void __launch_bounds__(256) copy_sketch_grouped_kernel(const BatchProb* __restrict__ probs,
                                                                  const int2* __restrict__ map, int it) {
  const int2 pm = map[blockIdx.x];
  const BatchProb& P = probs[pm.x];
  if (P.core == 0 || it != P.q) return;
  const int64_t i0 = (int64_t)pm.y * kBatchTile32;
  for (int e = threadIdx.x; e < P.l * kBatchTile32; e += blockDim.x) {
    const int j = e / kBatchTile32;
    const int64_t g = i0 + e % kBatchTile32;
    if (g < P.len2) P.P3[j * P.ld3 + g] = P.P2[j * P.ld2 + g];
  }
}

// one problem per block (map: (problem, 0)), the register QRCP sized by the class of l
template <int LQ>
__global__ void __launch_bounds__(LQ * kQrcpTPC) qrcp_grouped_kernel(const BatchProb* __restrict__ probs,
                                                                     const int2* __restrict__ map) {
  const BatchProb& P = probs[map[blockIdx.x].x];
  qrcp_reg_body<kQrcpTPC, float, float, true, LQ>(P.D, P.l, P.l, P.k, P.Qt, P.l, P.T, P.ldt, P.side == 1 ? 1 : 0,
                                                   P.perm, nullptr, P.status);
}

// U = Q1 Q~ (RIGHT; V for LEFT), row-major out
template <int LP>
__global__ void __launch_bounds__(256, LP == 32 ? 6 : (LP == 64 ? 4 : 1)) assemble_lmul_grouped_kernel(const BatchProb* __restrict__ probs,
                                                                       const int2* __restrict__ map) {
  const int2 pm = map[blockIdx.x];
  const BatchProb& P = probs[pm.x];
  float* out = P.side == 1 ? P.V : P.U;
  const int64_t ldo = P.side == 1 ? P.ldv : P.ldu;
  lmul_body<float, float, LP, kBatchLmulBI>(P.P1, P.ld1, P.len1, P.l, P.Qt, P.l, out, ldo, 1, 0, nullptr, 0, pm.y);
}

// V = Q2 P~ (RIGHT; U for LEFT)
__global__ void __launch_bounds__(256) assemble_gather_grouped_kernel(const BatchProb* __restrict__ probs,
                                                                      const int2* __restrict__ map) {
  const int2 pm = map[blockIdx.x];
  const BatchProb& P = probs[pm.x];
  float* out = P.side == 1 ? P.U : P.V;
  const int64_t ldo = P.side == 1 ? P.ldu : P.ldv;
  gather_cols_body<float>(P.P2, P.ld2, P.len2, P.l, P.perm, out, ldo, pm.y);
}

// ||A||_F^2 per problem: its first-pass partials summed in tile order
__global__ void fro2_grouped_kernel(const BatchProb* __restrict__ probs) {
  const BatchProb& P = probs[blockIdx.x];
  if (threadIdx.x != 0) return;
  double s = 0.0;
  if (P.want_fro2)
    for (int i = 0; i < P.nfparts; ++i) s += P.fparts[i];
  P.status->fro2_A = P.want_fro2 ? s : 0.0;
}

cudaError_t launch_stage_grouped(const BatchProb* P, const int2* map32_2, int nblocks, cudaStream_t st) {
  if (nblocks <= 0) return cudaSuccess;
  stage_grouped_kernel<<<nblocks, 256, 0, st>>>(P, map32_2);
  CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t launch_gram_grouped(const BatchProb* P, const int2* map_parts, int nparts, const int2* map_red,
                                int nred, int lp, int which, int it, int pass, cudaStream_t st) {
  if (nparts <= 0 || nred <= 0) return cudaSuccess;
  if (lp <= 32) {
    gram_partial_grouped_kernel<32><<<nparts, 256, 0, st>>>(P, map_parts, which, it, pass);
    CORUTV_COUNT_LAUNCH();
    gram_reduce_grouped_kernel<32><<<nred, 256, 0, st>>>(P, map_red, which, it, pass);
  } else if (lp <= 64) {
    gram_partial_grouped_kernel<64><<<nparts, 256, 0, st>>>(P, map_parts, which, it, pass);
    CORUTV_COUNT_LAUNCH();
    gram_reduce_grouped_kernel<64><<<nred, 256, 0, st>>>(P, map_red, which, it, pass);
  } else {
    gram_partial_grouped_kernel<128><<<nparts, 256, 0, st>>>(P, map_parts, which, it, pass);
    CORUTV_COUNT_LAUNCH();
    gram_reduce_grouped_kernel<128><<<nred, 256, 0, st>>>(P, map_red, which, it, pass);
  }
  CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t launch_cholinv_grouped(const BatchProb* P, int count, int lmax, int which, int it, int pass,
                                   float skip_tol, double shift_rel, double tol_rel, cudaStream_t st) {
  (void)which;
  if (count <= 0) return cudaSuccess;
  const int nb = (lmax + 3) / 4;
  const int threads = (nb * (nb + 1) / 2 + 31) / 32 * 32;
  cholinv_grouped_kernel<<<count, threads, 0, st>>>(P, it, pass, skip_tol, shift_rel, tol_rel);
  CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

template <int LP>
static cudaError_t lmul_orth_grouped_lp(const BatchProb* P, const int2* map, int nblocks, int which, int it,
                                        int pass, cudaStream_t st) {
  constexpr size_t sm = lmul_smem_bytes<float, LP, kBatchLmulBI>();
  static bool attr_set[kAttrDevices] = {};
  bool* flag = attr_flag(attr_set);
  if (!flag || !*flag) {
    cudaError_t e = cudaFuncSetAttribute(lmul_orth_grouped_kernel<LP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    if (flag) *flag = true;
  }
  lmul_orth_grouped_kernel<LP><<<nblocks, 256, sm, st>>>(P, map, which, it, pass);
  CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t launch_lmul_orth_grouped(const BatchProb* P, const int2* map, int nblocks, int lp, int which, int it,
                                     int pass, cudaStream_t st) {
  if (nblocks <= 0) return cudaSuccess;
  if (lp <= 32) return lmul_orth_grouped_lp<32>(P, map, nblocks, which, it, pass, st);
  if (lp <= 64) return lmul_orth_grouped_lp<64>(P, map, nblocks, which, it, pass, st);
  return lmul_orth_grouped_lp<128>(P, map, nblocks, which, it, pass, st);
}

cudaError_t launch_copy_sketch_grouped(const BatchProb* P, const int2* map32_2, int nblocks, int it,
                                       cudaStream_t st) {
  if (nblocks <= 0) return cudaSuccess;
  copy_sketch_grouped_kernel<<<nblocks, 256, 0, st>>>(P, map32_2, it);
  CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

template <int LQ>
static cudaError_t qrcp_grouped_lq(const BatchProb* P, const int2* map, int count, cudaStream_t st) {
  constexpr size_t sm = (size_t)LQ * (LQ + 4 * kQrcpTPC) * sizeof(float);
  static bool attr_set[kAttrDevices] = {};
  cudaError_t e = raise_smem_once(qrcp_grouped_kernel<LQ>, sm, attr_set);
  if (e != cudaSuccess) return e;
  qrcp_grouped_kernel<LQ><<<count, LQ * kQrcpTPC, sm, st>>>(P, map);
  CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t launch_qrcp_grouped(const BatchProb* P, const int2* map, int count, int lp, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  if (lp <= 32) return qrcp_grouped_lq<32>(P, map, count, st);
  if (lp <= 64) return qrcp_grouped_lq<64>(P, map, count, st);
  return qrcp_grouped_lq<kMaxL>(P, map, count, st);
}

template <int LP>
static cudaError_t assemble_lp(const BatchProb* P, const int2* map, int nblocks, cudaStream_t st) {
  constexpr size_t sm = lmul_smem_bytes<float, LP, kBatchLmulBI>();
  static bool attr_set[kAttrDevices] = {};
  bool* flag = attr_flag(attr_set);
  if (!flag || !*flag) {
    cudaError_t e = cudaFuncSetAttribute(assemble_lmul_grouped_kernel<LP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if (flag) *flag = true;
  }
  assemble_lmul_grouped_kernel<LP><<<nblocks, 256, sm, st>>>(P, map);
  CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t launch_assemble_grouped(const BatchProb* P, const int2* map_lmul1, int n1, const int2* map32_2, int n2,
                                    int lp, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (n1 > 0) {
    if (lp <= 32) e = assemble_lp<32>(P, map_lmul1, n1, st);
    else if (lp <= 64) e = assemble_lp<64>(P, map_lmul1, n1, st);
    else e = assemble_lp<128>(P, map_lmul1, n1, st);
    if (e != cudaSuccess) return e;
  }
  if (n2 > 0) {
    assemble_gather_grouped_kernel<<<n2, 256, 0, st>>>(P, map32_2);
    CORUTV_COUNT_LAUNCH();
  }
  return cudaGetLastError();
}

cudaError_t launch_fro2_grouped(const BatchProb* P, int count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  fro2_grouped_kernel<<<count, 32, 0, st>>>(P);
  CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ instantiations
#define INST(TC)                                                                                                   \
  template cudaError_t launch_gram<TC, TC>(const TC*, int64_t, const TC*, int64_t, int64_t, int, TC*, int, TC*,     \
                                           int64_t, cudaStream_t);                                                 \
  template cudaError_t launch_cholinv<TC>(const TC*, int64_t, int, double, double, TC*, TC*, int*, DevStatus*,     \
                                          double*, int*, float, cudaStream_t);                                     \
  template cudaError_t launch_lmul<TC>(const TC*, int64_t, int64_t, int, const TC*, int64_t, TC*, int64_t, bool,  \
                                       const int*, int, const int*, float*, int64_t, cudaStream_t);                \
  template cudaError_t launch_lmul_full<TC>(const TC*, int64_t, int64_t, int, const TC*, int64_t, TC*, int64_t,   \
                                            bool, cudaStream_t);                                                   \
  template cudaError_t launch_gather_cols<TC>(const TC*, int64_t, int64_t, int, const int32_t*, TC*, int64_t,     \
                                              cudaStream_t);                                                       \
  template cudaError_t launch_stage_transpose<TC>(const TC*, int64_t, int64_t, int, TC*, int64_t, float*, int64_t, \
                                                  cudaStream_t);                                                  \
  template cudaError_t launch_qrcp<TC>(const TC*, int64_t, int, int, TC*, int64_t, double*, int64_t, bool,         \
                                       int32_t*, double*, DevStatus*, cudaStream_t);                               \
  template cudaError_t launch_qrcp_f64io<TC>(const double*, int64_t, int, int, double*, int64_t, double*, int64_t, \
                                             int32_t*, double*, cudaStream_t);
INST(float)
INST(double)
#undef INST
template cudaError_t launch_gram_auto<float, float>(const float*, int64_t, const float*, int64_t, int64_t, int, float*,
                                                   int, DevStatus*, float*, int64_t, cudaStream_t, bool);
template cudaError_t launch_gram_auto<float, double>(const float*, int64_t, const float*, int64_t, int64_t, int,
                                                    float*, int, DevStatus*, double*, int64_t, cudaStream_t, bool);
template cudaError_t launch_gram_auto<double, double>(const double*, int64_t, const double*, int64_t, int64_t, int,
                                                     double*, int, DevStatus*, double*, int64_t, cudaStream_t,
                                                     bool);
template cudaError_t launch_gram<float, double>(const float*, int64_t, const float*, int64_t, int64_t, int, float*,
                                                 int, double*, int64_t, cudaStream_t);

}  // namespace corutv
