// CUDA-core (SIMT) streaming passes over A, the products of Sec. III
// (C1 = A Psi, C2 = A^T C1) and of Alg. 3 steps 3-4, in the storage
// precision (FP64 for FP64 data; FP32 accumulation otherwise), plus the
// ordered reduction of Stream-K partial tiles shared with the tensor-core
// passes.
//
// Layout: the skinny operand and the result are "skinny transposed": l rows
// of `len` contiguous elements.  dir AX: Ct[j][i] = sum_k Xt[j][k] A[i][k];
// dir ATY: Ct[j][c] = sum_r Xt[j][r] A[r][c].
#include "common.cuh"
#include "elem.cuh"
#include "internal.h"

namespace corutv {

namespace {

constexpr int kBN = 64;   // output positions per tile
constexpr int kBK = 32;   // reduction depth per shared-memory stage

template <typename TA, int DIR, int JPT>
__global__ void __launch_bounds__(256) pass_simt_kernel(PassArgs args) {
  using TC = typename Elem<TA>::acc;
  constexpr int LP = 16 * JPT;
  __shared__ TC As[kBN][kBK + 1];
  __shared__ TC Xs[LP][kBK + 1];

  const TA* A = static_cast<const TA*>(args.A);
  const TC* Xt = static_cast<const TC*>(args.Xt);
  TC* Ct = static_cast<TC*>(args.Ct);
  TC* P = static_cast<TC*>(args.partials);
  const int64_t len = args.len_out, K = args.K;
  const int64_t KB = cdiv_d(K, kBK);
  StreamK sk(cdiv_d(len, kBN), KB, gridDim.x);
  const int64_t s = sk.start(blockIdx.x), e = sk.start(blockIdx.x + 1);
  const int tid = threadIdx.x, ti = tid & 15, tj = tid >> 4;
  const int l = args.l;
  const int64_t sld = args.scale_ld;

  int64_t it = s;
  while (it < e) {
    const int64_t t = it / KB;
    const int64_t kb0 = it - t * KB;
    const int64_t kb1 = (e - t * KB < KB) ? (e - t * KB) : KB;
    const int64_t i0 = t * kBN;
    TC acc[JPT][4];
#pragma unroll
    for (int v = 0; v < JPT; ++v)
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[v][u] = TC(0);

    for (int64_t kb = kb0; kb < kb1; ++kb) {
      const int64_t k0 = kb * kBK;
      // stage A tile into As[i][kk]
      for (int x = tid; x < kBN * kBK; x += 256) {
        int ii, kk;
        if (DIR == 0) { ii = x / kBK; kk = x % kBK; }   // coalesced along k (A rows)
        else          { kk = x / kBN; ii = x % kBN; }   // coalesced along i (A columns)
        const int64_t gi = i0 + ii, gk = k0 + kk;
        TC val = TC(0);
        if (gi < len && gk < K)
          val = (DIR == 0) ? Elem<TA>::load(A, gi, gk, args.lda, args.scales, sld)
                           : Elem<TA>::load(A, gk, gi, args.lda, args.scales, sld);
        As[ii][kk] = val;
      }
      for (int x = tid; x < LP * kBK; x += 256) {
        const int jj = x / kBK, kk = x % kBK;
        const int64_t gk = k0 + kk;
        Xs[jj][kk] = (jj < l && gk < K) ? Xt[jj * args.ldx + gk] : TC(0);
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < kBK; ++kk) {
        TC a[4], xv[JPT];
#pragma unroll
        for (int u = 0; u < 4; ++u) a[u] = As[ti + 16 * u][kk];
#pragma unroll
        for (int v = 0; v < JPT; ++v) xv[v] = Xs[tj + 16 * v][kk];
#pragma unroll
        for (int v = 0; v < JPT; ++v)
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[v][u] = fma(xv[v], a[u], acc[v][u]);
      }
      __syncthreads();
    }

    const bool complete = (kb0 == 0 && kb1 == KB);
    if (complete) {
#pragma unroll
      for (int v = 0; v < JPT; ++v) {
        const int j = tj + 16 * v;
        if (j >= l) continue;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t gi = i0 + ti + 16 * u;
          if (gi < len) Ct[j * args.ldc + gi] = acc[v][u];
        }
      }
    } else {
      TC* slot = P + (int64_t)sk.slot(blockIdx.x, t) * LP * kBN;
#pragma unroll
      for (int v = 0; v < JPT; ++v)
#pragma unroll
        for (int u = 0; u < 4; ++u) slot[(tj + 16 * v) * kBN + ti + 16 * u] = acc[v][u];
    }
    it = t * KB + kb1;
  }
}

// Batched pass: block b computes, for problem map[b].x, the kBN output positions
// of tile t over K range s (map[b].y = s * tiles + t), direction and sizes from the
// problem's descriptor.  `which` picks the product (C1 = op1(A) X from P2 into P1,
// C2 = op2(A) Q1 from P1 into P2, or the core pass E from P2 into P3); problems
// past their last power step (or without an exact core) exit.  With one range the
// block writes its tile; with S ranges it writes a partial, and the last of the
// tile's S blocks to finish (a counter per tile, no waiting) adds the S partials in
// range order, so the sum does not depend on the schedule.  The C1 pass of step 0
// also folds sum(a^2) of the A slab it reads into fparts (one FP64 partial per
// block, summed per problem in order later).
template <typename TA, int JPT>
__global__ void __launch_bounds__(256) pass_simt_grouped_kernel(const BatchProb* __restrict__ probs,
                                                                const int2* __restrict__ map, int which, int it) {
  using TC = typename Elem<TA>::acc;
  constexpr int LP = 16 * JPT;
  __shared__ TC As[kBN][kBK + 1];
  __shared__ TC Xs[LP][kBK + 1];
  __shared__ double fred[8];
  const int2 pm = map[blockIdx.x];
  const BatchProb& P = probs[pm.x];
  if (which == kB_CORE ? P.core != 0 : it > P.q) return;
  const int dir = which == kB_C2 ? P.dir2 : P.dir1;
  const TC* Xt = which == kB_C2 ? P.P1 : P.P2;
  const int64_t ldx = which == kB_C2 ? P.ld1 : P.ld2;
  TC* Ct = which == kB_C1 ? P.P1 : (which == kB_C2 ? P.P2 : P.P3);
  const int64_t ldc = which == kB_C1 ? P.ld1 : (which == kB_C2 ? P.ld2 : P.ld3);
  const int64_t len = which == kB_C2 ? P.len2 : P.len1, K = which == kB_C2 ? P.len1 : P.len2;
  const bool fro = which == kB_C1 && it == 0 && P.want_fro2;
  const TA* A = static_cast<const TA*>(P.A);
  const int l = P.l;
  const int tid = threadIdx.x, ti = tid & 15, tj = tid >> 4;
  const int S = which == kB_C2 ? P.ks2 : P.ks1;
  const int64_t tiles = cdiv_d(len, kBN);
  const int64_t tile = pm.y % tiles;
  const int rs = (int)(pm.y / tiles);
  const int64_t KC = cdiv_d(cdiv_d(K, S), kBK) * kBK;      // K range of one split, whole stages
  const int64_t kbeg = rs * KC, kend = kbeg + KC < K ? kbeg + KC : K;
  const int64_t i0 = tile * kBN;
  TC acc[JPT][4];
#pragma unroll
  for (int v = 0; v < JPT; ++v)
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[v][u] = TC(0);
  float fsum = 0.f;
  double fro_acc = 0.0;
  for (int64_t k0 = kbeg; k0 < kend; k0 += kBK) {
    for (int x = tid; x < kBN * kBK; x += 256) {
      int ii, kk;
      if (dir == 0) { ii = x / kBK; kk = x % kBK; }   // coalesced along k (A rows)
      else          { kk = x / kBN; ii = x % kBN; }   // coalesced along i (A columns)
      const int64_t gi = i0 + ii, gk = k0 + kk;
      TC val = TC(0);
      if (gi < len && gk < kend)
        val = (dir == 0) ? Elem<TA>::load(A, gi, gk, P.lda, P.scales, P.sld)
                         : Elem<TA>::load(A, gk, gi, P.lda, P.scales, P.sld);
      As[ii][kk] = val;
      if (fro) fsum = fmaf((float)val, (float)val, fsum);
    }
    for (int x = tid; x < LP * kBK; x += 256) {
      const int jj = x / kBK, kk = x % kBK;
      const int64_t gk = k0 + kk;
      Xs[jj][kk] = (jj < l && gk < kend) ? Xt[jj * ldx + gk] : TC(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kBK; ++kk) {
      TC a[4], xv[JPT];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = As[ti + 16 * u][kk];
#pragma unroll
      for (int v = 0; v < JPT; ++v) xv[v] = Xs[tj + 16 * v][kk];
#pragma unroll
      for (int v = 0; v < JPT; ++v)
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[v][u] = fma(xv[v], a[u], acc[v][u]);
    }
    __syncthreads();
    if (fro) {           // fold the FP32 squares of this stage into FP64
      fro_acc += (double)fsum;
      fsum = 0.f;
    }
  }
  // one K range: the tile itself; several: this range's partial, [range][j][i] with pitch len
  TC* dst = S == 1 ? Ct : P.kparts + (int64_t)rs * l * len;
  const int64_t ldd = S == 1 ? ldc : len;
#pragma unroll
  for (int v = 0; v < JPT; ++v) {
    const int j = tj + 16 * v;
    if (j >= l) continue;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t gi = i0 + ti + 16 * u;
      if (gi < len) dst[j * ldd + gi] = acc[v][u];
    }
  }
  if (S > 1) {
    __shared__ int last;
    __threadfence();                     // this block's partial is visible before it is counted
    __syncthreads();
    if (tid == 0) last = atomicAdd(&P.kcount[tile], 1) == S - 1;
    __syncthreads();
    if (last) {
      __threadfence();
      for (int x = tid; x < l * kBN; x += 256) {
        const int j = x / kBN;
        const int64_t gi = i0 + x % kBN;
        if (gi >= len) continue;
        TC sum = TC(0);
        for (int r = 0; r < S; ++r) sum += __ldcg(P.kparts + ((int64_t)r * l + j) * len + gi);
        Ct[j * ldc + gi] = sum;
      }
      if (tid == 0) P.kcount[tile] = 0;   // ready for the next pass
    }
  }
  if (fro) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fro_acc += __shfl_xor_sync(0xffffffffu, fro_acc, o);
    if ((tid & 31) == 0) fred[tid >> 5] = fro_acc;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += fred[w];
      P.fparts[pm.y] = t;
    }
  }
}

template <typename TA>
cudaError_t launch_grouped_dt(const BatchProb* P, const int2* map, int nblocks, int lp, int which, int it,
                              cudaStream_t st) {
  if (lp <= 32) pass_simt_grouped_kernel<TA, 2><<<nblocks, 256, 0, st>>>(P, map, which, it);
  else if (lp <= 64) pass_simt_grouped_kernel<TA, 4><<<nblocks, 256, 0, st>>>(P, map, which, it);
  else pass_simt_grouped_kernel<TA, 8><<<nblocks, 256, 0, st>>>(P, map, which, it);
  CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pass_simt_grouped(const BatchProb* P, const int2* map, int nblocks, int lp, int a_dtype,
                                     int which, int it, cudaStream_t st) {
  static_assert(kBN == kBatchPassBN, "batched pass tile");
  if (nblocks <= 0) return cudaSuccess;
  switch (a_dtype) {
    case 1: return launch_grouped_dt<float>(P, map, nblocks, lp, which, it, st);
    case 2: return launch_grouped_dt<__nv_bfloat16>(P, map, nblocks, lp, which, it, st);
    case 3: return launch_grouped_dt<__nv_fp8_e4m3>(P, map, nblocks, lp, which, it, st);
    default: return cudaErrorInvalidValue;
  }
}

// Ordered sum of Stream-K partial tiles: tile t (BN output positions, LP rows)
// split across workers cf..cl is the sum of their slots in worker order.
// Block (t, g) handles rows 16 g .. 16 g + 15 of tile t; the slot list is
// resolved once per block.
template <typename TC>
__global__ void __launch_bounds__(256) streamk_reduce_kernel(TC* __restrict__ Ct, int64_t ldc,
                                                             const TC* __restrict__ P, int l, int LP, int BN,
                                                             int64_t len, int64_t KB, int64_t G) {
  constexpr int kMaxSplit = 64;
  __shared__ int64_t slot_off[kMaxSplit];
  __shared__ int nsplit;
  StreamK sk((len + BN - 1) / BN, KB, G);
  const int64_t t = blockIdx.x;
  const int row0 = blockIdx.y * 16;
  if (row0 >= l) return;
  if (threadIdx.x == 0) {
    const int64_t cf = sk.owner(t * KB), cl = sk.owner(t * KB + KB - 1);
    int ns = (int)(cl - cf + 1);
    if (cf == cl) ns = 0;                        // written directly by its only worker
    if (ns > kMaxSplit) ns = -1;                 // never happens for the grids used here
    nsplit = ns;
    for (int i = 0; i < ns && i < kMaxSplit; ++i) slot_off[i] = (int64_t)sk.slot(cf + i, t) * LP * BN;
  }
  __syncthreads();
  const int ns = nsplit;
  if (ns == 0) return;
  const int64_t p0 = t * BN;
  for (int x = threadIdx.x; x < 16 * BN; x += blockDim.x) {
    const int j = row0 + x / BN, ii = x % BN;
    const int64_t gi = p0 + ii;
    if (j >= l || gi >= len) continue;
    TC sum = TC(0);
    if (ns > 0) {
      for (int c = 0; c < ns; ++c) sum += P[slot_off[c] + (int64_t)j * BN + ii];
    } else {
      const int64_t cf = sk.owner(t * KB), cl = sk.owner(t * KB + KB - 1);
      for (int64_t c = cf; c <= cl; ++c) sum += P[((int64_t)sk.slot(c, t) * LP + j) * BN + ii];
    }
    Ct[j * ldc + gi] = sum;
  }
}

template __global__ void streamk_reduce_kernel<float>(float*, int64_t, const float*, int, int, int, int64_t, int64_t,
                                                      int64_t);
template __global__ void streamk_reduce_kernel<double>(double*, int64_t, const double*, int, int, int, int64_t,
                                                       int64_t, int64_t);

// FP32 version with 16-byte accesses: block (t, g) handles rows 8 g .. 8 g + 7 of tile t,
// a thread 4 consecutive positions; all slot loads are issued before the ordered sum.
__global__ void __launch_bounds__(256) streamk_reduce_f32v_kernel(float* __restrict__ Ct, int64_t ldc,
                                                                  const float* __restrict__ P, int l, int LP, int BN,
                                                                  int64_t len, int64_t KB, int64_t G) {
  constexpr int kMaxSplit = 64, kUnroll = 4;
  __shared__ int64_t slot_off[kMaxSplit];
  __shared__ int nsplit;
  StreamK sk((len + BN - 1) / BN, KB, G);
  const int64_t t = blockIdx.x;
  const int row0 = blockIdx.y * 8;
  if (row0 >= l) return;
  if (threadIdx.x == 0) {
    const int64_t cf = sk.owner(t * KB), cl = sk.owner(t * KB + KB - 1);
    int ns = (int)(cl - cf + 1);
    if (cf == cl) ns = 0;                        // written directly by its only worker
    if (ns > kMaxSplit) ns = kMaxSplit + 1;      // resolved per element below
    nsplit = ns;
    for (int i = 0; i < ns && i < kMaxSplit; ++i) slot_off[i] = (int64_t)sk.slot(cf + i, t) * LP * BN;
  }
  __syncthreads();
  const int ns = nsplit;
  if (ns == 0) return;
  const int64_t p0 = t * BN;
  const int q4 = BN / 4;
  for (int x = threadIdx.x; x < 8 * q4; x += blockDim.x) {
    const int j = row0 + x / q4, ii = 4 * (x % q4);
    const int64_t gi = p0 + ii;
    if (j >= l || gi >= len) continue;
    float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ns <= kMaxSplit) {
      for (int c0 = 0; c0 < ns; c0 += kUnroll) {
        float4 v[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
          if (c0 + u < ns) v[u] = *reinterpret_cast<const float4*>(P + slot_off[c0 + u] + (int64_t)j * BN + ii);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
          if (c0 + u < ns) {
            sum.x += v[u].x; sum.y += v[u].y; sum.z += v[u].z; sum.w += v[u].w;
          }
      }
    } else {
      const int64_t cf = sk.owner(t * KB), cl = sk.owner(t * KB + KB - 1);
      for (int64_t c = cf; c <= cl; ++c) {
        const float4 v = *reinterpret_cast<const float4*>(P + ((int64_t)sk.slot(c, t) * LP + j) * BN + ii);
        sum.x += v.x; sum.y += v.y; sum.z += v.z; sum.w += v.w;
      }
    }
    float* dst = Ct + j * ldc + gi;
    if (gi + 3 < len && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
      *reinterpret_cast<float4*>(dst) = sum;
    } else {
      const float sv[4] = {sum.x, sum.y, sum.z, sum.w};
      for (int u = 0; u < 4; ++u)
        if (gi + u < len) dst[u] = sv[u];
    }
  }
}

cudaError_t launch_streamk_reduce_f32(float* Ct, int64_t ldc, const float* P, int l, int LP, int BN, int64_t len,
                                      int64_t KB, int64_t G, cudaStream_t st) {
  const int64_t tiles = cdiv(len, BN);
  if (tiles <= 0) return cudaSuccess;
  if (BN % 4 == 0) {
    dim3 grid((unsigned)tiles, (unsigned)cdiv(l, 8));
    streamk_reduce_f32v_kernel<<<grid, 256, 0, st>>>(Ct, ldc, P, l, LP, BN, len, KB, G);
  } else {
    dim3 grid((unsigned)tiles, (unsigned)cdiv(l, 16));
    streamk_reduce_kernel<float><<<grid, 256, 0, st>>>(Ct, ldc, P, l, LP, BN, len, KB, G);
  }
  CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

int64_t simt_pass_grid(int64_t len, int64_t K, int sms) {
  const int64_t work = cdiv(len, kBN) * cdiv(K, kBK);
  int64_t G = (int64_t)sms * 4;
  return G < work ? G : work;
}

size_t simt_pass_partial_bytes(int64_t len, int64_t K, int l, int elem_bytes, int sms) {
  const int LP = l <= 32 ? 32 : (l <= 64 ? 64 : 128);
  return (size_t)2 * simt_pass_grid(len, K, sms) * LP * kBN * elem_bytes;
}

template <typename TA, int DIR>
static cudaError_t launch_jpt(const PassArgs& a, int64_t G, cudaStream_t st) {
  if (a.l <= 32) { pass_simt_kernel<TA, DIR, 2><<<(unsigned)G, 256, 0, st>>>(a); CORUTV_COUNT_LAUNCH(); }
  else if (a.l <= 64) { pass_simt_kernel<TA, DIR, 4><<<(unsigned)G, 256, 0, st>>>(a); CORUTV_COUNT_LAUNCH(); }
  else { pass_simt_kernel<TA, DIR, 8><<<(unsigned)G, 256, 0, st>>>(a); CORUTV_COUNT_LAUNCH(); }
  return cudaGetLastError();
}

template <typename TA>
static cudaError_t launch_dir(const PassArgs& a, int dir, int64_t G, cudaStream_t st) {
  return dir == 0 ? launch_jpt<TA, 0>(a, G, st) : launch_jpt<TA, 1>(a, G, st);
}

cudaError_t launch_pass_simt(const PassArgs& a, int dir, int a_dtype, int sms, cudaStream_t st) {
  const int64_t G = simt_pass_grid(a.len_out, a.K, sms);
  if (G <= 0) return cudaSuccess;
  cudaError_t err;
  if (a.kmark) a.kmark->start(st);
  switch (a_dtype) {
    case 0: err = launch_dir<double>(a, dir, G, st); break;
    case 1: err = launch_dir<float>(a, dir, G, st); break;
    case 2: err = launch_dir<__nv_bfloat16>(a, dir, G, st); break;
    case 3: err = launch_dir<__nv_fp8_e4m3>(a, dir, G, st); break;
    default: return cudaErrorInvalidValue;
  }
  if (err != cudaSuccess) return err;
  if (a.kmark) a.kmark->stop(st);
  const int LP = a.l <= 32 ? 32 : (a.l <= 64 ? 64 : 128);
  const int64_t tiles = cdiv(a.len_out, kBN), KB = cdiv(a.K, kBK);
  const dim3 rgrid((unsigned)tiles, (unsigned)cdiv(a.l, 16));
  if (a_dtype == 0) {
    streamk_reduce_kernel<double><<<rgrid, 256, 0, st>>>(static_cast<double*>(a.Ct), a.ldc,
                                                                   static_cast<const double*>(a.partials), a.l, LP,
                                                                   kBN, a.len_out, KB, G);
  } else {
    streamk_reduce_kernel<float><<<rgrid, 256, 0, st>>>(static_cast<float*>(a.Ct), a.ldc,
                                                                  static_cast<const float*>(a.partials), a.l, LP,
                                                                  kBN, a.len_out, KB, G);
  }
  CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

}  // namespace corutv
