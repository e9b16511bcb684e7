// Grouped TF32 tensor-core passes for batched solves: one launch computes
// Ct_p (l_p x len_p) = Xt_p (l_p x K_p) op_p(A_p) for every problem p of a
// table, with the same warp roles as pass_tc.cu (TMA producer, single-thread
// tcgen05.mma issuer, TMEM epilogue, converter warps rounding A tiles to TF32
// and transposing A^T tiles).  The (problem, tile, k-block) iterations of all
// problems are concatenated and split Stream-K style over one CTA per SM; each
// role walks its CTA's range forward, problem by problem, reading the
// problem's tensor maps (in device memory) from its table entry.  Tiles shared
// by several CTAs go through partial slots (a CTA's first partial segment in
// slot 2c, its last in 2c + 1) and an ordered reduction.  Every wait is bounded.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace corutv {

namespace {

constexpr int kBN = 256;          // output positions per tile
constexpr int kM = 128;           // MMA M (sketch rows, padded)
constexpr int kBK = 32;           // FP32 elements of K per stage
constexpr int kStages = 4;
constexpr int kATile = kBN * kBK * 4;   // 32 KB
constexpr int kXTile = kM * kBK * 4;    // 16 KB
constexpr int kStage = kATile + kXTile;
constexpr int kThreads = 320;     // 0 TMA, 1 MMA, 2..5 epilogue, 6..9 converter
constexpr int kSmem = kStages * kStage + 1024 + 512;

__host__ __device__ inline int64_t gstart(int64_t c, int64_t total, int64_t G) { return (c * total) / G; }
__host__ __device__ inline int64_t gowner(int64_t x, int64_t total, int64_t G) {
  int64_t c = ((x + 1) * G + total - 1) / total - 1;
  if (c < 0) c = 0;
  if (c > G - 1) c = G - 1;
  return c;
}

// problem of global iteration x (largest p with iter_base <= x)
__device__ inline int find_problem(const GPassProb* __restrict__ gp, int np, int64_t x) {
  int lo = 0, hi = np - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (gp[mid].iter_base <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ inline int64_t iter_end(const GPassProb& P) { return P.iter_base + P.tiles * P.KB; }

template <bool FRO>
__global__ void __launch_bounds__(kThreads, 1)
    pass_tc_grouped_kernel(const GPassProb* __restrict__ gp, int np, int64_t total, float* __restrict__ partials,
                           DevStatus* status, int keep_a) {
  extern __shared__ uint8_t smem_dyn[];
  uint8_t* smem = smem_dyn + ((1024u - (smem_u32(smem_dyn) & 1023u)) & 1023u);
  uint8_t* a_tiles = smem;
  uint8_t* x_tiles = smem + kStages * kATile;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * kStage);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * kStages + 4);
  volatile int* conv_abort = reinterpret_cast<volatile int*>(bars + 3 * kStages + 6);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + kStages), conv0 = smem_u32(bars + 2 * kStages);
  const uint32_t tfull0 = smem_u32(bars + 3 * kStages), tempty0 = smem_u32(bars + 3 * kStages + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t G = gridDim.x;
  const int64_t s = gstart(blockIdx.x, total, G), e = gstart(blockIdx.x + 1, total, G);

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
  int pi = find_problem(gp, np, s);

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      // keep_a: A is read again by the next launch (fused power steps), so it stays in L2
      const uint64_t pol_a = keep_a ? policy_evict_last() : policy_evict_first(), pol_x = policy_evict_last();
      int64_t n = 0;
      bool ok = true;
      int64_t pend = iter_end(gp[pi]);
      for (int64_t it = s; it < e; ++it, ++n) {
        while (it >= pend) pend = iter_end(gp[++pi]);
        const GPassProb& P = gp[pi];
        const int stage = (int)(n % kStages);
        const uint32_t ph = (uint32_t)((n / kStages) & 1);
        if (!mbar_wait(empty0 + 8 * stage, ph ^ 1, status)) { ok = false; break; }
        const int64_t local = it - P.iter_base, t = local / P.KB, kb = local - t * P.KB;
        const int k0 = (int)(kb * kBK), p0 = (int)(t * kBN);
        const CUtensorMap* mA = static_cast<const CUtensorMap*>(P.mapA);
        const CUtensorMap* mX = static_cast<const CUtensorMap*>(P.mapX);
        const uint32_t fb = full0 + 8 * stage;
        mbar_arrive_expect_tx(fb, kStage);
        const uint32_t adst = smem_u32(a_tiles + stage * kATile);
        if (P.dir == 0) {
          tma_load_2d(adst, mA, fb, k0, p0, pol_a);                                 // 256 rows x 32 cols
        } else {
#pragma unroll
          for (int c = 0; c < kBN / 32; ++c)                                        // 8 x (32 rows x 32 cols)
            tma_load_2d(adst + c * (kBK * 128), mA, fb, p0 + 32 * c, k0, pol_a);
        }
        tma_load_2d(smem_u32(x_tiles + stage * kXTile), mX, fb, k0, 0, pol_x);
      }
      const int64_t first = n > kStages ? n - kStages : 0;
      for (int64_t f = first; f < n; ++f) {
        const int stage = (int)(f % kStages);
        const uint32_t ph = (uint32_t)((f / kStages) & 1);
        if (ok) {
          if (!mbar_wait(empty0 + 8 * stage, ph, status)) ok = false;
        }
        if (!ok) mbar_wait(full0 + 8 * stage, ph, status);
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_tf32(kM, kBN, 0, 0);
      int64_t n = 0;
      int seg = 0;
      bool ok = true;
      int64_t it = s;
      int64_t pend = iter_end(gp[pi]);
      while (it < e && ok) {
        while (it >= pend) pend = iter_end(gp[++pi]);
        const GPassProb& P = gp[pi];
        const int64_t t = (it - P.iter_base) / P.KB;
        const int64_t tile_end = P.iter_base + (t + 1) * P.KB;
        const int64_t seg_end = e < tile_end ? e : tile_end;
        const int b = seg & 1;
        const uint32_t tph = (uint32_t)((seg >> 1) & 1);
        if (!mbar_wait(tempty0 + 8 * b, tph ^ 1, status)) { ok = false; break; }
        tc_fence_after();
        const uint32_t tacc = tmem_base + (uint32_t)(b * kBN);
        bool first = true;
        for (; it < seg_end; ++it, ++n) {
          const int stage = (int)(n % kStages);
          const uint32_t ph = (uint32_t)((n / kStages) & 1);
          if (!mbar_wait(conv0 + 8 * stage, ph, status)) { ok = false; break; }
          tc_fence_after();
          const uint32_t abase = smem_u32(a_tiles + stage * kATile);
          const uint32_t xbase = smem_u32(x_tiles + stage * kXTile);
#pragma unroll
          for (int kk = 0; kk < kBK / 8; ++kk)
            mma_tf32(tacc, smem_desc(xbase + kk * 32, 16, 1024), smem_desc(abase + kk * 32, 16, 1024), idesc,
                     (first && kk == 0) ? 0u : 1u);
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
    const int g = warp & 3, j = 32 * g + lane;
    int seg = 0;
    int64_t it = s;
    int64_t pend = iter_end(gp[pi]);
    while (it < e) {
      while (it >= pend) pend = iter_end(gp[++pi]);
      const GPassProb& P = gp[pi];
      const int64_t t = (it - P.iter_base) / P.KB;
      const int64_t tile_first = P.iter_base + t * P.KB, tile_end = tile_first + P.KB;
      const int64_t seg_end = e < tile_end ? e : tile_end;
      const int b = seg & 1;
      const uint32_t tph = (uint32_t)((seg >> 1) & 1);
      if (!mbar_wait(tfull0 + 8 * b, tph, status)) break;
      tc_fence_after();
      const bool complete = it == tile_first && seg_end == tile_end;
      const int64_t p0 = t * kBN;
      float* dst;
      int64_t lim;
      if (complete) {
        dst = P.Ct + (int64_t)j * P.ldc + p0;
        lim = P.len - p0;
      } else {
        const int64_t slot = 2 * (int64_t)blockIdx.x + (it == s ? 0 : 1);
        dst = partials + (slot * kM + j) * kBN;
        lim = kBN;
      }
#pragma unroll 1
      for (int c = 0; c < kBN / 32; ++c) {
        float v[32];
        tmem_ld32(tmem_base + (uint32_t)(b * kBN + 32 * c) + ((uint32_t)(32 * g) << 16), v);
        if (j < P.l) {
          const int64_t col0 = 32 * c;
          if (col0 + 32 <= lim) {
            float4* d4 = reinterpret_cast<float4*>(dst + col0);
#pragma unroll
            for (int q = 0; q < 8; ++q) d4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
          } else {
#pragma unroll
            for (int q = 0; q < 32; ++q)
              if (col0 + q < lim) dst[col0 + q] = v[q];
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty0 + 8 * b);
      ++seg;
      it = seg_end;
    }
  } else {
    // ---------------------------------------------------------------- converter (warps 6..9)
    const int ct = threadIdx.x - 192;
    if (ct == 0) *conv_abort = 0;
    asm volatile("bar.sync 1, 128;" ::: "memory");
    double fro = 0.0;
    int64_t n = 0;
    int64_t pend = iter_end(gp[pi]);
    int fro_p = pi;
    // sum(a^2) of this CTA's share of problem p, one FP64 value per converter warp
    auto flush = [&](int p) {
      if (!FRO) return;
      double v = fro;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      const GPassProb& Q = gp[p];
      if (lane == 0 && Q.fro) Q.fro[4 * (blockIdx.x - Q.owner_first) + (warp - 6)] = v;
      fro = 0.0;
    };
    for (int64_t it = s; it < e; ++it, ++n) {
      while (it >= pend) pend = iter_end(gp[++pi]);
      if (pi != fro_p) {
        flush(fro_p);
        fro_p = pi;
      }
      const int stage = (int)(n % kStages);
      const uint32_t ph = (uint32_t)((n / kStages) & 1);
      // the transposes synchronise the four converter warps: they give up together
      if (!mbar_wait(full0 + 8 * stage, ph, status)) *conv_abort = 1;
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (*conv_abort) break;
      uint8_t* tile = a_tiles + stage * kATile;
      const float part = gp[pi].dir == 0 ? tc_conv_rows_tf32<true, FRO>(tile, ct)
                                         : tc_conv_transpose_tf32<true, FRO>(tile, ct);
      fro += (double)part;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(conv0 + 8 * stage);
    }
    flush(fro_p);
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem_base) : "memory");
  }
}

// Ordered sum of the partial slots of split tiles.  A tile is split exactly when a CTA's first
// iteration lies inside it; block (c, g) takes the tile holding CTA c's first iteration if that
// tile is split and c is the first CTA to start inside it, and sums rows 4 g .. 4 g + 3 (a thread
// per column) over the CTAs that share the tile, in CTA order.  (One block per CTA boundary and
// row group, not per tile.)
__global__ void __launch_bounds__(256) grouped_reduce_kernel(const GPassProb* __restrict__ gp, int np,
                                                             int64_t total, int64_t G,
                                                             const float* __restrict__ partials) {
  static_assert(kBN == 256, "a thread per tile column");
  const int64_t c = blockIdx.x;
  if (c == 0) return;                                     // CTA 0 starts at a tile start
  const int64_t x = gstart(c, total, G);
  if (x >= total) return;
  const GPassProb& P = gp[find_problem(gp, np, x)];
  const int64_t t = (x - P.iter_base) / P.KB;
  const int64_t first_it = P.iter_base + t * P.KB, last_it = first_it + P.KB - 1;
  if (x == first_it) return;                              // c starts a tile: no split at this boundary
  if (gstart(c - 1, total, G) > first_it) return;         // an earlier CTA also starts inside the tile
  const int row0 = blockIdx.y * 4;
  if (row0 >= P.l) return;
  const int64_t cf = gowner(first_it, total, G), cl = gowner(last_it, total, G);
  const int ii = threadIdx.x;
  const int64_t p0 = t * kBN;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int64_t cc = cf; cc <= cl; ++cc) {
    const int64_t slot = 2 * cc + (gstart(cc, total, G) >= first_it ? 0 : 1);
    const float* src = partials + (slot * kM + row0) * kBN + ii;
#pragma unroll
    for (int r = 0; r < 4; ++r) acc[r] += src[r * kBN];
  }
  if (p0 + ii >= P.len) return;
#pragma unroll
  for (int r = 0; r < 4; ++r)
    if (row0 + r < P.l) P.Ct[(int64_t)(row0 + r) * P.ldc + p0 + ii] = acc[r];
}

// Xr = TF32(X) (round to nearest) for every problem of the table; block (map[b].x, map[b].y)
// covers 128 columns, four consecutive columns per thread and step (rows are 16-byte aligned)
__global__ void __launch_bounds__(256) grouped_round_kernel(const GPassProb* __restrict__ gp,
                                                            const int2* __restrict__ map) {
  const int2 pm = map[blockIdx.x];
  const GPassProb& P = gp[pm.x];
  const int64_t i0 = (int64_t)pm.y * 128;
  for (int e = threadIdx.x; e < P.l * 32; e += blockDim.x) {
    const int j = e >> 5;
    const int64_t i = i0 + 4 * (e & 31);
    if (i >= P.K) continue;
    if (i + 3 < P.K) {
      const float4 v = *reinterpret_cast<const float4*>(P.X + j * P.ldx + i);
      *reinterpret_cast<float4*>(P.Xr + j * P.ldr + i) =
          make_float4(to_tf32(v.x), to_tf32(v.y), to_tf32(v.z), to_tf32(v.w));
    } else {
      for (int q = 0; q < 4 && i + q < P.K; ++q) P.Xr[j * P.ldr + i + q] = to_tf32(P.X[j * P.ldx + i + q]);
    }
  }
}

}  // namespace

size_t tc_grouped_partial_bytes(int sms) { return (size_t)2 * sms * kM * kBN * sizeof(float); }

int64_t tc_grouped_tiles(int64_t len) { return cdiv(len, kBN); }
int64_t tc_grouped_kblocks(int64_t K) { return cdiv(K, kBK); }
int64_t tc_grouped_owner(int64_t x, int64_t total, int64_t G) { return gowner(x, total, G); }

cudaError_t launch_pass_tc_grouped(const GPassProb* gp, int np, int64_t total_iters, int64_t total_tiles, int lmax,
                                   const int2* round_map, int nround, float* partials, bool fro, int sms,
                                   DevStatus* status, bool keep_a, cudaStream_t st, KernelMark* km) {
  if (np <= 0 || total_iters <= 0) return cudaSuccess;
  if (nround > 0) {
    grouped_round_kernel<<<nround, 256, 0, st>>>(gp, round_map);
    CORUTV_COUNT_LAUNCH();
  }
  const int64_t G = total_iters < sms ? total_iters : sms;
  auto kern = fro ? pass_tc_grouped_kernel<true> : pass_tc_grouped_kernel<false>;
  // raised once per device and variant (the first, uncaptured run of a batch)
  static bool attr_set[2][64] = {};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 0 || dev >= 64 || !attr_set[fro ? 1 : 0][dev]) {
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (err != cudaSuccess) return err;
    if (dev >= 0 && dev < 64) attr_set[fro ? 1 : 0][dev] = true;
  }
  if (km) km->start(st);
  kern<<<(unsigned)G, kThreads, kSmem, st>>>(gp, np, total_iters, partials, status, keep_a ? 1 : 0);
  CORUTV_COUNT_LAUNCH();
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  if (km) km->stop(st);
  (void)total_tiles;
  dim3 rgrid((unsigned)G, (unsigned)cdiv(lmax, 4));
  grouped_reduce_kernel<<<rgrid, 256, 0, st>>>(gp, np, total_iters, G, partials);
  CORUTV_COUNT_LAUNCH();
  return cudaGetLastError();
}

}  // namespace corutv
