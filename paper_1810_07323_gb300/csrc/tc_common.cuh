// PTX helpers shared by the tensor-core pass kernels (pass_tc.cu, pass_tc_lp.cu):
// mbarriers with bounded waits, TMA tile loads, tcgen05 descriptors, fences,
// TMEM loads, the Stream-K epilogue and 2-D tensor-map encoding.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace corutv {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false (and the timeout bit set) if the phase did not complete in time.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, DevStatus* st) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  uint32_t spins = 0;
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((++spins & 255u) == 0 && globaltimer_ns() - t0 > kWaitBudgetNs) {
      if (st) {
        atomicOr(&st->flags, kStatTimeout);
        atomicAdd(&st->timeouts, 1);
      }
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y,
                                            uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%3, %4}], [%2], %5;" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y), "l"(policy)
      : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// Shared-memory matrix descriptor (sm_100 family): start, leading / stride byte
// offsets (>> 4), version 1 at bit 46, 128-byte swizzle (layout 2) at bits 61-63.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | (2ull << 61);
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Epilogue of a Stream-K pass kernel, run by four consecutive warps (warp & 3
// selects the TMEM lane quarter).  Tile segments of this CTA alternate between
// the two TMEM accumulators (columns [0, BN) and [BN, 2 BN)); a segment that
// covers all k-blocks of its tile is written to Ct (row j = sketch column,
// masked to the first l rows and `len` positions), any other segment to the
// CTA's partial slot for the ordered reduction.
template <int BN, int M>
__device__ __forceinline__ void tc_epilogue(float* Ct, int64_t ldc, float* partials, int64_t len, int l, int64_t KB,
                                            const StreamK& sk, int64_t s, int64_t e, uint32_t tmem_base,
                                            uint32_t tfull0, uint32_t tempty0, DevStatus* status) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = warp & 3;
  const int j = 32 * g + lane;
  int seg = 0;
  int64_t it = s;
  while (it < e) {
    const int64_t t = it / KB;
    const int64_t kb0 = it - t * KB;
    const int64_t kb1 = (e - t * KB < KB) ? (e - t * KB) : KB;
    const int b = seg & 1;
    const uint32_t tph = (uint32_t)((seg >> 1) & 1);
    if (!mbar_wait(tfull0 + 8 * b, tph, status)) break;
    tc_fence_after();
    const bool complete = (kb0 == 0 && kb1 == KB);
    const int64_t p0 = t * BN;
    float* dst;
    int64_t lim;
    if (complete) {
      dst = Ct + (int64_t)j * ldc + p0;
      lim = len - p0;
    } else {
      dst = partials + ((int64_t)sk.slot(blockIdx.x, t) * M + j) * BN;
      lim = BN;
    }
#pragma unroll 1
    for (int c = 0; c < BN / 32; ++c) {
      float v[32];
      tmem_ld32(tmem_base + (uint32_t)(b * BN + 32 * c) + ((uint32_t)(32 * g) << 16), v);
      if (j < l) {
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
    it = t * KB + kb1;
  }
}


// ------------------------------------------------------------------ TF32 helpers
// Instruction descriptor, kind::tf32: D fp32 (bit 4), A/B tf32 (2 at bits 7, 10),
// A major (bit 15), B major (bit 16), N >> 3 (bits 17-22), M >> 4 (bits 24-28).
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N, int a_mn_major, int b_mn_major) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)a_mn_major << 15) | ((uint32_t)b_mn_major << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ float sel_comp(const float4& v, int j) {
  float r = v.x;
  r = (j == 1) ? v.y : r;
  r = (j == 2) ? v.z : r;
  r = (j == 3) ? v.w : r;
  return r;
}

// FP32 -> TF32, round to nearest (ties away from zero); low 13 bits become zero.
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// ------------------------------------------------------------------ converter warps (FP32 A tiles)
// The four converter warps (ct = 0..127) prepare one 256-position x 32 FP32 A
// tile (32 KB, 128-byte swizzle) for kind::tf32 and return their share of
// sum(a^2) of the original values (FRO).  CONV rounds to TF32 (nearest).
constexpr int kTf32TileBytes = 256 * 32 * 4;

// rows of A (dir AX): already K-major, round in place
template <bool CONV, bool FRO>
__device__ __forceinline__ float tc_conv_rows_tf32(uint8_t* tile, int ct) {
  float part = 0.f;
  float4* a4 = reinterpret_cast<float4*>(tile);
#pragma unroll 4
  for (int q = ct; q < kTf32TileBytes / 16; q += 128) {
    float4 v = a4[q];
    if (FRO) part = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, part))));
    if (CONV) {
      v.x = to_tf32(v.x); v.y = to_tf32(v.y); v.z = to_tf32(v.z); v.w = to_tf32(v.w);
      a4[q] = v;
    }
  }
  return part;
}

// columns of A (dir ATY): the tile arrives as 8 column chunks [c][k][32 n]
// (128-byte swizzle) and is rewritten in place as the K-major tile [n][32 k].
// Thread block b covers k = 4 kb .. 4 kb + 3, n = 4 nb .. 4 nb + 3 (kb = q / 64,
// nb = q % 64).  All four warps synchronise (named barrier 1) between reading
// and writing.
template <bool CONV, bool FRO>
__device__ __forceinline__ float tc_conv_transpose_tf32(uint8_t* tile, int ct) {
  float part = 0.f;
  float4 blk[4][4];
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int q = ct + 128 * b, kb = q >> 6, nb = q & 63;
    const int c = nb >> 3, ch = nb & 7;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = 4 * kb + i;
      blk[b][i] = *reinterpret_cast<const float4*>(tile + c * 4096 + k * 128 + ((ch ^ (k & 7)) << 4));
    }
  }
  asm volatile("bar.sync 1, 128;" ::: "memory");
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int q = ct + 128 * b, kb = q >> 6, nb = q & 63;
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int j = (jj + (nb >> 1)) & 3;        // rotate rows: conflict-free stores
      float4 v;
      v.x = sel_comp(blk[b][0], j); v.y = sel_comp(blk[b][1], j);
      v.z = sel_comp(blk[b][2], j); v.w = sel_comp(blk[b][3], j);
      if (FRO) part = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, part))));
      if (CONV) { v.x = to_tf32(v.x); v.y = to_tf32(v.y); v.z = to_tf32(v.z); v.w = to_tf32(v.w); }
      const int nrow = 4 * nb + j;
      *reinterpret_cast<float4*>(tile + nrow * 128 + ((kb ^ (nrow & 7)) << 4)) = v;
    }
  }
  return part;
}

// ------------------------------------------------------------------ host side
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2-D row-major matrix (rows x cols, leading dimension ld elements of elem_bytes),
// box (box_cols x box_rows), 128-byte swizzle or none, zero fill out of bounds.
inline bool make_map_2d(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld, int elem_bytes,
                        CUtensorMapDataType dtype, int box_cols, int box_rows, bool swizzle128) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * elem_bytes)};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, dtype, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace corutv
