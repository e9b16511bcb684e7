// C-ABI front end of libcorutv: argument checks, workspace planning, and the
// schedule of one CoR-UTV solve (Alg. 2 / Alg. 3 of the paper, stabilised
// range finding) enqueued on the handle's stream.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/corutv.h"
#include "common.cuh"
#include "internal.h"
#include "handle.h"

using namespace corutv;

namespace corutv {
int64_t& launch_counter() {
  static thread_local int64_t n = 0;
  return n;
}
}  // namespace corutv

namespace {

// ---------------------------------------------------------------- sizes
constexpr int64_t kAlign = 256;

inline int elem_bytes(int dt) { return dt == CORUTV_F64 ? 8 : (dt == CORUTV_F32 ? 4 : (dt == CORUTV_BF16 ? 2 : 1)); }
inline int tc_bytes(int dt) { return dt == CORUTV_F64 ? 8 : 4; }   // sketch / compute precision
inline bool aligned16(const void* ptr) { return ((uintptr_t)ptr & 15u) == 0; }

struct Carve {
  char* base;
  size_t off = 0;
  explicit Carve(void* b) : base(static_cast<char*>(b)) {}
  void* take(size_t bytes) {
    off = (size_t)round_up((int64_t)off, kAlign);
    void* p = base ? base + off : nullptr;
    off += bytes;
    return p;
  }
};

// Workspace of one solve.
struct Plan {
  int64_t len1, len2;       // lengths of the first (C1) and second (C2) sketch
  int64_t ld1, ld2, ld3, ldr;
  int LP;                   // rows of every ST buffer (>= l, 128 on the tensor-core path)
  size_t pass_partials;
  int gparts;
  int fparts;
  // carved pointers
  DevStatus* status;
  void *P1, *P2, *P3, *Xr;
  void* partials;
  void* gram_parts;
  void *G, *D, *Qt;         // l x l Gram / core / Q~ in the compute type (FP64-sized)
  double* fro_parts;
  void *R, *Rinv;
  int* defic;
};

size_t plan_layout(Plan& pl, void* base) {
  Carve c(base);
  pl.status = static_cast<DevStatus*>(c.take(sizeof(DevStatus)));
  const int tb = 8;  // sized for the wider of the two compute types
  pl.P1 = c.take((size_t)pl.LP * pl.ld1 * tb);
  pl.P2 = c.take((size_t)pl.LP * pl.ld2 * tb);
  pl.P3 = c.take((size_t)pl.LP * pl.ld3 * tb);
  // the sketch operand of a tensor-core pass: TF32-rounded (first half), TF32 hi / lo split
  // (both halves), or BF16 hi / lo (first half)
  pl.Xr = c.take((size_t)2 * pl.LP * pl.ldr * 4);
  pl.partials = c.take(pl.pass_partials);
  pl.gram_parts = c.take((size_t)pl.gparts * kMaxL * kMaxL * tb);
  pl.G = c.take(sizeof(double) * kMaxL * kMaxL);
  pl.D = c.take(sizeof(double) * kMaxL * kMaxL);
  pl.Qt = c.take(sizeof(double) * kMaxL * kMaxL);
  pl.R = c.take((size_t)kMaxL * kMaxL * tb);
  pl.Rinv = c.take((size_t)kMaxL * kMaxL * tb);
  pl.defic = static_cast<int*>(c.take(sizeof(int) * kMaxL));
  pl.fro_parts = static_cast<double*>(c.take(sizeof(double) * pl.fparts));
  return (size_t)round_up((int64_t)c.off, kAlign);
}

int device_sms(int* sms_out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CORUTV_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CORUTV_ERR_CUDA;
  *sms_out = sms;
  return CORUTV_OK;
}

size_t pass_partial_bytes(int64_t m, int64_t n, int l, int a_dtype, int sms) {
  size_t b = 0;
  // both directions, both engines (the plan does not depend on the engine chosen later)
  b = std::max(b, simt_pass_partial_bytes(m, n, l, tc_bytes(a_dtype), sms));
  b = std::max(b, simt_pass_partial_bytes(n, m, l, tc_bytes(a_dtype), sms));
  if (a_dtype == CORUTV_F32) {
    b = std::max(b, tc_pass_partial_bytes(m, n, sms));
    b = std::max(b, tc_pass_partial_bytes(n, m, sms));
    b = std::max(b, tc3_pass_partial_bytes(sms));
  }
  // the correction pass of a BF16 / FP8 solve runs on FP32 A
  if (a_dtype == CORUTV_BF16 || a_dtype == CORUTV_FP8_E4M3) {
    b = std::max(b, tc_lp_partial_bytes(sms));
    b = std::max(b, tc_pass_partial_bytes(m, n, sms));
    b = std::max(b, tc3_pass_partial_bytes(sms));
    b = std::max(b, simt_pass_partial_bytes(m, n, l, 4, sms));
    b = std::max(b, simt_pass_partial_bytes(n, m, l, 4, sms));
  }
  return b;
}

void make_plan(const corutv_params* p, int sms, Plan& pl) {
  const bool right = p->side == CORUTV_SIDE_RIGHT;
  pl.len1 = right ? p->m : p->n;   // C1 = A Psi (right) or A^T Psi (left)
  pl.len2 = right ? p->n : p->m;
  pl.ld1 = ld_for(pl.len1);
  pl.ld2 = ld_for(pl.len2);
  pl.ld3 = std::max(pl.ld1, pl.ld2);
  pl.ldr = pl.ld3;
  pl.LP = kMaxL;
  pl.pass_partials = pass_partial_bytes(p->m, p->n, p->l, p->a_dtype, sms);
  pl.gparts = std::max(gram_parts(pl.len1, sms), gram_parts(pl.len2, sms));
  pl.fparts = fro2_parts(sms);
}

// engine allowed for a storage dtype
bool mma_fits_dtype(int a_dtype, int mma) {
  if (mma == CORUTV_MMA_AUTO || mma == CORUTV_MMA_SIMT) return true;
  if (mma == CORUTV_MMA_TF32 || mma == CORUTV_MMA_TF32_TRUNC || mma == CORUTV_MMA_TF32X3) return a_dtype == CORUTV_F32;
  if (mma == CORUTV_MMA_BF16X2) return a_dtype == CORUTV_BF16 || a_dtype == CORUTV_FP8_E4M3;
  return false;
}

int check_params(const corutv_params* p) {
  if (!p) return CORUTV_ERR_INVALID_ARG;
  for (int r : p->reserved)
    if (r != 0) return CORUTV_ERR_INVALID_ARG;
  if (p->a_dtype < CORUTV_F64 || p->a_dtype > CORUTV_FP8_E4M3) return CORUTV_ERR_INVALID_ARG;
  if (p->side != CORUTV_SIDE_RIGHT && p->side != CORUTV_SIDE_LEFT) return CORUTV_ERR_INVALID_ARG;
  if (p->core != CORUTV_CORE_EXACT && p->core != CORUTV_CORE_SKETCH) return CORUTV_ERR_INVALID_ARG;
  if (p->orth != CORUTV_ORTH_STABILISED && p->orth != CORUTV_ORTH_STRICT && p->orth != CORUTV_ORTH_LITERAL)
    return CORUTV_ERR_INVALID_ARG;
  if (p->orth == CORUTV_ORTH_LITERAL && p->core != CORUTV_CORE_EXACT) return CORUTV_ERR_UNSUPPORTED;
  if (p->mma < CORUTV_MMA_AUTO || p->mma > CORUTV_MMA_BF16X2) return CORUTV_ERR_INVALID_ARG;
  if (p->m <= 0 || p->n <= 0) return CORUTV_ERR_SHAPE;
  if (p->k < 1 || p->k > p->l) return CORUTV_ERR_INVALID_ARG;      // 1 <= k <= l (Sec. III)
  if (p->q < 0) return CORUTV_ERR_INVALID_ARG;
  if (p->l >= std::min(p->m, p->n)) return CORUTV_ERR_SHAPE;      // l < min(m, n) (Sec. III)
  if (p->l > (p->a_dtype == CORUTV_F64 ? kMaxL64 : kMaxL)) return CORUTV_ERR_SHAPE;
  if (!mma_fits_dtype(p->a_dtype, p->mma)) return CORUTV_ERR_UNSUPPORTED;
  if (p->factor != CORUTV_FACTOR_QRCP && p->factor != CORUTV_FACTOR_QLP) return CORUTV_ERR_INVALID_ARG;
  if (p->factor == CORUTV_FACTOR_QLP && p->a_dtype == CORUTV_F64) return CORUTV_ERR_UNSUPPORTED;
  if (p->small_f64 != 0 && p->small_f64 != 1) return CORUTV_ERR_INVALID_ARG;
  if (p->small_f64 && p->factor == CORUTV_FACTOR_QLP) return CORUTV_ERR_UNSUPPORTED;
  return CORUTV_OK;
}

int ensure_workspace(corutv_handle* h, size_t need) {
  if (h->ws && h->ws_bytes >= need) return CORUTV_OK;
  if (h->ws && !h->own_ws) return CORUTV_ERR_OOM;   // caller workspace too small
  if (h->ws) {
    cudaStreamSynchronize(h->stream);
    cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
  }
  void* p = nullptr;
  if (cudaMalloc(&p, need) != cudaSuccess) {
    cudaGetLastError();
    return CORUTV_ERR_OOM;
  }
  // zero once: rows >= l of the sketch buffers are read (never used) by the tensor-core passes
  if (cudaMemsetAsync(p, 0, need, h->stream) != cudaSuccess) {
    cudaFree(p);
    return CORUTV_ERR_CUDA;
  }
  h->ws = p;
  h->ws_bytes = need;
  h->own_ws = true;
  return CORUTV_OK;
}

#define CU(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) {                    \
      fprintf(stderr, "corutv: %s (%s:%d)\n", cudaGetErrorString(e_), __FILE__, __LINE__); \
      return CORUTV_ERR_CUDA;                   \
    }                                           \
  } while (0)

// engine for a pass; AUTO picks the tensor cores for FP32, BF16 and FP8 A whose rows TMA can address:
// split-operand FP32-class products for FP32 A, BF16 products for BF16 / FP8 A
int pick_mma(int a_dtype, int mma, bool tma_ok = true) {
  if (a_dtype == CORUTV_F64) return CORUTV_MMA_SIMT;
  if (mma != CORUTV_MMA_AUTO) return mma;
  if (!tma_ok) return CORUTV_MMA_SIMT;
  return a_dtype == CORUTV_F32 ? CORUTV_MMA_TF32X3 : CORUTV_MMA_BF16X2;
}


inline bool tma_rows_ok(const void* A, int64_t lda, int a_dtype) {
  return aligned16(A) && (lda * elem_bytes(a_dtype)) % 16 == 0;
}

int run_pass(corutv_handle* h, int dir, int a_dtype, int mma, const void* A, int64_t lda, int64_t m, int64_t n,
             const float* scales, const void* Xt, int64_t ldx, int l, void* Ct, int64_t ldc, void* partials,
             float* Xr, int64_t ldr, double* fro_parts, int phase = kPhPass, bool x_rounded = false) {
  PassArgs a{};
  a.A = A;
  a.lda = lda;
  a.m = m;
  a.n = n;
  a.scales = scales;
  a.scale_ld = cdiv(n, 128);
  a.Xt = Xt;
  a.ldx = ldx;
  a.l = l;
  a.Ct = Ct;
  a.ldc = ldc;
  a.partials = partials;
  a.len_out = dir == CORUTV_DIR_AX ? m : n;
  a.K = dir == CORUTV_DIR_AX ? n : m;
  const int eng = pick_mma(a_dtype, mma, tma_rows_ok(A, lda, a_dtype));
  if (eng != CORUTV_MMA_SIMT && !tma_rows_ok(A, lda, a_dtype)) return CORUTV_ERR_ALIGN;
  const double bytes = (double)m * n * elem_bytes(a_dtype) + (double)l * (a.K + a.len_out) * tc_bytes(a_dtype);
  PhaseTimer tm(h, phase, bytes);
  // tracing of the resident passes: events around the pass kernel alone as well
  KernelMark km;
  if (h->tracing && phase == kPhPass) {
    km.a = ev_get(h);
    km.b = ev_get(h);
    a.kmark = &km;
  }
  struct MarkRec {
    corutv_handle* h;
    KernelMark* km;
    double bytes;
    ~MarkRec() {
      if (!km->a) return;
      if (km->state == 2) {
        h->recs.push_back(TraceRec{kPhPassKernel, km->a, km->b, bytes});
      } else {
        // no kernel ran (or the launch failed): the events go back unrecorded
        h->ev_pool.push_back(km->a);
        h->ev_pool.push_back(km->b);
      }
    }
  } mark_rec{h, &km, bytes};
  if (eng == CORUTV_MMA_SIMT) {
    if (fro_parts) return CORUTV_ERR_UNSUPPORTED;
    CU(launch_pass_simt(a, dir, a_dtype, h->sms, h->stream));
  } else if (eng == CORUTV_MMA_BF16X2) {
    if (!tc_lp_supported(dir, a_dtype, l)) return CORUTV_ERR_UNSUPPORTED;
    // the BF16 hi / lo parts of the sketch operand share the buffer of the rounded TF32 operand
    void* Xh = Xr;
    void* Xl = reinterpret_cast<char*>(Xr) + (size_t)kMaxL * ldr * 2;
    CU(launch_pass_tc_lp(a, dir, a_dtype, h->sms, h->status, fro_parts, Xh, Xl, ldr, h->stream));
    if (fro_parts) {
      sum_parts_kernel<<<1, 32, 0, h->stream>>>(fro_parts, tc_lp_grid(a.len_out, a.K, h->sms), nullptr, h->status);
      CORUTV_COUNT_LAUNCH();
      CU(cudaGetLastError());
    }
  } else if (eng == CORUTV_MMA_TF32X3) {
    if (!tc3_pass_supported(dir, a_dtype, l)) return CORUTV_ERR_UNSUPPORTED;
    // the sketch operand split into its TF32 part (first half of the operand buffer) and the
    // BF16 pairs of the cross terms (second half, 2 ldr BF16 per row)
    float* Xc = Xr + (size_t)kMaxL * ldr;
    CU(launch_split_tf32(static_cast<const float*>(Xt), ldx, Xr, Xc, ldr, l, a.K, h->stream));
    CU(launch_pass_tc3(a, dir, h->sms, h->status, fro_parts, Xr, Xc, ldr, h->stream));
    if (fro_parts) {
      sum_parts_kernel<<<1, 32, 0, h->stream>>>(fro_parts, tc3_pass_grid(a.len_out, a.K, h->sms), nullptr,
                                                h->status);
      CORUTV_COUNT_LAUNCH();
      CU(cudaGetLastError());
    }
  } else {
    if (!tc_pass_supported(dir, a_dtype, eng, l)) return CORUTV_ERR_UNSUPPORTED;
    if (eng == CORUTV_MMA_TF32) {
      // the sketch operand rounded to TF32 (nearest) once per pass -- already done by its producer
      // when x_rounded; A is rounded tile by tile in the kernel
      if (!x_rounded) CU(launch_round_tf32(static_cast<const float*>(Xt), ldx, Xr, ldr, l, a.K, h->stream));
      a.Xt = Xr;
      a.ldx = ldr;
    }
    CU(launch_pass_tc(a, dir, a_dtype, eng, h->sms, h->status, fro_parts, h->stream));
    if (fro_parts) {
      sum_parts_kernel<<<1, 32, 0, h->stream>>>(fro_parts, tc_pass_grid(a.len_out, a.K, h->sms), nullptr,
                                                h->status);
      CORUTV_COUNT_LAUNCH();
      CU(cudaGetLastError());
    }
  }
  return CORUTV_OK;
}

// A held in host memory (Grace LPDDR, read over NVLink-C2C) instead of HBM: every pass
// streams it through the handle's ring, one row chunk at a time -- the externally stored
// matrix of Sec. I that the method reads only 2q + 3 times (Sec. IV-C).
struct HostSrc {
  const char* A;            // host, row-major, pitch lda elements
  int64_t lda;
  int es;                   // bytes per element
  int64_t chunk;            // rows per chunk (a multiple of 128)
  int64_t ldd;              // pitch of a ring buffer (elements; 16-byte rows for TMA)
  char* buf[HostRing::kBufs];
  void* acc;                // ATY: the product of one chunk, added into the output
  double* fro_chunk;        // ||A_c||_F^2 of every chunk (first pass, on request)
  int64_t seq = 0;          // chunks issued so far: the ring position
  double h2d_bytes = 0.0;
};

// One pass over A: resident (run_pass) or streamed chunk by chunk.  For a chunk of rows
// [r0, r0 + rows): A X gives columns r0.. of the ST output directly; A^T Y takes columns
// r0.. of the ST operand Y and its product is summed over the chunks.  The copy of chunk
// c + 1 (and c + 2) runs on the copy stream while the pass reads chunk c.
template <typename TC>
int do_pass(corutv_handle* h, HostSrc* hs, const Plan& pl, int dir, int a_dtype, int mma, const void* A, int64_t lda,
            int64_t m, int64_t n, const float* scales, TC* Xt, int64_t ldx, int l, TC* Ct, int64_t ldc, float* Xr,
            int64_t ldr, double* fro_parts, int phase, bool x_rounded, bool chunk_fro2 = false) {
  if (!hs)
    return run_pass(h, dir, a_dtype, mma, A, lda, m, n, scales, Xt, ldx, l, Ct, ldc, pl.partials, Xr, ldr, fro_parts,
                    phase, x_rounded);
  HostRing& R = h->ring;
  int64_t c = 0;
  for (int64_t r0 = 0; r0 < m; r0 += hs->chunk, ++c) {
    const int64_t rows = std::min(hs->chunk, m - r0);
    const int b = (int)(hs->seq % HostRing::kBufs);
    if (hs->seq >= HostRing::kBufs) CU(cudaStreamWaitEvent(R.copy, R.freed[b], 0));
    CU(cudaMemcpy2DAsync(hs->buf[b], (size_t)hs->ldd * hs->es, hs->A + (size_t)r0 * hs->lda * hs->es,
                         (size_t)hs->lda * hs->es, (size_t)n * hs->es, (size_t)rows, cudaMemcpyHostToDevice, R.copy));
    CU(cudaEventRecord(R.filled[b], R.copy));
    CU(cudaStreamWaitEvent(h->stream, R.filled[b], 0));
    int rc;
    if (dir == CORUTV_DIR_AX) {
      rc = run_pass(h, dir, a_dtype, mma, hs->buf[b], hs->ldd, rows, n, nullptr, Xt, ldx, l, Ct + r0, ldc,
                    pl.partials, Xr, ldr, nullptr, phase, x_rounded);
    } else {
      TC* out = r0 == 0 ? Ct : static_cast<TC*>(hs->acc);
      rc = run_pass(h, dir, a_dtype, mma, hs->buf[b], hs->ldd, rows, n, nullptr, Xt + r0, ldx, l, out, ldc,
                    pl.partials, Xr ? Xr + r0 : nullptr, ldr, nullptr, phase, x_rounded);
      if (!rc && r0 > 0) CU(launch_add_st<TC>(static_cast<const TC*>(hs->acc), ldc, l, n, Ct, ldc, h->stream));
    }
    if (rc) return rc;
    if (chunk_fro2)
      CU(launch_fro2(a_dtype, hs->buf[b], hs->ldd, rows, n, nullptr, 0, pl.fro_parts, pl.fparts, hs->fro_chunk + c,
                     h->stream));
    CU(cudaEventRecord(R.freed[b], h->stream));
    ++hs->seq;
    hs->h2d_bytes += (double)rows * n * hs->es;
  }
  if (chunk_fro2) {
    sum_parts_kernel<<<1, 32, 0, h->stream>>>(hs->fro_chunk, (int)c, nullptr, pl.status);
    CORUTV_COUNT_LAUNCH();
    CU(cudaGetLastError());
  }
  return CORUTV_OK;
}

// Shifted CholeskyQR on an ST block (in place).  passes = 3: shifted
// CholeskyQR3, Q with orthonormal columns; on the FP32 path the third pass is
// skipped when the Gram matrix of the second pass's Q is the identity within
// kSkipTol32.  passes = 1: one shifted pass, Q spans range(C) and is well
// conditioned (used for the sketches the power iteration only multiplies
// again).  R_out (may be null): the product R = R_3 R_2 R_1 with C = Q R (FP64,
// ld l); it uses the D and Qt scratch blocks, free outside a solve.
// round_out (FP32, may be null): the last pass also writes Q rounded to TF32 (ld ldr), the
// operand of the next TF32 pass.  tc_gram: the sketches come from tensor-core passes (TF32 or
// BF16 products, relative errors >= 2^-17), so the shifted first pass may form its Gram from the
// 3xTF32 tensor-core partials (~1e-6); every other Gram uses FP32 products.
// small64 (FP32 blocks): the Gram partials are reduced in FP64 and factored by the FP64
// Cholesky (R^-1 rounded to FP32 for Q = C R^-1); the shift and the dependence threshold stay
// those of FP32 products, and every pass is factored (no early exit of the third).
template <typename TC>
int orth_st(corutv_handle* h, TC* Ct, int64_t ldc, int64_t len, int l, const Plan& pl, int passes, double* Rout,
            float* round_out = nullptr, int64_t ldr = 0, bool tc_gram = false, bool small64 = false) {
  const bool f64 = sizeof(TC) == 8;
  PhaseTimer tm(h, kPhOrth);
  if constexpr (sizeof(TC) == 4) {
    if (small64) {
      for (int pass = 0; pass < passes; ++pass) {
        CU((launch_gram_auto<float, double>(Ct, ldc, Ct, ldc, len, l, static_cast<float*>(pl.gram_parts), h->sms,
                                            pl.status, static_cast<double*>(pl.G), kMaxL, h->stream,
                                            tc_gram && pass == 0)));
        double* rpass = Rout ? (pass == 0 ? Rout : static_cast<double*>(pl.D)) : nullptr;
        CU(launch_cholinv_f64<float>(static_cast<const double*>(pl.G), kMaxL, l, pass == 0 ? kShiftRel32 : 0.0,
                                     kTolRel32, static_cast<float*>(pl.R), static_cast<float*>(pl.Rinv), pl.defic,
                                     pl.status, rpass, h->stream));
        CU(launch_lmul<float>(Ct, ldc, len, l, static_cast<const float*>(pl.Rinv), kMaxL, Ct, ldc, false, pl.defic,
                              pass, nullptr, pass == passes - 1 ? round_out : nullptr, ldr, h->stream));
        if (Rout && pass > 0) {
          CU(launch_upper_mul(static_cast<const double*>(pl.D), Rout, static_cast<double*>(pl.Qt), l, h->stream));
          CU(cudaMemcpyAsync(Rout, pl.Qt, sizeof(double) * l * l, cudaMemcpyDeviceToDevice, h->stream));
        }
      }
      return CORUTV_OK;
    }
  }
  for (int pass = 0; pass < passes; ++pass) {
    // Only the shifted first pass may take the tensor-core Gram: its shift (kShiftRel32 trace(G))
    // dominates the 3xTF32 error, so R stays well defined.  The unshifted passes factor the Gram
    // of an already-processed basis whose smallest eigenvalues reach ~1e-7 of the largest once the
    // power steps have sharpened the spectrum; there the tensor core's accumulation error is of the
    // same size and would spoil R (and with it the range), so those Grams use FP32 products.
    CU((launch_gram_auto<TC, TC>(Ct, ldc, Ct, ldc, len, l, static_cast<TC*>(pl.gram_parts), h->sms, pl.status,
                                 static_cast<TC*>(pl.G), kMaxL, h->stream, tc_gram && pass == 0)));
    const double shift = pass == 0 ? (f64 ? kShiftRel64 : kShiftRel32) : 0.0;
    const double tol = f64 ? kTolRel64 : kTolRel32;
    int* skip = (!f64 && passes == 3 && pass == 2) ? &pl.status->orth_skip : nullptr;
    double* rpass = Rout ? (pass == 0 ? Rout : static_cast<double*>(pl.D)) : nullptr;
    CU(launch_cholinv<TC>(static_cast<const TC*>(pl.G), kMaxL, l, shift, tol, static_cast<TC*>(pl.R), static_cast<TC*>(pl.Rinv), pl.defic,
                          pl.status, rpass, skip, kSkipTol32, h->stream));
    CU(launch_lmul<TC>(Ct, ldc, len, l, static_cast<const TC*>(pl.Rinv), kMaxL, Ct, ldc, false, pl.defic, pass,
                       skip, pass == passes - 1 ? round_out : nullptr, ldr, h->stream));
    if (Rout && pass > 0) {
      // R <- R_pass R
      CU(launch_upper_mul(static_cast<const double*>(pl.D), Rout, static_cast<double*>(pl.Qt), l, h->stream));
      CU(cudaMemcpyAsync(Rout, pl.Qt, sizeof(double) * l * l, cudaMemcpyDeviceToDevice, h->stream));
    }
  }
  return CORUTV_OK;
}

// CholeskyQR passes for the sketches of power step `it`: the last step's sketches
// become Q1 and Q2 and are orthonormalised in full; earlier ones only feed the next
// product, which needs a well-conditioned basis of the same range (one shifted pass),
// unless the caller asks for ORTH_STRICT.
int orth_passes(const corutv_params* p, int it) {
  return (it == p->q || p->orth == CORUTV_ORTH_STRICT) ? 3 : 1;
}

// The steps of one solve, as labelled below: S0 stage Psi; S1 C1 = op1(A) X (Alg. 3 step 3); S2 orthonormalise
// C1; S3 C2 = op2(A) Q1, the other direction (Alg. 3 step 4); S4 orthonormalise C2; S5 the core D = Q1^T A Q2
// (Alg. 2 step 5); S6 QRCP (or QLP) of D (Alg. 2 step 6); S7 U, V and T (Alg. 2 step 7); S9 the readout
// ||A||_F^2 (with ||T||_F^2 it gives ||A - U T V^T||_F^2 for the exact core).
// A_ref (FP32, lda_ref) non-null: correction pass -- the core D of S5 is computed from A_ref
// with the Q1, Q2 found by the passes over A (stored in BF16 / FP8), and ||A_ref||_F^2 is the
// readout.
template <typename TC>
int solve_impl(corutv_handle* h, const corutv_params* p, const Plan& pl, const void* A, int64_t lda,
               const float* scales, const float* A_ref, int64_t lda_ref, const void* Phi, int64_t ldphi, void* U,
               int64_t ldu, double* T, int64_t ldt, void* V, int64_t ldv, int32_t* perm, HostSrc* hs = nullptr) {
  const bool right = p->side == CORUTV_SIDE_RIGHT;
  const int l = p->l;
  // RIGHT: first product A X (dir AX), second A^T Q1 (dir ATY); LEFT: swapped.
  const int dir1 = right ? CORUTV_DIR_AX : CORUTV_DIR_ATY;
  const int dir2 = right ? CORUTV_DIR_ATY : CORUTV_DIR_AX;
  TC* P1 = static_cast<TC*>(pl.P1);
  TC* P2 = static_cast<TC*>(pl.P2);
  TC* P3 = static_cast<TC*>(pl.P3);
  int passes = 0;

  CU(cudaMemsetAsync(pl.status, 0, sizeof(DevStatus), h->stream));
  // TF32 passes over A: the producers of each sketch operand (the staging of Psi, the last
  // CholeskyQR pass) also write its TF32-rounded copy into Xr for the next pass
  const int eng = pick_mma(p->a_dtype, p->mma, tma_rows_ok(A, lda, p->a_dtype));
  // ORTH_LITERAL (Alg. 3 as printed): no orthonormalisation between the products, so the passes
  // round their own (raw) sketch operands
  const bool literal = p->orth == CORUTV_ORTH_LITERAL;
  const bool pre_round = sizeof(TC) == 4 && eng == CORUTV_MMA_TF32 && !literal;
  float* Xr = static_cast<float*>(pl.Xr);
  float* Xr_out = pre_round ? Xr : nullptr;
  // Gram engine: the 3xTF32 tensor-core partials where the passes themselves run on the tensor cores
  const bool tc_gram = sizeof(TC) == 4 && (eng == CORUTV_MMA_TF32 || eng == CORUTV_MMA_TF32_TRUNC ||
                                           eng == CORUTV_MMA_TF32X3 || eng == CORUTV_MMA_BF16X2);
  // FP32-path sketches with FP64 small factorisations: FP64 Gram reductions, Cholesky, core and QRCP
  const bool small64 = sizeof(TC) == 4 && p->small_f64 != 0;
  {
    // S0: stage Psi^T into P2 (the "X" of the first product)
    PhaseTimer tm(h, kPhAsm);
    CU(launch_stage_transpose<TC>(static_cast<const TC*>(Phi), ldphi, pl.len2, l, P2, pl.ld2, Xr_out, pl.ldr,
                                  h->stream));
  }
  // S9: ||A||_F^2 fused into the first pass where the tensor-core engine runs it
  const int ref_mma = p->mma == CORUTV_MMA_SIMT ? CORUTV_MMA_SIMT : CORUTV_MMA_AUTO;
  const bool fuse_fro2 =
      !hs && p->want_fro2 && (A_ref ? pick_mma(CORUTV_F32, ref_mma, tma_rows_ok(A_ref, lda_ref, CORUTV_F32))
                             : pick_mma(p->a_dtype, p->mma, tma_rows_ok(A, lda, p->a_dtype))) != CORUTV_MMA_SIMT;
  for (int it = 0; it <= p->q; ++it) {
    // S1: C1 = A X  (Alg. 3 step 3)
    int rc = do_pass<TC>(h, hs, pl, dir1, p->a_dtype, p->mma, A, lda, p->m, p->n, scales, P2, pl.ld2, l, P1,
                         pl.ld1, Xr, pl.ldr, (it == 0 && fuse_fro2 && !A_ref) ? pl.fro_parts : nullptr, kPhPass,
                         pre_round, hs && it == 0 && p->want_fro2);
    if (rc) return rc;
    ++passes;
    // S2: orth(C1) (literal: C1 stays as it is)
    if (!literal) {
      rc = orth_st<TC>(h, P1, pl.ld1, pl.len1, l, pl, orth_passes(p, it), nullptr, Xr_out, pl.ldr, tc_gram,
                       small64);
      if (rc) return rc;
    }
    // S3: C2 = A^T Q1  (Alg. 3 step 4; literal: A^T C1)
    rc = do_pass<TC>(h, hs, pl, dir2, p->a_dtype, p->mma, A, lda, p->m, p->n, scales, P1, pl.ld1, l, P2, pl.ld2,
                     Xr, pl.ldr, nullptr, kPhPass, pre_round);
    if (rc) return rc;
    ++passes;
    if (it == p->q && p->core == CORUTV_CORE_SKETCH)
      CU(cudaMemcpy2DAsync(P3, pl.ld3 * sizeof(TC), P2, pl.ld2 * sizeof(TC), pl.len2 * sizeof(TC), l,
                           cudaMemcpyDeviceToDevice, h->stream));
    // S4: orth(C2) (literal: only after the last step)
    if (!literal) {
      rc = orth_st<TC>(h, P2, pl.ld2, pl.len2, l, pl, orth_passes(p, it), nullptr, Xr_out, pl.ldr, tc_gram,
                       small64);
      if (rc) return rc;
    }
  }
  if (literal) {
    // Alg. 3 step 6: Q1, Q2 from the last C1, C2 (shifted CholeskyQR3)
    int rc = orth_st<TC>(h, P1, pl.ld1, pl.len1, l, pl, 3, nullptr, nullptr, pl.ldr, tc_gram, small64);
    if (!rc) rc = orth_st<TC>(h, P2, pl.ld2, pl.len2, l, pl, 3, nullptr, nullptr, pl.ldr, tc_gram, small64);
    if (rc) return rc;
  }
  // S5: core D = Q1^T A Q2 (Alg. 2 step 5); small64: D reduced in FP64
  auto core_gram = [&](const TC* X, int64_t ldx, const TC* Y, int64_t ldy, int64_t len) -> cudaError_t {
    if constexpr (sizeof(TC) == 4) {
      if (small64)
        return launch_gram_auto<float, double>(X, ldx, Y, ldy, len, l, static_cast<float*>(pl.gram_parts), h->sms,
                                               pl.status, static_cast<double*>(pl.D), kMaxL, h->stream, tc_gram);
    }
    return launch_gram_auto<TC, TC>(X, ldx, Y, ldy, len, l, static_cast<TC*>(pl.gram_parts), h->sms, pl.status,
                                    static_cast<TC*>(pl.D), kMaxL, h->stream, tc_gram);
  };
  if (A_ref) {
    // correction pass: E = A_ref Q2 over the FP32 matrix (||A_ref||^2 fused where the tensor cores run it)
    int rc = run_pass(h, dir1, CORUTV_F32, ref_mma, A_ref, lda_ref, p->m, p->n, nullptr, P2, pl.ld2, l, P3,
                      pl.ld3, pl.partials, Xr, pl.ldr, fuse_fro2 ? pl.fro_parts : nullptr, kPhCorr);
    if (rc) return rc;
    ++passes;
    PhaseTimer tm(h, kPhCore);
    CU(core_gram(P1, pl.ld1, P3, pl.ld3, pl.len1));   // D = Q1^T E
  } else if (p->core == CORUTV_CORE_EXACT) {
    int rc = do_pass<TC>(h, hs, pl, dir1, p->a_dtype, p->mma, A, lda, p->m, p->n, scales, P2, pl.ld2, l, P3,
                         pl.ld3, Xr, pl.ldr, nullptr, kPhPass, pre_round);   // E = A Q2 (ST, len1)
    if (rc) return rc;
    ++passes;
    PhaseTimer tm(h, kPhCore);
    CU(core_gram(P1, pl.ld1, P3, pl.ld3, pl.len1));   // D = Q1^T E
  } else {
    PhaseTimer tm(h, kPhCore);
    // D = Q1^T A Q2 = (A^T Q1)^T Q2 = C2^T Q2 with the saved C2 (ST, len2)
    CU(core_gram(P3, pl.ld3, P2, pl.ld2, pl.len2));
  }
  const bool qlp = p->factor == CORUTV_FACTOR_QLP;
  {
    // S6: QRCP of D (Alg. 2 step 6); T = R~ (RIGHT) or R~^T (LEFT); small64: the FP64 QRCP of the FP64
    // D, its Q~ (FP64) in the G block
    PhaseTimer tm(h, kPhQrcp);
    if (small64)
      CU(launch_qrcp<double>(static_cast<const double*>(pl.D), kMaxL, l, p->k, static_cast<double*>(pl.G), kMaxL, T,
                             ldt, !right, perm, nullptr, pl.status, h->stream));
    else
      CU(launch_qrcp<TC>(static_cast<const TC*>(pl.D), kMaxL, l, p->k, static_cast<TC*>(pl.Qt), kMaxL, T, ldt,
                         !right && !qlp, perm, nullptr, pl.status, h->stream));
    if constexpr (sizeof(TC) == 4) {
      if (qlp) {
        // QLP: R~^T = Qh Rh; T = L = Rh^T (RIGHT) or Rh (LEFT); the Q2 side becomes Q2 P~ Qh
        CU(launch_qlp_second(T, ldt, l, p->k, static_cast<float*>(pl.G), right,
                             reinterpret_cast<int32_t*>(static_cast<float*>(pl.R)), pl.status, h->stream));
        CU(launch_perm_rows(static_cast<const float*>(pl.G), perm, l, static_cast<float*>(pl.Rinv), h->stream));
      }
    }
  }
  // S7: assembly (Alg. 2 step 7): Q1 Q~ and Q2 P~ (Q2 P~ Qh for the QLP)
  PhaseTimer tm_asm(h, kPhAsm);
  TC* out1 = static_cast<TC*>(right ? U : V);
  TC* out2 = static_cast<TC*>(right ? V : U);
  const int64_t ld1o = right ? ldu : ldv, ld2o = right ? ldv : ldu;
  if constexpr (sizeof(TC) == 4) {
    if (small64)
      CU(launch_lmul_full_f64s(P1, pl.ld1, pl.len1, l, static_cast<const double*>(pl.G), kMaxL, out1, ld1o, true,
                               h->stream));
  }
  if (!small64)
    CU(launch_lmul_full<TC>(P1, pl.ld1, pl.len1, l, static_cast<const TC*>(pl.Qt), kMaxL, out1, ld1o, true,
                            h->stream));
  if (qlp)
    CU(launch_lmul_full<TC>(P2, pl.ld2, pl.len2, l, static_cast<const TC*>(pl.Rinv), l, out2, ld2o, true,
                            h->stream));
  else
    CU(launch_gather_cols<TC>(P2, pl.ld2, pl.len2, l, perm, out2, ld2o, h->stream));
  // S9: ||A||_F^2 on request
  if (p->want_fro2 && !fuse_fro2 && !hs) {
    const int fdt = A_ref ? CORUTV_F32 : p->a_dtype;
    PhaseTimer tm(h, kPhFro2, (double)p->m * p->n * elem_bytes(fdt));
    CU(launch_fro2(fdt, A_ref ? static_cast<const void*>(A_ref) : A, A_ref ? lda_ref : lda, p->m, p->n,
                   A_ref ? nullptr : scales, cdiv(p->n, 128), pl.fro_parts, pl.fparts, &pl.status->fro2_A,
                   h->stream));
    ++passes;
  }
  h->last_passes = passes;
  h->last_shift = sizeof(TC) == 8 ? kShiftRel64 : kShiftRel32;
  return CORUTV_OK;
}

constexpr int64_t kRingChunkBytes = 256ll << 20;   // default chunk of a host-streamed A

// Direct device reads of page-locked host memory (through its host address, which the
// device can dereference): 16-byte loads in a grid-stride loop, folded into one word per
// block so the loads are not removed.  The rate of the host link seen by a kernel, beside
// the copy engine's (cudaMemcpyAsync) used by the host-streamed passes.
__device__ unsigned long long g_host_read_sink;
__global__ void __launch_bounds__(512) host_read_kernel(const uint4* __restrict__ src, int64_t n16) {
  uint32_t acc = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n16; i += (int64_t)gridDim.x * blockDim.x) {
    const uint4 v = src[i];
    acc ^= v.x ^ v.y ^ v.z ^ v.w;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc ^= __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc == 0x9E3779B9u) atomicAdd(&g_host_read_sink, 1ull);
}

int ensure_ring(corutv_handle* h, size_t need) {
  HostRing& R = h->ring;
  if (!R.copy) {
    if (cudaStreamCreateWithFlags(&R.copy, cudaStreamNonBlocking) != cudaSuccess) return CORUTV_ERR_CUDA;
    for (int b = 0; b < HostRing::kBufs; ++b)
      if (cudaEventCreateWithFlags(&R.filled[b], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&R.freed[b], cudaEventDisableTiming) != cudaSuccess)
        return CORUTV_ERR_CUDA;
    if (cudaEventCreateWithFlags(&R.start, cudaEventDisableTiming) != cudaSuccess) return CORUTV_ERR_CUDA;
  }
  if (R.mem && R.bytes >= need) return CORUTV_OK;
  if (R.mem) {
    cudaStreamSynchronize(h->stream);
    cudaStreamSynchronize(R.copy);
    cudaFree(R.mem);
    R.mem = nullptr;
    R.bytes = 0;
  }
  if (cudaMalloc(&R.mem, need) != cudaSuccess) {
    cudaGetLastError();
    R.mem = nullptr;
    return CORUTV_ERR_OOM;
  }
  R.bytes = need;
  return CORUTV_OK;
}

}  // namespace

void ring_free(corutv_handle* h) {
  HostRing& R = h->ring;
  if (R.copy) cudaStreamSynchronize(R.copy);
  if (R.mem) cudaFree(R.mem);
  for (int b = 0; b < HostRing::kBufs; ++b) {
    if (R.filled[b]) cudaEventDestroy(R.filled[b]);
    if (R.freed[b]) cudaEventDestroy(R.freed[b]);
  }
  if (R.start) cudaEventDestroy(R.start);
  if (R.copy) cudaStreamDestroy(R.copy);
  R = HostRing{};
}

// =============================================================================== exported
extern "C" {

int corutv_version(void) { return CORUTV_ABI_VERSION; }

const char* corutv_status_string(int s) {
  switch (s) {
    case CORUTV_OK: return "ok";
    case CORUTV_ERR_INVALID_ARG: return "invalid argument";
    case CORUTV_ERR_SHAPE: return "invalid shape";
    case CORUTV_ERR_ALIGN: return "misaligned pointer or row pitch";
    case CORUTV_ERR_OOM: return "out of device memory / workspace too small";
    case CORUTV_ERR_CUDA: return "CUDA error";
    case CORUTV_ERR_TIMEOUT: return "device wait timed out";
    case CORUTV_ERR_CHOL_BREAKDOWN: return "Cholesky breakdown";
    case CORUTV_ERR_BUSY: return "busy";
    case CORUTV_PENDING: return "pending";
    case CORUTV_ERR_UNSUPPORTED: return "unsupported combination";
    default: return "unknown status";
  }
}

int corutv_create(corutv_handle** out, void* stream) {
  if (!out) return CORUTV_ERR_INVALID_ARG;
  *out = nullptr;
  corutv_handle* h = new (std::nothrow) corutv_handle();
  if (!h) return CORUTV_ERR_OOM;
  h->stream = static_cast<cudaStream_t>(stream);
  if (cudaGetDevice(&h->device) != cudaSuccess || device_sms(&h->sms) != CORUTV_OK) {
    delete h;
    return CORUTV_ERR_CUDA;
  }
  *out = h;
  return CORUTV_OK;
}

int corutv_destroy(corutv_handle* h) {
  if (!h) return CORUTV_ERR_INVALID_ARG;
  cudaStreamSynchronize(h->stream);
  if (h->own_ws && h->ws) cudaFree(h->ws);
  for (const TraceRec& r : h->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  batch_state_free(h->batch);
  rpca_free(h);
  ring_free(h);
  resid_free(h);
  delete h;
  return CORUTV_OK;
}

int corutv_set_stream(corutv_handle* h, void* stream) {
  if (!h) return CORUTV_ERR_INVALID_ARG;
  h->stream = static_cast<cudaStream_t>(stream);
  return CORUTV_OK;
}

int corutv_workspace_size(const corutv_params* p, size_t* bytes) {
  if (!bytes) return CORUTV_ERR_INVALID_ARG;
  int rc = check_params(p);
  if (rc) return rc;
  int sms = 0;
  rc = device_sms(&sms);
  if (rc) return rc;
  Plan pl{};
  make_plan(p, sms, pl);
  *bytes = plan_layout(pl, nullptr);
  return CORUTV_OK;
}

int corutv_set_workspace(corutv_handle* h, void* dptr, size_t bytes) {
  if (!h) return CORUTV_ERR_INVALID_ARG;
  if (dptr && ((uintptr_t)dptr % kAlign)) return CORUTV_ERR_ALIGN;
  cudaStreamSynchronize(h->stream);
  if (h->own_ws && h->ws) cudaFree(h->ws);
  h->ws = dptr;
  h->ws_bytes = dptr ? bytes : 0;
  h->own_ws = false;
  if (dptr && cudaMemsetAsync(dptr, 0, bytes, h->stream) != cudaSuccess) return CORUTV_ERR_CUDA;
  return CORUTV_OK;
}

static int solve_common(corutv_handle* h, const corutv_params* p, const void* A, int64_t lda,
                        const float* a_tile_scales, const float* A_ref, int64_t lda_ref, const void* Phi,
                        int64_t ldphi, void* U, int64_t ldu, double* T, int64_t ldt, void* V, int64_t ldv,
                        int32_t* perm) {
  if (!h) return CORUTV_ERR_INVALID_ARG;
  int rc = check_params(p);
  if (rc) return rc;
  if (!A || !Phi || !U || !T || !V || !perm) return CORUTV_ERR_INVALID_ARG;
  if (p->a_dtype == CORUTV_FP8_E4M3 && !a_tile_scales) return CORUTV_ERR_INVALID_ARG;
  const int l = p->l;
  if (lda < p->n || ldphi < l || ldu < l || ldt < l || ldv < l) return CORUTV_ERR_SHAPE;
  if (pick_mma(p->a_dtype, p->mma, tma_rows_ok(A, lda, p->a_dtype)) != CORUTV_MMA_SIMT &&
      !tma_rows_ok(A, lda, p->a_dtype))
    return CORUTV_ERR_ALIGN;
  if (A_ref && lda_ref < p->n) return CORUTV_ERR_SHAPE;
  Plan pl{};
  make_plan(p, h->sms, pl);
  const size_t need = plan_layout(pl, nullptr);
  rc = ensure_workspace(h, need);
  if (rc) return rc;
  plan_layout(pl, h->ws);
  h->status = pl.status;
  h->last = *p;
  h->have_last = true;
  const int64_t l0 = launch_counter();
  if (p->a_dtype == CORUTV_F64)
    rc = solve_impl<double>(h, p, pl, A, lda, a_tile_scales, nullptr, 0, Phi, ldphi, U, ldu, T, ldt, V, ldv, perm);
  else
    rc = solve_impl<float>(h, p, pl, A, lda, a_tile_scales, A_ref, lda_ref, Phi, ldphi, U, ldu, T, ldt, V, ldv,
                           perm);
  h->launches += launch_counter() - l0;
  if (h->tracing) h->acc.solves += 1;
  return rc;
}

int corutv_solve(corutv_handle* h, const corutv_params* p, const void* A, int64_t lda, const float* a_tile_scales,
                 const void* Phi, int64_t ldphi, void* U, int64_t ldu, double* T, int64_t ldt, void* V, int64_t ldv,
                 int32_t* perm) {
  return solve_common(h, p, A, lda, a_tile_scales, nullptr, 0, Phi, ldphi, U, ldu, T, ldt, V, ldv, perm);
}

int corutv_solve_corrected(corutv_handle* h, const corutv_params* p, const void* A, int64_t lda,
                           const float* a_tile_scales, const float* A_ref, int64_t lda_ref, const void* Phi,
                           int64_t ldphi, void* U, int64_t ldu, double* T, int64_t ldt, void* V, int64_t ldv,
                           int32_t* perm) {
  if (!p || !A_ref) return CORUTV_ERR_INVALID_ARG;
  if (p->a_dtype != CORUTV_BF16 && p->a_dtype != CORUTV_FP8_E4M3) return CORUTV_ERR_INVALID_ARG;
  if (p->core != CORUTV_CORE_EXACT) return CORUTV_ERR_INVALID_ARG;
  return solve_common(h, p, A, lda, a_tile_scales, A_ref, lda_ref, Phi, ldphi, U, ldu, T, ldt, V, ldv, perm);
}

int corutv_solve_host(corutv_handle* h, const corutv_params* p, const void* A, int64_t lda, int64_t chunk_rows,
                      const void* Phi, int64_t ldphi, void* U, int64_t ldu, double* T, int64_t ldt, void* V,
                      int64_t ldv, int32_t* perm) {
  if (!h) return CORUTV_ERR_INVALID_ARG;
  int rc = check_params(p);
  if (rc) return rc;
  if (p->a_dtype != CORUTV_F32 && p->a_dtype != CORUTV_F64) return CORUTV_ERR_UNSUPPORTED;
  if (!A || !Phi || !U || !T || !V || !perm) return CORUTV_ERR_INVALID_ARG;
  const int l = p->l;
  if (lda < p->n || ldphi < l || ldu < l || ldt < l || ldv < l) return CORUTV_ERR_SHAPE;
  if (chunk_rows < 0 || chunk_rows % 128) return CORUTV_ERR_SHAPE;
  const int es = elem_bytes(p->a_dtype);
  const int64_t ldd = round_up(p->n, 16 / es);   // 16-byte rows: TMA reads the ring buffers
  int64_t chunk = chunk_rows;
  if (chunk == 0) chunk = std::max<int64_t>(128, kRingChunkBytes / (ldd * es) / 128 * 128);
  chunk = std::min(chunk, round_up(p->m, 128));
  const int64_t nchunks = cdiv(p->m, chunk);
  Plan pl{};
  make_plan(p, h->sms, pl);
  pl.pass_partials = std::max(pl.pass_partials, pass_partial_bytes(chunk, p->n, l, p->a_dtype, h->sms));
  rc = ensure_workspace(h, plan_layout(pl, nullptr));
  if (rc) return rc;
  plan_layout(pl, h->ws);
  // the ring: kBufs chunk buffers, the accumulator of the A^T Y products, one double per chunk
  const size_t buf_bytes = (size_t)round_up(chunk * ldd * es, kAlign);
  const size_t acc_bytes = (size_t)round_up((int64_t)kMaxL * pl.ld3 * tc_bytes(p->a_dtype), kAlign);
  rc = ensure_ring(h, HostRing::kBufs * buf_bytes + acc_bytes + sizeof(double) * nchunks);
  if (rc) return rc;
  HostRing& R = h->ring;
  HostSrc hs{};
  hs.A = static_cast<const char*>(A);
  hs.lda = lda;
  hs.es = es;
  hs.chunk = chunk;
  hs.ldd = ldd;
  for (int b = 0; b < HostRing::kBufs; ++b) hs.buf[b] = static_cast<char*>(R.mem) + b * buf_bytes;
  hs.acc = static_cast<char*>(R.mem) + HostRing::kBufs * buf_bytes;
  hs.fro_chunk = reinterpret_cast<double*>(static_cast<char*>(hs.acc) + acc_bytes);
  h->status = pl.status;
  h->last = *p;
  h->have_last = true;
  // the copies of this solve wait for the work already on the solve's stream: an earlier
  // solve may still be reading the ring
  CU(cudaEventRecord(R.start, h->stream));
  CU(cudaStreamWaitEvent(R.copy, R.start, 0));
  const int64_t l0 = launch_counter();
  if (p->a_dtype == CORUTV_F64)
    rc = solve_impl<double>(h, p, pl, hs.buf[0], ldd, nullptr, nullptr, 0, Phi, ldphi, U, ldu, T, ldt, V, ldv, perm,
                            &hs);
  else
    rc = solve_impl<float>(h, p, pl, hs.buf[0], ldd, nullptr, nullptr, 0, Phi, ldphi, U, ldu, T, ldt, V, ldv, perm,
                           &hs);
  h->launches += launch_counter() - l0;
  if (h->tracing) h->acc.solves += 1;
  return rc;
}

int corutv_host_read_time(corutv_handle* h, const void* host, size_t bytes, float* ms) {
  if (!h || !host || !ms) return CORUTV_ERR_INVALID_ARG;
  if (!aligned16(host) || bytes % 16 || bytes == 0) return CORUTV_ERR_ALIGN;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, host) != cudaSuccess || at.type != cudaMemoryTypeHost) {
    cudaGetLastError();
    return CORUTV_ERR_INVALID_ARG;   // not page-locked host memory known to CUDA
  }
  const void* dev = at.devicePointer ? at.devicePointer : host;
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  CU(cudaEventRecord(e0, h->stream));
  host_read_kernel<<<4 * h->sms, 512, 0, h->stream>>>(static_cast<const uint4*>(dev), (int64_t)(bytes / 16));
  CORUTV_COUNT_LAUNCH();
  CU(cudaGetLastError());
  CU(cudaEventRecord(e1, h->stream));
  CU(cudaEventSynchronize(e1));
  CU(cudaEventElapsedTime(ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return CORUTV_OK;
}

int corutv_quantize(corutv_handle* h, int dtype, const float* A, int64_t lda, int64_t m, int64_t n, void* out,
                    int64_t ldo, float* tile_scales) {
  if (!h || !A || !out) return CORUTV_ERR_INVALID_ARG;
  if (dtype != CORUTV_BF16 && dtype != CORUTV_FP8_E4M3) return CORUTV_ERR_INVALID_ARG;
  if (dtype == CORUTV_FP8_E4M3 && !tile_scales) return CORUTV_ERR_INVALID_ARG;
  if (m <= 0 || n <= 0 || lda < n || ldo < n) return CORUTV_ERR_SHAPE;
  if (cdiv(m, 128) > 65535) return CORUTV_ERR_SHAPE;
  const int64_t l0 = launch_counter();
  {
    PhaseTimer tm(h, kPhQuant);
    CU(launch_quantize(dtype, A, lda, m, n, out, ldo, tile_scales, h->stream));
  }
  h->launches += launch_counter() - l0;
  return CORUTV_OK;
}

int corutv_info_wait(corutv_handle* h, corutv_info* out) {
  if (!h || !out) return CORUTV_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return CORUTV_ERR_CUDA;
  memset(out, 0, sizeof(*out));
  if (!h->have_last || !h->status) return CORUTV_ERR_INVALID_ARG;
  DevStatus st{};
  if (cudaMemcpy(&st, h->status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) return CORUTV_ERR_CUDA;
  out->status = (st.flags & kStatTimeout) ? CORUTV_ERR_TIMEOUT : CORUTV_OK;
  out->passes_over_A = h->last_passes;
  out->hbm_passes_over_A = h->last_passes;
  out->chol_fallbacks = st.chol_fallbacks;
  out->chol_shift_rel = h->last_shift;
  out->fro2_A = h->last.want_fro2 ? st.fro2_A : NAN;
  out->fro2_T = st.fro2_T;
  out->fro2_Tk = st.fro2_Tk;
  return CORUTV_OK;
}

int corutv_set_tracing(corutv_handle* h, int enable) {
  if (!h) return CORUTV_ERR_INVALID_ARG;
  h->tracing = enable != 0;
  return CORUTV_OK;
}

int corutv_trace_read(corutv_handle* h, corutv_trace* out) {
  if (!h || !out) return CORUTV_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return CORUTV_ERR_CUDA;
  corutv_trace t = h->acc;
  for (const TraceRec& r : h->recs) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    switch (r.phase) {
      case kPhPass: t.pass_ms += ms; t.pass_bytes += r.bytes; t.pass_launches += 1; break;
      case kPhOrth: t.orth_ms += ms; break;
      case kPhCore: t.core_ms += ms; break;
      case kPhQrcp: t.qrcp_ms += ms; break;
      case kPhAsm: t.assembly_ms += ms; break;
      case kPhFro2: t.fro2_ms += ms; break;
      case kPhCorr: t.corr_ms += ms; t.corr_bytes += r.bytes; t.corr_launches += 1; break;
      case kPhQuant: t.quant_ms += ms; break;
      case kPhPassKernel: t.pass_kernel_ms += ms; t.pass_kernel_launches += 1; break;
      default: break;
    }
    h->ev_pool.push_back(r.a);
    h->ev_pool.push_back(r.b);
  }
  h->recs.clear();
  t.launches = h->launches;
  *out = t;
  h->acc = corutv_trace{};
  h->launches = 0;
  return CORUTV_OK;
}

// ------------------------------------------------------------------ building blocks
static int block_ws(corutv_handle* h, int64_t m, int64_t n, int l, int a_dtype, Plan& pl) {
  corutv_params p{};
  p.m = m;
  p.n = n;
  p.k = 1;
  p.l = l;
  p.a_dtype = a_dtype;
  make_plan(&p, h->sms, pl);
  pl.len1 = std::max(m, n);
  pl.len2 = pl.len1;
  pl.ld1 = pl.ld2 = pl.ld3 = 64;   // sketch buffers unused by the building blocks
  pl.ldr = ld_for(std::max(m, n));
  pl.gparts = gram_parts(std::max(m, n), h->sms);
  const size_t need = plan_layout(pl, nullptr);
  int rc = ensure_workspace(h, need);
  if (rc) return rc;
  plan_layout(pl, h->ws);
  h->status = pl.status;
  // the building blocks report through the same status block as a solve
  h->have_last = true;
  h->last = corutv_params{};
  h->last_passes = 0;
  return CORUTV_OK;
}

int corutv_pass(corutv_handle* h, int dir, int a_dtype, int mma, const void* A, int64_t lda, int64_t m, int64_t n,
                const float* a_tile_scales, const void* Xt, int64_t ldx, int32_t l, void* Ct, int64_t ldc) {
  if (!h || !A || !Xt || !Ct) return CORUTV_ERR_INVALID_ARG;
  if (dir != CORUTV_DIR_AX && dir != CORUTV_DIR_ATY) return CORUTV_ERR_INVALID_ARG;
  if (a_dtype < CORUTV_F64 || a_dtype > CORUTV_FP8_E4M3 || mma < 0 || mma > CORUTV_MMA_BF16X2)
    return CORUTV_ERR_INVALID_ARG;
  if (!mma_fits_dtype(a_dtype, mma)) return CORUTV_ERR_UNSUPPORTED;
  if (a_dtype == CORUTV_FP8_E4M3 && !a_tile_scales) return CORUTV_ERR_INVALID_ARG;
  if (m <= 0 || n <= 0 || l < 1 || l > kMaxL || lda < n) return CORUTV_ERR_SHAPE;
  const int64_t klen = dir == CORUTV_DIR_AX ? n : m, olen = dir == CORUTV_DIR_AX ? m : n;
  if (ldx < klen || ldc < olen) return CORUTV_ERR_SHAPE;
  if (!aligned16(Xt) || (ldx * tc_bytes(a_dtype)) % 16) return CORUTV_ERR_ALIGN;
  if (!aligned16(Ct) || (ldc * tc_bytes(a_dtype)) % 16) return CORUTV_ERR_ALIGN;
  Plan pl{};
  int rc = block_ws(h, m, n, l, a_dtype, pl);
  if (rc) return rc;
  CU(cudaMemsetAsync(pl.status, 0, sizeof(DevStatus), h->stream));
  const int64_t l0 = launch_counter();
  rc = run_pass(h, dir, a_dtype, mma, A, lda, m, n, a_tile_scales, Xt, ldx, l, Ct, ldc, pl.partials,
                static_cast<float*>(pl.Xr), pl.ldr, nullptr);
  h->launches += launch_counter() - l0;
  h->have_last = true;
  h->last = corutv_params{};
  return rc;
}

int corutv_orthonormalize(corutv_handle* h, int dtype, void* Ct, int64_t ldc, int64_t len, int32_t l,
                          double* R_out) {
  if (!h || !Ct) return CORUTV_ERR_INVALID_ARG;
  if (dtype != CORUTV_F32 && dtype != CORUTV_F64) return CORUTV_ERR_INVALID_ARG;
  if (l < 1 || l > (dtype == CORUTV_F64 ? kMaxL64 : kMaxL) || len < l || ldc < len) return CORUTV_ERR_SHAPE;
  Plan pl{};
  int rc = block_ws(h, len, len, l, dtype, pl);
  if (rc) return rc;
  CU(cudaMemsetAsync(pl.status, 0, sizeof(DevStatus), h->stream));
  if (dtype == CORUTV_F64) return orth_st<double>(h, static_cast<double*>(Ct), ldc, len, l, pl, 3, R_out);
  return orth_st<float>(h, static_cast<float*>(Ct), ldc, len, l, pl, 3, R_out);
}

int corutv_gram(corutv_handle* h, int dtype, const void* Xt, int64_t ldx, const void* Yt, int64_t ldy, int64_t len,
                int32_t l, double* G) {
  if (!h || !Xt || !Yt || !G) return CORUTV_ERR_INVALID_ARG;
  if (dtype != CORUTV_F32 && dtype != CORUTV_F64) return CORUTV_ERR_INVALID_ARG;
  if (l < 1 || l > kMaxL || len < 1 || ldx < len || ldy < len) return CORUTV_ERR_SHAPE;
  Plan pl{};
  int rc = block_ws(h, len, len, l, dtype, pl);
  if (rc) return rc;
  if (dtype == CORUTV_F64)
    CU((launch_gram<double, double>(static_cast<const double*>(Xt), ldx, static_cast<const double*>(Yt), ldy, len, l,
                                   static_cast<double*>(pl.gram_parts), gram_parts(len, h->sms), G, l, h->stream)));
  else
    CU((launch_gram_auto<float, double>(static_cast<const float*>(Xt), ldx, static_cast<const float*>(Yt), ldy, len, l,
                                  static_cast<float*>(pl.gram_parts), h->sms, pl.status, G, l, h->stream, false)));
  return CORUTV_OK;
}

int corutv_qrcp(corutv_handle* h, int dtype, const double* D, int64_t ldd, int32_t l, int32_t k, double* Q,
                double* R, int32_t* perm, double* fro2) {
  if (!h || !D || !Q || !R || !perm) return CORUTV_ERR_INVALID_ARG;
  if (dtype != CORUTV_F32 && dtype != CORUTV_F64) return CORUTV_ERR_INVALID_ARG;
  if (l < 1 || l > (dtype == CORUTV_F64 ? kMaxL64 : kMaxL) || ldd < l || k < 0 || k > l) return CORUTV_ERR_SHAPE;
  if (dtype == CORUTV_F64)
    CU(launch_qrcp_f64io<double>(D, ldd, l, k, Q, l, R, l, perm, fro2, h->stream));
  else
    CU(launch_qrcp_f64io<float>(D, ldd, l, k, Q, l, R, l, perm, fro2, h->stream));
  return CORUTV_OK;
}

int corutv_fro2(corutv_handle* h, int a_dtype, const void* A, int64_t lda, int64_t m, int64_t n,
                const float* a_tile_scales, double* out) {
  if (!h || !A || !out) return CORUTV_ERR_INVALID_ARG;
  if (a_dtype < CORUTV_F64 || a_dtype > CORUTV_FP8_E4M3) return CORUTV_ERR_INVALID_ARG;
  if (a_dtype == CORUTV_FP8_E4M3 && !a_tile_scales) return CORUTV_ERR_INVALID_ARG;
  if (m <= 0 || n <= 0 || lda < n) return CORUTV_ERR_SHAPE;
  Plan pl{};
  int rc = block_ws(h, m, n, 1, a_dtype, pl);
  if (rc) return rc;
  CU(launch_fro2(a_dtype, A, lda, m, n, a_tile_scales, cdiv(n, 128), pl.fro_parts, pl.fparts, out, h->stream));
  return CORUTV_OK;
}

}  // extern "C"
