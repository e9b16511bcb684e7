// Internal launch interface between the C-ABI front end and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "common.cuh"

namespace corutv {

// ---------------------------------------------------------------- CholeskyQR constants
constexpr double kShiftRel32 = 1e-5;    // first CholeskyQR pass, FP32 arithmetic (relative to trace(G))
constexpr double kShiftRel64 = 1e-12;   // first CholeskyQR pass, FP64 arithmetic
constexpr double kTolRel32 = 1e-7;      // dependent-column threshold, FP32
constexpr double kTolRel64 = 1e-14;     // dependent-column threshold, FP64
// Skip the third FP32 CholeskyQR pass when max |Q^T Q - I| after the second is at most
// this: a further FP32 pass reaches ~c u32 l (1e-6 .. 1e-5 for l <= 128) and gains nothing
constexpr float kSkipTol32 = 2e-6f;

// leading dimension of skinny-transposed workspace buffers of length len
inline int64_t ld_for(int64_t len) { return round_up(len < 1 ? 1 : len, 64); }

// Kernels launched by this host thread (read around a solve for its launch count).
int64_t& launch_counter();
#define CORUTV_COUNT_LAUNCH() (++::corutv::launch_counter())

// One streaming pass over A: dir 0 (AX): Ct (l x m) = (A X)^T with Xt (l x n);
// dir 1 (ATY): Ct (l x n) = (A^T Y)^T with Xt (l x m).
// CUDA events around the main kernel of one pass (tracing): the launchers record `a` right
// before the pass kernel and `b` right after it, so the pair times that kernel alone (not the
// operand preparation or the split-tile reduction around it).
struct KernelMark {
  cudaEvent_t a = nullptr, b = nullptr;
  int state = 0;   // 0: nothing recorded, 1: started, 2: both recorded
  void start(cudaStream_t st) {
    if (a && state == 0) { cudaEventRecord(a, st); state = 1; }
  }
  void stop(cudaStream_t st) {
    if (b && state == 1) { cudaEventRecord(b, st); state = 2; }
  }
};

struct PassArgs {
  const void* A;
  int64_t lda;
  int64_t m, n;
  const float* scales;   // FP8 tile scales (ceil(m/128) x ceil(n/128)) or null
  int64_t scale_ld;      // ceil(n/128)
  const void* Xt;
  int64_t ldx;
  int l;
  void* Ct;
  int64_t ldc;
  void* partials;        // Stream-K partial slots
  int64_t len_out, K;    // AX: (m, n); ATY: (n, m)
  KernelMark* kmark;     // host-side, may be null: events around the pass kernel
};

// pass_simt.cu
int64_t simt_pass_grid(int64_t len, int64_t K, int sms);
size_t simt_pass_partial_bytes(int64_t len, int64_t K, int l, int elem_bytes, int sms);
cudaError_t launch_pass_simt(const PassArgs& a, int dir, int a_dtype, int sms, cudaStream_t st);

cudaError_t launch_streamk_reduce_f32(float* Ct, int64_t ldc, const float* P, int l, int LP, int BN, int64_t len,
                                      int64_t KB, int64_t G, cudaStream_t st);

// pass_tc.cu (tcgen05 kind::tf32 + TMA, FP32 A)
size_t tc_pass_partial_bytes(int64_t len, int64_t K, int sms);
int tc_pass_grid(int64_t len, int64_t K, int sms);
bool tc_pass_supported(int dir, int a_dtype, int mma, int l);
cudaError_t launch_pass_tc(const PassArgs& a, int dir, int a_dtype, int mma, int sms, DevStatus* status,
                           double* fro_parts, cudaStream_t st);
cudaError_t launch_round_tf32(const float* X, int64_t ldx, float* Xr, int64_t ldr, int l, int64_t len,
                              cudaStream_t st);

// pass_tc3.cu (split-operand products: a tcgen05 kind::tf32 MMA of the TF32 parts plus a kind::f16
// MMA of the BF16 cross terms; FP32 A in TMEM as the M operand; the sketch operand split into Xh
// (TF32, l rows of K, leading dimension ldxs) and Xc (BF16 pairs, l rows of 2 round_up(K, 8),
// leading dimension 2 ldxs))
size_t tc3_pass_partial_bytes(int sms);
int tc3_pass_grid(int64_t len, int64_t K, int sms);
bool tc3_pass_supported(int dir, int a_dtype, int l);
cudaError_t launch_pass_tc3(const PassArgs& a, int dir, int sms, DevStatus* status, double* fro_parts,
                            const float* Xh, const void* Xc, int64_t ldxs, cudaStream_t st);
cudaError_t launch_split_tf32(const float* X, int64_t ldx, float* Xh, void* Xc, int64_t ldr, int l, int64_t len,
                              cudaStream_t st);

// pass_tc_lp.cu (tcgen05 kind::f16 + TMA, BF16 A or FP8 A with tile scales; the FP32
// sketch operand is split into BF16 hi / lo parts Xh, Xl: l rows of K, leading dimension ldxs)
size_t tc_lp_partial_bytes(int sms);
int tc_lp_grid(int64_t len, int64_t K, int sms);
bool tc_lp_supported(int dir, int a_dtype, int l);
cudaError_t launch_pass_tc_lp(const PassArgs& a, int dir, int a_dtype, int sms, DevStatus* status,
                              double* fro_parts, void* Xh, void* Xl, int64_t ldxs, cudaStream_t st);

// quant.cu: FP32 A -> BF16, or FP8 e4m3 with one power-of-two scale per 128 x 128 tile
cudaError_t launch_quantize(int dtype, const float* A, int64_t lda, int64_t m, int64_t n, void* out, int64_t ldo,
                            float* scales, cudaStream_t st);

__global__ void sum_parts_kernel(const double* __restrict__ parts, int n, double* out, DevStatus* status);
// dst[a][t] += src[a][t], a < l, t < len (ST blocks)
template <typename TC>
cudaError_t launch_add_st(const TC* src, int64_t lds, int l, int64_t len, TC* dst, int64_t ldd, cudaStream_t st);


// small.cu
// G = X Y^T (l x l, type TG) of two ST blocks: per-CTA partials, then an ordered reduction
template <typename TC, typename TG>
cudaError_t launch_gram(const TC* Xt, int64_t ldx, const TC* Yt, int64_t ldy, int64_t len, int l, TC* parts,
                        int gparts, TG* G, int64_t ldg, cudaStream_t st);
int gram_parts(int64_t len, int sms);
// gram_tc.cu: 3xTF32 tensor-core Gram partials (FP32 ST blocks whose rows TMA can address)
int gram_tc_parts(int64_t len, int sms);
bool gram_tc_ok(const float* X, int64_t ldx, const float* Y, int64_t ldy, int l);
cudaError_t launch_gram_tc_partials(const float* X, int64_t ldx, const float* Y, int64_t ldy, int64_t len, int l,
                                    float* parts, int sms, DevStatus* status, cudaStream_t st);
// G = X Y^T choosing the engine: FP32 blocks on the tensor cores (3xTF32 partials, ~1e-6 relative)
// where TMA can read them and allow_tc, else the CUDA-core FP32 partials (~u32); then the ordered
// reduction.  parts holds at least gram_parts(len, sms) blocks of 128 x 128 TC.
template <typename TC, typename TG>
cudaError_t launch_gram_auto(const TC* Xt, int64_t ldx, const TC* Yt, int64_t ldy, int64_t len, int l, TC* parts,
                             int sms, DevStatus* status, TG* G, int64_t ldg, cudaStream_t st, bool allow_tc);
constexpr int kRedWarps = 8;   // Gram reduction: warps per CTA; a CTA reduces 32 consecutive elements
// skip_flag (FP32 only, may be null): skip the factorisation when max |G - I| <= skip_tol
// (writes *skip_flag = 1 and R_out = I); launch_lmul with the same flag then does nothing
template <typename TC>
cudaError_t launch_cholinv(const TC* G, int64_t ldg, int l, double shift_rel, double tol_rel, TC* R, TC* Rinv,
                           int* defic, DevStatus* status, double* Rout, int* skip_flag, float skip_tol,
                           cudaStream_t st);
// FP64 elimination of an FP64 Gram matrix (l <= 128); R and R^-1 written in TO (FP64, or FP32
// for FP32 sketches whose small factorisations run in FP64)
template <typename TO>
cudaError_t launch_cholinv_f64(const double* G, int64_t ldg, int l, double shift_rel, double tol_rel, TO* R,
                               TO* Rinv, int* defic, DevStatus* status, double* Rout, cudaStream_t st);
// Out = S^T In on FP32 ST blocks with a full FP64 l x l S (staged in FP32)
cudaError_t launch_lmul_full_f64s(const float* In, int64_t ldi, int64_t len, int l, const double* S, int64_t lds,
                                  float* Out, int64_t ldo, bool out_rowmajor, cudaStream_t st);
// Out = S^T In on ST blocks (S upper triangular); rows j with defic[j] set (defic may be
// null) receive the deterministic replacement vector of `pass` instead.  round_out (FP32
// only, may be null): also write the result rounded to TF32 (ld ldr), the operand of the
// next TF32 pass.
template <typename TC>
cudaError_t launch_lmul(const TC* In, int64_t ldi, int64_t len, int l, const TC* S, int64_t lds, TC* Out,
                        int64_t ldo, bool out_rowmajor, const int* defic, int pass, const int* skip_flag,
                        float* round_out, int64_t ldr, cudaStream_t st);
// Out = S^T In for a full l x l S
template <typename TC>
cudaError_t launch_lmul_full(const TC* In, int64_t ldi, int64_t len, int l, const TC* S, int64_t lds, TC* Out,
                             int64_t ldo, bool out_rowmajor, cudaStream_t st);
// C = A B for upper-triangular l x l FP64 matrices (row-major, ld l; C distinct from A, B)
cudaError_t launch_upper_mul(const double* A, const double* B, double* C, int l, cudaStream_t st);
template <typename TC>
cudaError_t launch_gather_cols(const TC* St, int64_t lds, int64_t len, int l, const int32_t* perm, TC* Out,
                               int64_t ldo, cudaStream_t st);
template <typename TC>
cudaError_t launch_stage_transpose(const TC* Phi, int64_t ldphi, int64_t len, int l, TC* Xt, int64_t ldx,
                                   float* round_out, int64_t ldr, cudaStream_t st);
// QRCP of the l x l core (TC = FP32: D and Q~ in FP32; FP64: in FP64); R (= T) is FP64
template <typename TC>
cudaError_t launch_qrcp(const TC* D, int64_t ldd, int l, int k, TC* Q, int64_t ldq, double* R, int64_t ldr,
                        bool r_transposed, int32_t* perm, double* fro2, DevStatus* status, cudaStream_t st);
// the same from an FP64 D to an FP64 Q~, with the arithmetic of TC (the building-block call)
template <typename TC>
cudaError_t launch_qrcp_f64io(const double* D, int64_t ldd, int l, int k, double* Q, int64_t ldq, double* R,
                              int64_t ldr, int32_t* perm, double* fro2, cudaStream_t st);
// QLP (second half): unpivoted QR of R~^T held in R; R receives L = Rh^T (to_lower) or Rh; Qh FP32
cudaError_t launch_qlp_second(double* R, int64_t ldr, int l, int k, float* Qh, bool to_lower, int32_t* perm_scratch,
                              DevStatus* status, cudaStream_t st);
// S[perm[j]][c] = Qh[j][c] (l x l)
cudaError_t launch_perm_rows(const float* Qh, const int32_t* perm, int l, float* S, cudaStream_t st);
cudaError_t launch_fro2(int a_dtype, const void* A, int64_t lda, int64_t m, int64_t n, const float* scales,
                        int64_t sld, double* parts, int nparts, double* out, cudaStream_t st);
int fro2_parts(int sms);

// ------------------------------------------------------------------ batched solves
// One problem of a batched solve as the grouped kernels see it (an array of these
// lives in device memory).  RIGHT: C1 = A X (dir1 = AX, len1 = m), C2 = A^T Q1
// (len2 = n); LEFT: the same on A^T.  l x l blocks are packed (ld l).
struct BatchProb {
  const void* A;
  int64_t lda;
  const float* scales;
  int64_t sld;
  const float* Phi;
  int64_t ldphi;
  float* U;
  int64_t ldu;
  double* T;
  int64_t ldt;
  float* V;
  int64_t ldv;
  int32_t* perm;
  int64_t m, n, len1, len2;
  int l, k, q, side, core, orth, want_fro2, dir1, dir2;
  float *P1, *P2, *P3;
  int64_t ld1, ld2, ld3;
  float* gparts;        // Gram partial blocks (LP x LP each)
  int gp1, gp2;         // partial blocks for sketches of length len1 / len2
  float *G, *D, *Qt;    // l x l Gram / core / Q~ (FP32)
  float *R, *Rinv;
  int* defic;
  double* fparts;       // ||A||^2 partials, one per block of the first pass
  int nfparts;
  DevStatus* status;
  int ks1, ks2;         // SIMT passes: K splits of the len1-output (C1, core) and len2-output (C2) passes
  float* kparts;        // their partial products, [split][l][len] (null when neither pass splits)
  int* kcount;          // per output tile: splits finished so far (zero between passes)
  int fuse;             // fused power steps: P2 holds W = op2(A) C1 during orth(C1)
};

// Block -> (problem, local block) maps drive every grouped launch.
enum BatchSketch : int { kB_C1 = 0, kB_C2 = 1, kB_CORE = 2 };          // pass outputs
enum BatchGram : int { kG_ORTH1 = 0, kG_ORTH2 = 1, kG_CORE_EXACT = 2, kG_CORE_SKETCH = 3,
                       kG_ORTH1_W = 4 };   // ORTH1_W: orth(C1)'s R^-1 applied to W (fused power steps)

// batched SIMT pass (pass_simt.cu): one CTA per 64 output positions and K range; a problem
// whose K exceeds 2 kBatchSplitK is split into ceil(K / kBatchSplitK) ranges (at most
// kBatchMaxSplit), summed in range order by the last CTA of each tile
constexpr int kBatchPassBN = 64;
constexpr int64_t kBatchSplitK = 2048;
constexpr int kBatchMaxSplit = 64;
inline int batch_ksplit(int64_t K, int64_t splitk = kBatchSplitK) {
  if (K <= 2 * splitk) return 1;
  const int64_t s = (K + splitk - 1) / splitk;
  return (int)(s < kBatchMaxSplit ? s : kBatchMaxSplit);
}
cudaError_t launch_pass_simt_grouped(const BatchProb* P, const int2* map, int nblocks, int lp, int a_dtype,
                                     int which, int it, cudaStream_t st);
// batched TF32 tensor-core pass (pass_tc_grouped.cu): one table entry per problem taking
// part, problems in table order, iterations (tile, k-block) concatenated
struct GPassProb {
  const void* mapA;          // CUtensorMap of A (device memory) for this problem's direction
  const void* mapX;          // CUtensorMap of Xr: l rows x K columns, box 32 x 128
  float* Ct;
  int64_t ldc;
  const float* X;            // sketch operand (ST); rounded to TF32 into Xr before the pass
  int64_t ldx;
  float* Xr;
  int64_t ldr;
  int64_t len, K, KB, tiles, iter_base, tile_base, owner_first;
  double* fro;               // 4 FP64 partials of sum(a^2) per CTA sharing the problem, or null
  int l, dir;
};
size_t tc_grouped_partial_bytes(int sms);
int64_t tc_grouped_tiles(int64_t len);
int64_t tc_grouped_kblocks(int64_t K);
int64_t tc_grouped_owner(int64_t x, int64_t total, int64_t G);
cudaError_t launch_pass_tc_grouped(const GPassProb* gp, int np, int64_t total_iters, int64_t total_tiles, int lmax,
                                   const int2* round_map, int nround, float* partials, bool fro, int sms,
                                   DevStatus* status, bool keep_a, cudaStream_t st, KernelMark* km = nullptr);

// Grouped kind::f16 passes (pass_tc_lp_grouped.cu) for batched BF16 / FP8 problems.  Work is
// cut into units that depend on the problem alone -- one 256-position output tile and one K range
// of kLpUnitK (whole 64-element k-blocks) -- so a problem's result does not depend on the other
// problems of its batch: every unit starts its TMEM accumulator from zero, and a tile cut into S
// K ranges is summed in range order by a separate reduction.  A CTA runs a contiguous run of
// units (table cta_first, balanced by k-blocks on the host).
constexpr int kLpUnitBN = 256;
constexpr int kLpUnitBK = 64;
constexpr int64_t kLpUnitK = 2048;
constexpr int kLpMaxSplit = 64;
inline int lp_unit_split(int64_t K) {
  if (K <= 2 * kLpUnitK) return 1;
  const int64_t s = (K + kLpUnitK - 1) / kLpUnitK;
  return (int)(s < kLpMaxSplit ? s : kLpMaxSplit);
}
struct GLpProb {
  const void* mapA;          // CUtensorMap of A (device memory) in this problem's direction
  const void* mapXh;         // CUtensorMaps of the BF16 parts of the sketch operand: l rows x K,
  const void* mapXl;         //   box 64 x 128, 128-byte swizzle
  float* Ct;
  int64_t ldc;
  float* kparts;             // [split][l][ldk] partial products when S > 1
  int64_t ldk;
  const float* X;            // FP32 sketch operand (ST), split into Xh / Xl before the pass
  int64_t ldx;
  void* Xh;                  // BF16, l rows, leading dimension ldxs
  void* Xl;
  int64_t ldxs;
  const float* scales;       // FP8: tile scales (srows x scols, leading dimension sld)
  int64_t sld, srows, scols;
  double* fro;               // one FP64 sum(a^2) per unit, or null
  int64_t len, K, KB, kbc;   // kbc: k-blocks per unit (the last unit of a tile may hold fewer)
  int64_t tiles, units, unit_base;
  int S, l, dir;
};
// units of one problem's pass and their k-blocks
inline int64_t lp_unit_kblocks(int64_t K) { return (K + kLpUnitBK - 1) / kLpUnitBK; }
inline int64_t lp_unit_kbc(int64_t K) {
  const int64_t KB = lp_unit_kblocks(K), S = lp_unit_split(K);
  return (KB + S - 1) / S;
}
inline int lp_unit_nsplit(int64_t K) {
  const int64_t KB = lp_unit_kblocks(K), c = lp_unit_kbc(K);
  return (int)((KB + c - 1) / c);
}
cudaError_t launch_pass_lp_grouped(const GLpProb* gp, int np, bool fp8, bool fro, const int* cta_first, int G,
                                   const int2* split_map, int nsplit, const int2* red_map, int nred, int lmax,
                                   DevStatus* status, bool keep_a, cudaStream_t st, KernelMark* km = nullptr);

// grouped small kernels (small.cu)
constexpr int kBatchGramCols = 512;   // columns per Gram partial block
constexpr int kBatchLmulBI = 128;     // columns per lmul tile
constexpr int kBatchTile32 = 32;      // columns per stage / gather / copy tile
cudaError_t launch_stage_grouped(const BatchProb* P, const int2* map32_2, int nblocks, cudaStream_t st);
cudaError_t launch_gram_grouped(const BatchProb* P, const int2* map_parts, int nparts, const int2* map_red,
                                int nred, int lp, int which, int it, int pass, cudaStream_t st);
cudaError_t launch_cholinv_grouped(const BatchProb* P, int count, int lmax, int which, int it, int pass,
                                   float skip_tol, double shift_rel, double tol_rel, cudaStream_t st);
cudaError_t launch_lmul_orth_grouped(const BatchProb* P, const int2* map, int nblocks, int lp, int which, int it,
                                     int pass, cudaStream_t st);
cudaError_t launch_copy_sketch_grouped(const BatchProb* P, const int2* map32_2, int nblocks, int it,
                                       cudaStream_t st);
cudaError_t launch_qrcp_grouped(const BatchProb* P, const int2* map, int count, int lp, cudaStream_t st);
cudaError_t launch_assemble_grouped(const BatchProb* P, const int2* map_lmul1, int n1, const int2* map32_2, int n2,
                                    int lp, cudaStream_t st);
cudaError_t launch_fro2_grouped(const BatchProb* P, int count, cudaStream_t st);

}  // namespace corutv
