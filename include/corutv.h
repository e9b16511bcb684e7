/*
 * corutv.h -- C ABI of libcorutv, a GB300 (sm_103a) implementation of the
 * hot path of Compressed Randomized UTV (CoR-UTV):
 *
 *   M. F. Kaloorazi and R. C. de Lamare, "Compressed Randomized UTV
 *   Decompositions for Low-Rank Approximations and Big Data Applications",
 *   arXiv:1810.07323.  Citations below name its sections, equations and
 *   algorithms.
 *
 * Problem (Sec. III, Alg. 2 and Alg. 3): given A (m x n), integers
 * k <= l < min(m, n), q >= 0 and a Gaussian test matrix Psi (n x l, passed in
 * by the caller), compute A ~ U T V^T with U (m x l) and V (n x l) having
 * orthonormal columns and T (l x l) triangular.
 *
 * Conventions shared by every call
 *   - Matrices are ROW-MAJOR with an explicit leading dimension (elements).
 *   - Unless stated otherwise pointers are DEVICE pointers owned by the
 *     caller; the library never frees them.  Inputs are read-only.
 *   - `stream` arguments are cudaStream_t values passed as void*.  Work is
 *     enqueued asynchronously on that stream; a call returns once the work is
 *     enqueued.  Argument checks happen first and, on failure, nothing is
 *     enqueued and the call returns the error code.
 *   - "Skinny transposed" (ST) layout: an (len x l) block held as its
 *     transpose, l rows of `len` contiguous elements, leading dimension
 *     ld >= len, ld a multiple of 4 and the base 16-byte aligned.  The
 *     building-block calls below read and write sketches in this layout.
 *   - Device-side conditions (a bounded wait that expired, a Cholesky
 *     breakdown that was repaired) are recorded in the handle's status words
 *     and returned by corutv_info_wait().
 *   - A handle must not be used from two host threads at once.
 */
#ifndef CORUTV_H
#define CORUTV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CORUTV_ABI_VERSION 8

typedef enum {
  CORUTV_OK = 0,
  CORUTV_ERR_INVALID_ARG = 1,   /* null pointer, bad enum, k/l/q out of range */
  CORUTV_ERR_SHAPE = 2,         /* l >= min(m, n), leading dimension too small, l beyond the kernel limit */
  CORUTV_ERR_ALIGN = 3,         /* base not 16-byte aligned or row pitch not a multiple of 16 bytes */
  CORUTV_ERR_OOM = 4,           /* workspace allocation failed or caller workspace too small */
  CORUTV_ERR_CUDA = 5,          /* a CUDA runtime/driver call failed */
  CORUTV_ERR_TIMEOUT = 6,       /* a device-side bounded wait expired (reported by corutv_info_wait) */
  CORUTV_ERR_CHOL_BREAKDOWN = 7,/* reserved: breakdowns are repaired, never returned by this version */
  CORUTV_ERR_BUSY = 8,          /* serving queue full */
  CORUTV_PENDING = 9,           /* serving request not finished */
  CORUTV_ERR_UNSUPPORTED = 10   /* combination not built (e.g. a dtype on a path that lacks it) */
} corutv_status;

typedef enum { CORUTV_SIDE_RIGHT = 0, CORUTV_SIDE_LEFT = 1 } corutv_side;
typedef enum { CORUTV_CORE_EXACT = 0, CORUTV_CORE_SKETCH = 1 } corutv_core;
typedef enum {
  CORUTV_ORTH_STABILISED = 0, /* the last power step's sketches (Q1, Q2) by shifted CholeskyQR3;
                                 earlier sketches by one shifted CholeskyQR pass (a well-conditioned
                                 basis of the same range: the same Q1, Q2 in exact arithmetic) */
  CORUTV_ORTH_STRICT = 1,     /* every sketch by shifted CholeskyQR3 */
  CORUTV_ORTH_LITERAL = 2     /* Alg. 3 as printed: the power steps multiply by A and A^T with no
                                 orthonormalisation in between (C1 = A C2, C2 = A^T C1), and only
                                 the last C1 and C2 are orthonormalised (shifted CholeskyQR3).  The
                                 same Q1, Q2 in exact arithmetic; in floating point the columns of
                                 C1, C2 align with the leading singular vectors as q grows, so
                                 trailing directions are lost, and the entries grow like
                                 ||A||^(2q+1) (FP32 range).  corutv_solve / corutv_solve_host with
                                 core EXACT only (SKETCH: ERR_UNSUPPORTED; batched: ERR_UNSUPPORTED) */
} corutv_orth;
typedef enum { CORUTV_F64 = 0, CORUTV_F32 = 1, CORUTV_BF16 = 2, CORUTV_FP8_E4M3 = 3 } corutv_dtype;
typedef enum {
  CORUTV_MMA_AUTO = 0,       /* F32 A: TF32X3 (split operands, FP32-class); BF16 / FP8 A: BF16X2; F64 A:
                                SIMT.  Falls back to SIMT where TMA cannot address the rows of A (see
                                corutv_solve) */
  CORUTV_MMA_TF32 = 1,       /* tcgen05 kind::tf32 with both operands rounded to nearest TF32
                                (A tile by tile in shared memory): unbiased products, ~2^-11 relative */
  CORUTV_MMA_TF32X3 = 2,     /* split-operand FP32-class products on the tensor cores: every FP32 value
                                v = h + c with h = TF32(v), c = BF16(v - h) (|v - h - c| <= 2^-19 |v|);
                                a x ~ h_a h_x (kind::tf32, exact products) + [c_a, bf16(h_a)] . [bf16(h_x),
                                c_x] (one kind::f16 MMA for both cross terms): <= 2^-16.9 relative per
                                product, then the tensor core's FP32 accumulation (measured ~1e-6 relative
                                at K = 4096, growing with K; FP32 CUDA-core products: ~2e-7) */
  CORUTV_MMA_SIMT = 3,       /* CUDA-core FMA in the storage precision (FP32 or FP64 products) */
  CORUTV_MMA_TF32_TRUNC = 4, /* tcgen05 kind::tf32 reading raw FP32 (the tensor core drops the low
                                13 mantissa bits: products shrink by ~3.5e-4 on average) */
  CORUTV_MMA_BF16X2 = 5      /* BF16 / FP8 A only: tcgen05 kind::f16 on BF16 A tiles (FP8 tiles are
                                dequantised to BF16 in shared memory, e4m3 value x tile scale, exact
                                when the scale is a power of two) against the sketch operand split
                                into BF16 hi + lo parts (~16 bits kept); FP32 accumulation */
} corutv_mma;

typedef enum { CORUTV_DIR_AX = 0, CORUTV_DIR_ATY = 1 } corutv_dir;

/* Rank-revealing factorisation of the l x l core D (Alg. 2 step 6). */
typedef enum {
  CORUTV_FACTOR_QRCP = 0,    /* D = Q~ R~ P~^T (Eq. (D = Q~ R~ P~^T)): T = R~ (URV) */
  CORUTV_FACTOR_QLP = 1      /* QLP (Stewart): the QRCP, then R~^T = Qh Rh, so D = Q~ L (P~ Qh)^T with
                                L = Rh^T: T = L lower triangular and V = Q2 P~ Qh (RIGHT; LEFT gives the
                                transposes); the diagonal of L tracks the singular values more closely.
                                FP32-path solves only (F64 returns UNSUPPORTED); perm keeps the QRCP
                                pivots */
} corutv_factor;

/* Parameters of one solve (Alg. 2 / Alg. 3). */
typedef struct {
  int64_t m, n;          /* shape of A */
  int32_t k;             /* target rank: validated (1 <= k <= l) and used for the rank-k readout */
  int32_t l;             /* sample size l, k <= l < min(m, n), l <= 128 */
  int32_t q;             /* power steps, q >= 0 (q = 0 is Alg. 2) */
  int32_t side;          /* corutv_side: RIGHT = Alg. 2/3 (Psi is n x l, T upper);
                            LEFT = the m < n modification of Sec. III: Alg. 2/3 on A^T with
                            Psi m x l (sketch A^T Psi first), T lower (ULV form) */
  int32_t core;          /* corutv_core: EXACT = one more pass, D = Q1^T (A Q2) (Alg. 2 step 5);
                            SKETCH = D = (A^T Q1)^T Q2 from the last sketch, no extra pass */
  int32_t orth;          /* corutv_orth (both orthonormalise every sketch before the next product) */
  int32_t a_dtype;       /* corutv_dtype of A (and of Psi, U, V: F64 for F64, F32 otherwise) */
  int32_t mma;           /* corutv_mma for the passes over A */
  int32_t want_fro2;     /* 1: also compute ||A||_F^2 into the info (fused into the first pass on the
                            tensor-core engine, one extra read of A otherwise) */
  int32_t factor;        /* corutv_factor of the core (QRCP by default) */
  int32_t small_f64;     /* 1: the small factorisations of an F32 / BF16 / FP8 solve in FP64 -- the
                            Gram matrices of CholeskyQR reduced in FP64 (from FP32-product partials)
                            and factored by an FP64 Cholesky, the core D reduced in FP64 and its QRCP
                            in FP64 (factor QLP: ERR_UNSUPPORTED).  0 (default): in FP32.  F64 A:
                            always FP64 */
  int32_t reserved[5];   /* must be zero */
} corutv_params;

/* Device-side outcome of the last solve on a handle. */
typedef struct {
  int32_t status;          /* corutv_status of the device work (OK or ERR_TIMEOUT) */
  int32_t passes_over_A;   /* streaming passes over A enqueued by the solve */
  int32_t chol_fallbacks;  /* sketch columns found numerically dependent and replaced */
  int32_t hbm_passes_over_A; /* of those passes, the ones that stream A from memory (HBM, or host
                              memory for corutv_solve_host) rather than re-read it from L2: fewer
                              than passes_over_A when a batched problem fuses its power steps
                              (corutv_problem.fuse_power), passes_over_A otherwise */
  double chol_shift_rel;   /* shift of the first CholeskyQR pass, relative to trace(C^T C) */
  double fro2_A;           /* ||A||_F^2 if want_fro2, else NaN */
  double fro2_T;           /* ||T||_F^2 */
  double fro2_Tk;          /* ||T(1:k, :)||_F^2 */
} corutv_info;

typedef struct corutv_handle corutv_handle;

/* ABI version (CORUTV_ABI_VERSION). */
int corutv_version(void);

/* Human-readable name of a status code (static storage). */
const char* corutv_status_string(int status);

/* Create a handle bound to `stream` (a cudaStream_t, may be NULL for the
 * legacy default stream) on the current device.  The handle owns no user
 * data; it lazily owns a device workspace unless one is set.  */
int corutv_create(corutv_handle** out, void* stream);

/* Synchronise the handle's stream and free what the handle owns. */
int corutv_destroy(corutv_handle* h);

/* Rebind the handle to another stream (work already enqueued stays where it is). */
int corutv_set_stream(corutv_handle* h, void* stream);

/* Bytes of device workspace a solve with parameters `p` needs (sketches
 * C1 (m x l) and C2 (n x l) in ST layout, the core pass product, split-K
 * partials, Gram partials, l x l factors and status words). */
int corutv_workspace_size(const corutv_params* p, size_t* bytes);

/* Use caller-owned device memory [dptr, dptr + bytes) as workspace (256-byte
 * aligned).  Passing NULL returns the handle to lazy self-allocation.  The
 * memory must stay valid until the handle's stream has finished the solves
 * that use it. */
int corutv_set_workspace(corutv_handle* h, void* dptr, size_t bytes);

/*
 * corutv_solve -- one CoR-UTV factorisation (Alg. 2 for q = 0, Alg. 3 for q >= 1).
 *
 *   A      device, m x n row-major, leading dimension lda >= n, dtype a_dtype.
 *          The tensor-core passes read A with TMA and need a 16-byte aligned base and
 *          lda * sizeof(dtype) a multiple of 16; mma = AUTO falls back to the SIMT
 *          passes when that does not hold, an explicit TF32 mode returns ERR_ALIGN.
 *   a_tile_scales  FP8 only: ceil(m/128) x ceil(n/128) float scales (row-major); element
 *          (i, j) of A is e4m3 code (i, j) times scale (i / 128, j / 128); else NULL.
 *          corutv_quantize writes both.  The FP8 tensor-core pass needs lda a multiple
 *          of 16, the BF16 one a multiple of 8 (16-byte row pitch).
 *   Phi    device, the Gaussian test matrix Psi (Sec. III): n x l (RIGHT) or m x l
 *          (LEFT) row-major, ldphi >= l, F64 for a_dtype F64 else F32.
 *   U      device out, m x l row-major (ldu >= l), same dtype as Phi.
 *   T      device out, l x l row-major FP64 (ldt >= l): upper triangular (RIGHT,
 *          URV) or lower triangular (LEFT, ULV); diag(T) >= 0, non-increasing.
 *   V      device out, n x l row-major (ldv >= l), same dtype as Phi.
 *   perm   device out, int32[l]: the QRCP pivots of the core (Sec. III, Eq. (D = Q~ R~ P~^T)).
 *          RIGHT: V[:, j] = Q2[:, perm[j]]; LEFT: U[:, j] is the permuted basis.
 *
 * Range finding is stabilised: every sketch is normalised (Sec. III, QR of
 * C1 and C2) before the next product, which in exact arithmetic yields the
 * same Q1, Q2 as the literal loop of Alg. 3.  The final Q1, Q2 come from
 * shifted CholeskyQR3 (see corutv_orth for the intermediate sketches).  The
 * small factorisations run in the precision of the sketches: FP64 A gets FP64
 * Gram matrices, Cholesky and QRCP; every other dtype gets FP32 ones -- Gram
 * partials from FP32 products (3xTF32 tensor-core products for the shifted
 * first pass and the core when the passes run on the tensor cores), reduced
 * with compensated FP32 sums -- unless p->small_f64 asks for FP64 Gram
 * reductions, Cholesky factors, core and QRCP.  On the FP32 path the third
 * CholeskyQR pass is skipped when the second already gives max |Q^T Q - I| <= 2e-6.
 * Returns a validation error synchronously; device conditions via corutv_info_wait.
 */
int corutv_solve(corutv_handle* h, const corutv_params* p,
                 const void* A, int64_t lda, const float* a_tile_scales,
                 const void* Phi, int64_t ldphi,
                 void* U, int64_t ldu, double* T, int64_t ldt,
                 void* V, int64_t ldv, int32_t* perm);

/*
 * corutv_solve_host -- corutv_solve for an A that stays in HOST memory (Grace LPDDR,
 * read over NVLink-C2C): the matrix "stored externally" of Sec. I, which the
 * method reads only 2q + 3 times (Sec. IV-C; 2q + 2 with core = SKETCH).  Every
 * pass streams A through a ring of three device buffers, chunk_rows rows at a
 * time: the copy of the next chunks runs on the handle's copy stream while the
 * pass kernels read the current one, so device memory holds three chunks, the
 * sketches and the outputs, whatever m.  A X writes each chunk's rows of the
 * sketch directly; A^T Y sums the chunks' products (one extra l x n add per chunk).
 *   A        HOST, m x n row-major, lda >= n elements, F32 or F64 (a_dtype; BF16 /
 *            FP8 return ERR_UNSUPPORTED).  Page-locked memory (cudaHostAlloc /
 *            cudaHostRegister) gives full C2C bandwidth; pageable memory works but
 *            each copy is staged by the driver.  The caller keeps A unchanged and
 *            alive until the solve is complete (corutv_info_wait or a stream sync).
 *   chunk_rows  rows per chunk, a multiple of 128 (ERR_SHAPE otherwise); 0 picks
 *            about 256 MiB per chunk.  Clamped to m rounded up to 128.
 * Phi, U, T, V, perm and the engines as corutv_solve (device); want_fro2 sums
 * ||A_c||_F^2 over the chunks of the first pass.  The device allocations (ring
 * and workspace) are made on first use and kept by the handle.
 */
int corutv_solve_host(corutv_handle* h, const corutv_params* p, const void* A, int64_t lda, int64_t chunk_rows,
                      const void* Phi, int64_t ldphi, void* U, int64_t ldu, double* T, int64_t ldt,
                      void* V, int64_t ldv, int32_t* perm);

/*
 * corutv_host_read_time -- the host link as a kernel sees it, for the host-streamed solve
 * (no counterpart in the paper): a kernel on the handle's stream reads `bytes` of
 * page-locked HOST memory directly through its address (16-byte loads over all SMs) and
 * *ms receives the kernel's duration (CUDA events; the call synchronises).  host must be
 * 16-byte aligned and bytes a non-zero multiple of 16 (ERR_ALIGN); memory that CUDA does
 * not know as page-locked host memory gives ERR_INVALID_ARG.  bytes / ms compares with
 * the copy engine's rate (cudaMemcpyAsync), which corutv_solve_host uses.
 */
int corutv_host_read_time(corutv_handle* h, const void* host, size_t bytes, float* ms);

/*
 * corutv_solve_corrected -- corutv_solve for A stored in BF16 or FP8 (a_dtype) plus
 * the FP32 correction pass: the range finding (the products of Alg. 3 steps 3-4
 * and their orthonormalisations: every pass over A but the core's) runs on the
 * low-precision A, then the core D = Q1^T A_ref Q2 (Alg. 2
 * step 5) is computed by one pass over the FP32 matrix A_ref (m x n row-major,
 * lda_ref >= n, device) with the Q1, Q2 found.  Because D is the projection of
 * A_ref onto the two bases, T then carries no storage error of A; only the
 * subspaces do.  Requires p->core == EXACT; want_fro2 reports ||A_ref||_F^2.
 * The pass over A_ref uses the FP32-class split-operand engine TF32X3 (SIMT when
 * p->mma is SIMT or TMA cannot address A_ref's rows).  Other arguments as
 * corutv_solve.
 */
int corutv_solve_corrected(corutv_handle* h, const corutv_params* p,
                           const void* A, int64_t lda, const float* a_tile_scales,
                           const float* A_ref, int64_t lda_ref,
                           const void* Phi, int64_t ldphi,
                           void* U, int64_t ldu, double* T, int64_t ldt,
                           void* V, int64_t ldv, int32_t* perm);

/*
 * corutv_quantize -- storage conversion of an FP32 A (m x n row-major, lda) for the
 * low-precision passes (no counterpart in the paper):
 *   dtype BF16: out (m x n, ldo, __nv_bfloat16) = A rounded to nearest even;
 *               tile_scales unused (may be NULL).
 *   dtype FP8_E4M3: for every 128 x 128 tile (ragged at the edges) the scale
 *               s = smallest power of two >= fl32(amax(|tile|) / 448) (s = 1 for an
 *               all-zero tile) goes to tile_scales[(i/128) * ceil(n/128) + j/128] and
 *               out (m x n, ldo bytes per row) holds e4m3(a / s), rounded to nearest
 *               even with saturation at +-448.  a / s is exact, so each entry is
 *               rounded once.
 * A must be finite.  Device pointers; enqueued on the handle's stream.
 */
int corutv_quantize(corutv_handle* h, int dtype, const float* A, int64_t lda, int64_t m, int64_t n,
                    void* out, int64_t ldo, float* tile_scales);

/* ------------------------------------------------------------------------
 * Batched solves: many independent problems of different shapes in one call.
 * ---------------------------------------------------------------------- */

/* One problem of a batched solve: the fields of corutv_params and the pointer
 * arguments of corutv_solve (same meaning, layouts and ownership). */
typedef struct {
  int64_t m, n;
  int32_t k, l, q, side, core, orth;
  int32_t a_dtype;       /* F32, BF16 or FP8_E4M3 (Psi, U, V are FP32; T FP64) */
  int32_t mma;           /* AUTO or SIMT: the batched passes run on the CUDA cores */
  int32_t want_fro2;
  int32_t fuse_power;    /* 1: fused power steps (Alg. 3 steps 3-4, read A once per step): the second
                            product of every power step is formed from the unnormalised first,
                            W = op2(A) C1, in the launch right after C1's, while A is still in L2
                            (problems are taken in groups of at most ~80 MB of A), and
                            C2 = op2(A) Q1 = W R1^-1 follows by applying the R^-1 of each
                            CholeskyQR pass of orth(C1) to W as well; A then crosses HBM
                            q + 1 (+ 1 for the exact core) times.  Exact in exact arithmetic;
                            in floating point W R1^-1 carries the rounding of W amplified by up
                            to cond(C1), so it suits well-conditioned sketches.  Tensor-core
                            engines only (ignored for problems on the CUDA cores).  0: off */
  const void* A;
  int64_t lda;
  const float* a_tile_scales;
  const void* Phi;
  int64_t ldphi;
  void* U;
  int64_t ldu;
  double* T;
  int64_t ldt;
  void* V;
  int64_t ldv;
  int32_t* perm;
  int64_t reserved[4];   /* must be zero */
} corutv_problem;

/* Device workspace a batch needs (sketches, Gram partials and l x l factors of
 * every problem, plus the grouped-launch tables). */
int corutv_batch_workspace_size(int count, const corutv_problem* probs, size_t* bytes);

/*
 * corutv_solve_batched -- `count` independent CoR-UTV solves (Alg. 2 / Alg. 3,
 * each with its own m, n, k, l, q, side, core, dtype and pointers; probs is a
 * host array).  Every step of the schedule runs as one grouped launch over all
 * problems (problems beyond their last power step skip the loop's launches),
 * so the launch count does not grow with `count`.  FP32 batches whose rows TMA
 * can address (16-byte aligned base and row pitch) run every pass as one
 * grouped TF32 tensor-core launch (mma AUTO or TF32; rounded operands, FP32
 * accumulation, problems' (tile, k-block) iterations concatenated and split
 * evenly over the SMs).  BF16 / FP8 problems whose rows TMA can address (mma
 * AUTO) run theirs as grouped kind::f16 launches of per-problem work units (a
 * 256-position tile and a K range of at most 2048, each started from zero, tiles
 * cut into several ranges summed in range order), so each such problem's result
 * is the same bits in any batch.  The rest (mma SIMT, unaligned rows) run on the
 * CUDA cores with FP32 accumulation, one CTA per 64 output positions and K range.  Orthonormalisation and QRCP as in
 * corutv_solve.  Limits: l <= 128; a_dtype F64 and the BF16X2 / TF32_TRUNC
 * modes return ERR_UNSUPPORTED (TF32 needs FP32 storage).  The handle keeps a workspace and the tables of the last
 * problem set; calling again with an identical problem array (same shapes,
 * pointers and parameters) replays a CUDA graph of the whole batch (not on the
 * legacy default stream, and not while tracing: traced runs launch directly so
 * every phase gets its own event pair).  Validation errors return synchronously and enqueue
 * nothing.  infos: NULL (the call returns once the work is enqueued; read the
 * outcome with corutv_batch_info_wait) or a host array of `count` entries (the
 * call waits for the batch and fills it).
 */
int corutv_solve_batched(corutv_handle* h, int count, const corutv_problem* probs, corutv_info* infos);

/* Synchronise the handle's stream and return the outcome of each problem of the
 * last batch (count must equal that batch's count). */
int corutv_batch_info_wait(corutv_handle* h, int count, corutv_info* infos);

/*
 * corutv_set_autotune -- shapes of the batched plan picked by measurement (no
 * counterpart in the paper).  mode 1: the first corutv_solve_batched call with a new
 * problem set (never a graph replay) runs a coordinate search -- the order of the
 * problems in the tensor-core pass tables (as given / largest reduction first), the
 * columns per Gram partial block (256, 512, 1024, 2048) and, for CUDA-core passes, the
 * K range of one split (1024, 2048, 4096) -- timing whole batches (one warm run, the
 * faster of two timed runs per candidate) and builds the plan with the fastest shapes;
 * the search's runs write the problems' outputs, which the final run then overwrites.
 * The choice is cached per key (storage dtype, pass engine, l class of the largest l,
 * power-of-two buckets of the mean m, mean n and count, largest q) in the JSON file
 * cache_path (NULL: the file named by the environment variable CORUTV_AUTOTUNE_CACHE, or
 * no file) and on the handle; a key found in either is used without a search (the handle's
 * own earlier searches come first).  mode 0 (the default): the
 * fixed shapes.  The next batched call on the handle builds a new plan.  Different
 * shapes change the order of floating-point sums, not the arithmetic.
 */
int corutv_set_autotune(corutv_handle* h, int mode, const char* cache_path);

typedef struct {
  int32_t tuned;        /* 1: the current plan's shapes come from the autotuner */
  int32_t from_cache;   /* 1: read from the cache file (no search ran) */
  int32_t gram_cols;    /* columns per Gram partial block */
  int32_t split_k;      /* K range of one split of the CUDA-core passes */
  int32_t tc_order;     /* tensor-core pass tables: 0 problems as given, 1 largest reduction first */
  int32_t reserved0;
  double tuned_ms;      /* whole-batch time of the chosen shapes in the search (0 if from the cache) */
  double default_ms;    /* whole-batch time of the fixed shapes in the search (0 if from the cache) */
} corutv_batch_tuning;

/* The shapes of the handle's current batched plan (ERR_INVALID_ARG before any batch). */
int corutv_batch_tuning_read(corutv_handle* h, corutv_batch_tuning* out);

/* ------------------------------------------------------------------------
 * Serving: a request queue in front of corutv_solve_batched (no counterpart in
 * the paper; each request is one solve of Alg. 2 / Alg. 3).
 * ---------------------------------------------------------------------- */

typedef struct corutv_server corutv_server;

/*
 * Start a server on `device`: a worker thread forms batches from pending
 * requests -- one storage dtype per batch, at most max_slots requests, admitted
 * while the sum of their HBM footprints (A as stored, m x lda elements, plus the
 * batch workspace of the request) stays within hbm_budget bytes -- and runs them
 * with corutv_solve_batched on two handles and streams in turn (the next batch
 * is formed and enqueued while the previous one runs).  A request whose
 * footprint alone exceeds the budget finishes with ERR_OOM.  queue_capacity
 * bounds the requests waiting for admission.
 */
int corutv_server_create(corutv_server** out, int device, size_t hbm_budget, int max_slots, int queue_capacity);

/*
 * Queue one solve (device pointers as in corutv_solve_batched; the caller keeps
 * A, Psi and the outputs valid and untouched until the request has finished).
 * Never blocks: returns ERR_BUSY when the queue is full, a validation error for
 * an invalid problem, else OK with *ticket set.
 */
int corutv_server_submit(corutv_server* s, const corutv_problem* p, uint64_t* ticket);

/*
 * CORUTV_PENDING while the request is queued or running; once it has finished,
 * its final status (OK, ERR_OOM, ERR_TIMEOUT, ERR_CUDA ...) with *info filled
 * (info may be NULL) -- the ticket is then released.  Unknown tickets:
 * ERR_INVALID_ARG.
 */
int corutv_server_poll(corutv_server* s, uint64_t ticket, corutv_info* info);

/* Counters: batches launched, requests finished, requests waiting (any may be NULL). */
int corutv_server_stats(corutv_server* s, int64_t* batches, int64_t* solved, int64_t* pending);

/* Library kernels launched by the server's batches so far (direct launches and the kernels of
 * replayed CUDA graphs), counted on the host as they are enqueued. */
int corutv_server_launches(corutv_server* s, int64_t* launches);

/* Stop accepting requests, finish the queued ones, stop the worker, free everything. */
int corutv_server_destroy(corutv_server* s);

/* ------------------------------------------------------------------------
 * Robust PCA by ALM-CoRUTV (Sec. V, Alg. 5): M = L + S with L low-rank and S
 * sparse, one CoR-UTV solve per iteration.
 * ---------------------------------------------------------------------- */

typedef struct {
  int64_t m, n;          /* shape of M */
  int32_t k, l, q;       /* the CoR-UTV of every iteration (Alg. 2 / 3): k <= l < min(m, n), l <= 128 */
  int32_t side;          /* corutv_side of that CoR-UTV (Phi n x l for RIGHT, m x l for LEFT) */
  int32_t mma;           /* corutv_mma of its passes: AUTO or SIMT = FP32 products on the CUDA cores;
                            TF32 = tensor cores (its ~2^-11 product errors can keep extra diagonals of T
                            above the late, small thresholds 1 / mu) */
  int32_t max_iter;      /* iteration limit (>= 1) */
  double lambda;         /* weight of ||S||_1 (Sec. V); the customary choice is 1 / sqrt(max(m, n)) */
  double mu0, rho, mu_bar;   /* penalty schedule: mu_{j+1} = min(rho mu_j, mu_bar), rho >= 1 */
  double tol;            /* stop when ||M - L - S||_F / ||M||_F < tol (Sec. VI-C uses 1e-5) */
  int32_t reserved[4];   /* must be zero */
} corutv_rpca_params;

typedef struct {
  int32_t status;        /* corutv_status of the device work */
  int32_t iters;         /* iterations run */
  int32_t rank;          /* r of the last thresholding (diagonals of T above 1 / mu) */
  int32_t converged;     /* 1 if the stopping rule was met */
  double zeta;           /* ||M - L - S||_F / ||M||_F after the last iteration */
  double mu;             /* penalty after the last update */
} corutv_rpca_info;

/*
 * corutv_rpca -- Alg. 5 (ALM-CoRUTV) with Y_0 = S_0 = 0: per iteration
 *   L = C_{1/mu}(M - S + Y / mu)     C_delta(B) = U(:,1:r) T(1:r,:) V^T, r = #{T_jj > delta},
 *                                    U, T, V the CoR-UTV of B with the caller's Phi (Sec. V)
 *   S = S_{lambda/mu}(M - L + Y / mu)  (shrinkage, sgn(x) max(|x| - delta, 0))
 *   Y = Y + mu (M - L - S),  mu = min(rho mu, mu_bar)
 * until ||M - L - S||_F / ||M||_F < tol or max_iter iterations.  All matrices
 * are FP32, row-major, device, caller-owned: M (m x n, ldm) is read-only;
 * L, S and Y (m x n, each ld >= n and a multiple of 4, 16-byte aligned, as the
 * tensor-core passes read L's memory as the iteration's B) receive the
 * results (Y the final multiplier); Phi as for corutv_solve, reused by every
 * iteration.  The call returns when the iterations are done (it reads the
 * residual back once per iteration); info (host) receives the outcome.  The
 * handle keeps a lazily allocated buffer for the factors of the iterations.
 */
int corutv_rpca(corutv_handle* h, const corutv_rpca_params* p, const float* M, int64_t ldm, const float* Phi,
                int64_t ldphi, float* L, int64_t ldl, float* S, int64_t lds, float* Y, int64_t ldy,
                corutv_rpca_info* info);

/*
 * corutv_residual_norm2 -- the spectral quality readout (e_k,2 of Sec. VI-B): an
 * estimate of ||A - U(:,1:k) T(1:k,:) V^T||_2 by `iters` power iterations on
 * R^T R from the caller's start vector, R applied as an operator (each
 * iteration reads A twice: y = R x, x = R^T y / ||R^T y||); *out = ||R x|| for
 * the final x (0 if an iterate vanishes).  The estimate is a lower bound that
 * converges to ||R||_2 at the rate (sigma_2(R) / sigma_1(R))^(2 iters).
 *   a_dtype  F32 or F64 (others: ERR_UNSUPPORTED); A, U, V and x0 in that type.
 *   A        device, m x n row-major, lda >= n.
 *   U, V     device, m x l and n x l row-major (ldu, ldv >= l): a solve's outputs.
 *   T        device, l x l row-major FP64 (ldt >= l).  1 <= k <= l <= 128.
 *   x0       device, n elements: the start vector (normalised here; any
 *            non-zero vector, e.g. Gaussian, drawn by the caller).
 * FP32 A: the length-n and length-m dot products use compensated (Dot2)
 * arithmetic and the low-rank part is formed in FP64 before the subtraction;
 * norms in FP64.  Synchronous on the handle's stream (the result is a host
 * double); the handle keeps a lazily allocated buffer of the vectors.
 */
int corutv_residual_norm2(corutv_handle* h, int a_dtype, const void* A, int64_t lda, int64_t m, int64_t n,
                          const void* U, int64_t ldu, const double* T, int64_t ldt, const void* V, int64_t ldv,
                          int l, int k, const void* x0, int iters, double* out);

/* Synchronise the handle's stream and return the outcome of the last solve. */
int corutv_info_wait(corutv_handle* h, corutv_info* out);

/* Per-phase device time accumulated since the last corutv_trace_read (tracing
 * records a CUDA event pair around every phase of every solve on the handle's
 * stream; it costs a few microseconds per solve). */
typedef struct {
  int32_t solves;          /* solves traced */
  int32_t pass_launches;   /* streaming passes over A */
  int64_t launches;        /* library kernels launched (all phases) */
  double pass_ms;          /* device time inside the passes (including split-tile reduction) */
  double pass_bytes;       /* algorithmic bytes of those passes: A + skinny operand + result */
  double orth_ms;          /* CholeskyQR orthonormalisation */
  double core_ms;          /* core reduction (D = Q1^T E or C2^T Q2) */
  double qrcp_ms;          /* QRCP of D */
  double assembly_ms;      /* U = Q1 Q~, V = Q2 P~ and staging of Psi */
  double fro2_ms;          /* ||A||_F^2 */
  int32_t corr_launches;   /* FP32 correction passes (corutv_solve_corrected), not counted above */
  int32_t reserved1;
  double corr_ms;          /* device time inside the correction passes */
  double corr_bytes;       /* algorithmic bytes of those passes */
  double quant_ms;         /* corutv_quantize calls on the handle */
  int32_t pass_kernel_launches;  /* passes of single-problem solves (the launches counted in
                                    pass_launches; batched solves record none) timed kernel-only */
  int32_t reserved2;
  double pass_kernel_ms;   /* device time of those passes' main kernels alone: without the
                              sketch-operand split or rounding before them and the split-tile
                              reduction after them */
} corutv_trace;

/* Enable (1) or disable (0) tracing on the handle. */
int corutv_set_tracing(corutv_handle* h, int enable);

/* Synchronise, return and reset the accumulated trace. */
int corutv_trace_read(corutv_handle* h, corutv_trace* out);

/* ------------------------------------------------------------------------
 * Building blocks (the steps of the hot path, exported for testing and for
 * callers that drive their own schedule).  All take the handle for its
 * stream and workspace.
 * ---------------------------------------------------------------------- */

/*
 * One streaming pass over A (Sec. III: C1 = A Psi, C2 = A^T C1; Alg. 3 steps 3-4).
 *   dir = AX : Ct (l x m, ST) = (A X)^T    with Xt (l x n, ST) = X^T
 *   dir = ATY: Ct (l x n, ST) = (A^T Y)^T  with Xt (l x m, ST) = Y^T
 * A: m x n row-major (lda), dtype a_dtype (F64 needs mma SIMT or AUTO; TF32 modes need F32,
 * BF16X2 needs BF16 or FP8).
 * Rows l..(ST rows) of Xt are ignored.
 */
int corutv_pass(corutv_handle* h, int dir, int a_dtype, int mma,
                const void* A, int64_t lda, int64_t m, int64_t n, const float* a_tile_scales,
                const void* Xt, int64_t ldx, int32_t l, void* Ct, int64_t ldc);

/*
 * Orthonormalise a tall-skinny block in place (Sec. III: C = Q R), ST layout:
 * Ct is l x len (ldc), F32 or F64 (dtype F32/F64).  Shifted CholeskyQR3:
 * R from the Cholesky factor of the Gram matrix (FP64 Gram and Cholesky for
 * F64 blocks; FP32-product partials, a compensated FP32 reduction and an FP32
 * Cholesky for F32 blocks), Q = C R^-1, three times, the first with a diagonal
 * shift (the FP32 third pass is skipped when the second already gives
 * max |Q^T Q - I| <= 2e-6).  If R_out != NULL it
 * receives the l x l upper-triangular R = R_3 R_2 R_1 (row-major FP64, ld l)
 * with C = Q R.
 */
int corutv_orthonormalize(corutv_handle* h, int dtype, void* Ct, int64_t ldc,
                          int64_t len, int32_t l, double* R_out);

/* G (l x l, FP64 row-major, ld l) = X Y^T for ST blocks Xt, Yt (l x len):
 * the Gram matrix C^T C of CholeskyQR, or Q1^T E for the core. */
int corutv_gram(corutv_handle* h, int dtype, const void* Xt, int64_t ldx,
                const void* Yt, int64_t ldy, int64_t len, int32_t l, double* G);

/*
 * QRCP of the l x l core D (FP64 row-major, ldd): D P = Q R (Sec. III,
 * Eq. (D = Q~ R~ P~^T); Alg. 2 step 6).  Householder with Businger-Golub
 * pivoting, column norms recomputed exactly each step, lowest index wins a
 * tie, diag(R) >= 0.  Arithmetic in `dtype` (F32 or F64).  Outputs
 * Q (l x l FP64), R (l x l FP64, upper), perm (int32[l], (D P)[:, j] = D[:, perm[j]]),
 * fro2 (FP64[2]: ||R||_F^2 and ||R(1:k,:)||_F^2) -- fro2 may be NULL.
 */
int corutv_qrcp(corutv_handle* h, int dtype, const double* D, int64_t ldd, int32_t l, int32_t k,
                double* Q, double* R, int32_t* perm, double* fro2);

/* ||A||_F^2 of an m x n row-major A (dtype, lda) into *out (device FP64). */
int corutv_fro2(corutv_handle* h, int a_dtype, const void* A, int64_t lda,
                int64_t m, int64_t n, const float* a_tile_scales, double* out);

/* ------------------------------------------------------------------------
 * Allocation-free variant (no counterpart in the paper).
 * ---------------------------------------------------------------------- */

/* Size of the device array that corutv_gram_noalloc uses for its partial sums.
 * A GPU holds it once the library's device code is loaded there (under lazy
 * module loading, the CUDA default, at the library's first kernel launch or
 * symbol lookup on that device) until its context is destroyed or the process
 * exits. */
#define CORUTV_NOALLOC_SCRATCH_BYTES (4u << 20)

/*
 * corutv_gram_noalloc -- the product G = X Y^T of corutv_gram (l x l, FP64,
 * row-major, ld l, from skinny-transposed Xt, Yt of l rows and `len` columns,
 * dtype F32 or F64) for callers that must not allocate device memory after
 * start-up: a latency-bound loop in which cudaMalloc could synchronise the
 * device, or a process whose device memory belongs to another allocator (a
 * framework's caching pool) where an extra cudaMalloc may fail or fragment it.
 *
 *   - It takes a stream (cudaStream_t as void*) instead of a handle and calls
 *     no cudaMalloc, cudaFree or allocating library routine.  Inputs and the
 *     output G are the caller's device memory.
 *   - Partial sums go to a fixed device array of CORUTV_NOALLOC_SCRATCH_BYTES
 *     (32 partial blocks of up to 128 x 128 FP64): l > 128 is rejected with
 *     CORUTV_ERR_SHAPE.  The array is fully rewritten by each call, so nothing
 *     has to be cleared between calls.
 *   - The first call on a device looks up the array's device address with that
 *     device current (cudaGetSymbolAddress) and caches it with the device's
 *     current context (a new context, e.g. after cudaDeviceReset, is looked up
 *     again).  Under lazy module loading that first call may itself load the
 *     library's device code on the device, the 4 MiB array included, which
 *     allocates and synchronises: make it once at start-up, before any stream
 *     capture, so that later calls allocate nothing.
 *   - All calls on a device share the one array: calls whose work overlaps on
 *     the GPU (different streams, or different host threads) race and give wrong
 *     results.  Serialise them.
 */
int corutv_gram_noalloc(void* stream, int dtype, const void* Xt, int64_t ldx, const void* Yt, int64_t ldy,
                        int64_t len, int32_t l, double* G);

#ifdef __cplusplus
}
#endif
#endif /* CORUTV_H */
