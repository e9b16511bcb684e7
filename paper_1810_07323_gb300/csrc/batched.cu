// Batched CoR-UTV solves (corutv_solve_batched): the schedule of one solve
// (Alg. 2 / Alg. 3, stabilised range finding) with every step a grouped launch
// over all problems of the batch.  The host builds, once per problem set, a
// device table of per-problem descriptors (BatchProb) and block -> (problem,
// local block) maps for each kind of grouped launch; repeated calls with the
// same problem set replay a CUDA graph of the whole sequence.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/corutv.h"
#include "common.cuh"
#include "handle.h"
#include "internal.h"

namespace corutv {

struct BatchState {
  std::vector<unsigned char> key;     // bytes of the problem array the tables were built for
  void* ws = nullptr;                 // device: tables + per-problem buffers (owned)
  size_t ws_bytes = 0;
  void* host = nullptr;               // pinned staging of the tables
  size_t host_bytes = 0;
  size_t table_bytes = 0;
  BatchProb* dprobs = nullptr;
  DevStatus* dstatus = nullptr;
  int count = 0;
  std::vector<int> passes;            // passes over A per problem
  std::vector<int> want_fro2;
  // grouped-launch maps (device) and their block counts
  int2 *t1 = nullptr, *t2 = nullptr, *g1 = nullptr, *g2 = nullptr, *red = nullptr, *lm1 = nullptr,
       *lm2 = nullptr, *s2 = nullptr;
  int nt1 = 0, nt2 = 0, ng1 = 0, ng2 = 0, nred = 0, nlm1 = 0, nlm2 = 0, ns2 = 0;
  int lp = 32, lmax = 1, maxq = 0, a_dtype = CORUTV_F32;
  bool any_exact = false, any_sketch = false, any_fro2 = false;
  std::vector<char> multi_pass;       // per power step: some problem runs more than one CholeskyQR pass
  std::vector<double> pass_bytes;     // algorithmic bytes of each grouped pass: [3 * it + which]
  cudaGraphExec_t exec = nullptr;
  int64_t launches_per_run = 0;
};

void batch_state_free(BatchState* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->ws) cudaFree(b->ws);
  if (b->host) cudaFreeHost(b->host);
  delete b;
}

}  // namespace corutv

using namespace corutv;

namespace {

constexpr size_t kBAlign = 256;

size_t align_up(size_t x) { return (x + kBAlign - 1) / kBAlign * kBAlign; }

int validate(const corutv_problem& p) {
  if (p.reserved0) return CORUTV_ERR_INVALID_ARG;
  for (int64_t r : p.reserved)
    if (r) return CORUTV_ERR_INVALID_ARG;
  if (p.a_dtype == CORUTV_F64) return CORUTV_ERR_UNSUPPORTED;
  if (p.a_dtype < CORUTV_F32 || p.a_dtype > CORUTV_FP8_E4M3) return CORUTV_ERR_INVALID_ARG;
  if (p.mma != CORUTV_MMA_AUTO && p.mma != CORUTV_MMA_SIMT) {
    if (p.mma < CORUTV_MMA_AUTO || p.mma > CORUTV_MMA_BF16X2) return CORUTV_ERR_INVALID_ARG;
    return CORUTV_ERR_UNSUPPORTED;
  }
  if (p.side != CORUTV_SIDE_RIGHT && p.side != CORUTV_SIDE_LEFT) return CORUTV_ERR_INVALID_ARG;
  if (p.core != CORUTV_CORE_EXACT && p.core != CORUTV_CORE_SKETCH) return CORUTV_ERR_INVALID_ARG;
  if (p.orth != CORUTV_ORTH_STABILISED && p.orth != CORUTV_ORTH_STRICT) return CORUTV_ERR_INVALID_ARG;
  if (p.m <= 0 || p.n <= 0) return CORUTV_ERR_SHAPE;
  if (p.k < 1 || p.k > p.l) return CORUTV_ERR_INVALID_ARG;      // 1 <= k <= l (Sec. III)
  if (p.q < 0) return CORUTV_ERR_INVALID_ARG;
  if (p.l >= std::min(p.m, p.n) || p.l > kMaxL) return CORUTV_ERR_SHAPE;   // l < min(m, n) (Sec. III)
  if (!p.A || !p.Phi || !p.U || !p.T || !p.V || !p.perm) return CORUTV_ERR_INVALID_ARG;
  if (p.a_dtype == CORUTV_FP8_E4M3 && !p.a_tile_scales) return CORUTV_ERR_INVALID_ARG;
  if (p.lda < p.n || p.ldphi < p.l || p.ldu < p.l || p.ldt < p.l || p.ldv < p.l) return CORUTV_ERR_SHAPE;
  return CORUTV_OK;
}

// Sizes of one problem's buffers (FP32 sketches and factors, FP64 l x l blocks).
struct ProbSizes {
  int64_t len1, len2, ld1, ld2, ld3;
  int gp1, gp2, nf;
  size_t sk1, sk2, sk3, gparts, ll8, ll4, defic, fparts, status;
};

ProbSizes prob_sizes(const corutv_problem& p, int lp) {
  ProbSizes z{};
  const bool right = p.side == CORUTV_SIDE_RIGHT;
  z.len1 = right ? p.m : p.n;
  z.len2 = right ? p.n : p.m;
  z.ld1 = ld_for(z.len1);
  z.ld2 = ld_for(z.len2);
  z.ld3 = std::max(z.ld1, z.ld2);
  z.gp1 = (int)std::max<int64_t>(1, cdiv(z.len1, kBatchGramCols));
  z.gp2 = (int)std::max<int64_t>(1, cdiv(z.len2, kBatchGramCols));
  z.nf = (int)cdiv(z.len1, kBatchPassBN);
  z.sk1 = sizeof(float) * p.l * z.ld1;
  z.sk2 = sizeof(float) * p.l * z.ld2;
  z.sk3 = sizeof(float) * p.l * z.ld3;
  z.gparts = sizeof(float) * (size_t)std::max(z.gp1, z.gp2) * lp * lp;
  z.ll8 = sizeof(double) * p.l * p.l;
  z.ll4 = sizeof(float) * p.l * p.l;
  z.defic = sizeof(int) * p.l;
  z.fparts = sizeof(double) * z.nf;
  z.status = sizeof(DevStatus);
  return z;
}

size_t prob_bytes(const ProbSizes& z) {
  return align_up(z.sk1) + align_up(z.sk2) + align_up(z.sk3) + align_up(z.gparts) + 3 * align_up(z.ll8) +
         2 * align_up(z.ll4) + align_up(z.defic) + align_up(z.fparts) + align_up(z.status);
}

int lp_for(int lmax) { return lmax <= 32 ? 32 : (lmax <= 64 ? 64 : 128); }

// Host tables: the BatchProb array then the block maps, in one contiguous block.
struct Tables {
  std::vector<BatchProb> probs;
  std::vector<int2> t1, t2, g1, g2, red, lm1, lm2, s2;
};

void add_blocks(std::vector<int2>& v, int p, int64_t n) {
  for (int64_t b = 0; b < n; ++b) v.push_back(make_int2(p, (int)b));
}

size_t tables_bytes(const Tables& t, int count) {
  size_t b = align_up(sizeof(BatchProb) * count);
  for (const std::vector<int2>* v : {&t.t1, &t.t2, &t.g1, &t.g2, &t.red, &t.lm1, &t.lm2, &t.s2})
    b += align_up(sizeof(int2) * std::max<size_t>(1, v->size()));
  return b;
}

#define CUB(x)                                                                         \
  do {                                                                                 \
    cudaError_t e_ = (x);                                                              \
    if (e_ != cudaSuccess) {                                                           \
      fprintf(stderr, "corutv: %s (%s:%d)\n", cudaGetErrorString(e_), __FILE__, __LINE__); \
      return CORUTV_ERR_CUDA;                                                          \
    }                                                                                  \
  } while (0)

// Build tables and buffers for a new problem set (the stream is idle).
int build(corutv_handle* h, BatchState* B, int count, const corutv_problem* probs) {
  int lmax = 1, maxq = 0;
  for (int i = 0; i < count; ++i) {
    lmax = std::max(lmax, (int)probs[i].l);
    maxq = std::max(maxq, (int)probs[i].q);
  }
  const int lp = lp_for(lmax);
  Tables T;
  T.probs.resize(count);
  std::vector<ProbSizes> sz(count);
  size_t per = 0;
  for (int i = 0; i < count; ++i) {
    sz[i] = prob_sizes(probs[i], lp);
    per += prob_bytes(sz[i]);
    const corutv_problem& p = probs[i];
    add_blocks(T.t1, i, cdiv(sz[i].len1, kBatchPassBN));
    add_blocks(T.t2, i, cdiv(sz[i].len2, kBatchPassBN));
    add_blocks(T.g1, i, sz[i].gp1);
    add_blocks(T.g2, i, sz[i].gp2);
    add_blocks(T.red, i, cdiv((int64_t)4 * p.l * p.l, 256));
    add_blocks(T.lm1, i, cdiv(sz[i].len1, kBatchLmulBI));
    add_blocks(T.lm2, i, cdiv(sz[i].len2, kBatchLmulBI));
    add_blocks(T.s2, i, cdiv(sz[i].len2, kBatchTile32));
  }
  const size_t tb = tables_bytes(T, count);
  const size_t need = tb + align_up(sizeof(DevStatus) * count) + per;
  if (!B->ws || B->ws_bytes < need) {
    if (B->ws) cudaFree(B->ws);
    B->ws = nullptr;
    B->ws_bytes = 0;
    if (cudaMalloc(&B->ws, need) != cudaSuccess) {
      cudaGetLastError();
      return CORUTV_ERR_OOM;
    }
    B->ws_bytes = need;
  }
  if (!B->host || B->host_bytes < tb) {
    if (B->host) cudaFreeHost(B->host);
    B->host = nullptr;
    B->host_bytes = 0;
    if (cudaMallocHost(&B->host, tb) != cudaSuccess) {
      cudaGetLastError();
      return CORUTV_ERR_OOM;
    }
    B->host_bytes = tb;
  }
  char* d = static_cast<char*>(B->ws);
  char* hbase = static_cast<char*>(B->host);
  // the tables: same offsets on host and device
  size_t off = 0;
  B->dprobs = reinterpret_cast<BatchProb*>(d + off);
  off += align_up(sizeof(BatchProb) * count);
  auto place = [&](std::vector<int2>& v, int2** dptr, int* n) {
    *dptr = reinterpret_cast<int2*>(d + off);
    *n = (int)v.size();
    if (!v.empty()) memcpy(hbase + off, v.data(), sizeof(int2) * v.size());
    off += align_up(sizeof(int2) * std::max<size_t>(1, v.size()));
  };
  place(T.t1, &B->t1, &B->nt1);
  place(T.t2, &B->t2, &B->nt2);
  place(T.g1, &B->g1, &B->ng1);
  place(T.g2, &B->g2, &B->ng2);
  place(T.red, &B->red, &B->nred);
  place(T.lm1, &B->lm1, &B->nlm1);
  place(T.lm2, &B->lm2, &B->nlm2);
  place(T.s2, &B->s2, &B->ns2);
  B->table_bytes = off;
  // statuses, then the per-problem buffers
  B->dstatus = reinterpret_cast<DevStatus*>(d + off);
  off += align_up(sizeof(DevStatus) * count);
  B->passes.assign(count, 0);
  B->want_fro2.assign(count, 0);
  B->multi_pass.assign(maxq + 1, 0);
  B->any_exact = B->any_sketch = B->any_fro2 = false;
  for (int i = 0; i < count; ++i) {
    const corutv_problem& p = probs[i];
    const ProbSizes& z = sz[i];
    BatchProb& P = T.probs[i];
    memset(&P, 0, sizeof(P));
    P.A = p.A;
    P.lda = p.lda;
    P.scales = p.a_tile_scales;
    P.sld = cdiv(p.n, 128);
    P.Phi = static_cast<const float*>(p.Phi);
    P.ldphi = p.ldphi;
    P.U = static_cast<float*>(p.U);
    P.ldu = p.ldu;
    P.T = p.T;
    P.ldt = p.ldt;
    P.V = static_cast<float*>(p.V);
    P.ldv = p.ldv;
    P.perm = p.perm;
    P.m = p.m;
    P.n = p.n;
    P.len1 = z.len1;
    P.len2 = z.len2;
    P.l = p.l;
    P.k = p.k;
    P.q = p.q;
    P.side = p.side;
    P.core = p.core;
    P.orth = p.orth;
    P.want_fro2 = p.want_fro2 ? 1 : 0;
    const bool right = p.side == CORUTV_SIDE_RIGHT;
    P.dir1 = right ? CORUTV_DIR_AX : CORUTV_DIR_ATY;
    P.dir2 = right ? CORUTV_DIR_ATY : CORUTV_DIR_AX;
    P.ld1 = z.ld1;
    P.ld2 = z.ld2;
    P.ld3 = z.ld3;
    P.gp1 = z.gp1;
    P.gp2 = z.gp2;
    P.nfparts = z.nf;
    P.status = B->dstatus + i;
    P.P1 = reinterpret_cast<float*>(d + off);
    off += align_up(z.sk1);
    P.P2 = reinterpret_cast<float*>(d + off);
    off += align_up(z.sk2);
    P.P3 = reinterpret_cast<float*>(d + off);
    off += align_up(z.sk3);
    P.gparts = reinterpret_cast<float*>(d + off);
    off += align_up(z.gparts);
    P.G = reinterpret_cast<double*>(d + off);
    off += align_up(z.ll8);
    P.D = reinterpret_cast<double*>(d + off);
    off += align_up(z.ll8);
    P.Qt = reinterpret_cast<double*>(d + off);
    off += align_up(z.ll8);
    P.R = reinterpret_cast<float*>(d + off);
    off += align_up(z.ll4);
    P.Rinv = reinterpret_cast<float*>(d + off);
    off += align_up(z.ll4);
    P.defic = reinterpret_cast<int*>(d + off);
    off += align_up(z.defic);
    P.fparts = reinterpret_cast<double*>(d + off);
    off += align_up(z.fparts);
    off += align_up(z.status);
    B->passes[i] = 2 * (p.q + 1) + (p.core == CORUTV_CORE_EXACT ? 1 : 0);
    B->want_fro2[i] = P.want_fro2;
    B->any_exact |= p.core == CORUTV_CORE_EXACT;
    B->any_sketch |= p.core == CORUTV_CORE_SKETCH;
    B->any_fro2 |= P.want_fro2 != 0;
    for (int it = 0; it <= p.q; ++it)
      if (it == p.q || p.orth == CORUTV_ORTH_STRICT) B->multi_pass[it] = 1;
  }
  // algorithmic bytes of every grouped pass (A as stored + sketch operand + result of the
  // problems taking part): index 3 * it + which, the core pass at 3 * (maxq + 1) + kB_CORE
  B->pass_bytes.assign(3 * (maxq + 2), 0.0);
  for (int i = 0; i < count; ++i) {
    const corutv_problem& p = probs[i];
    const int eb = p.a_dtype == CORUTV_F32 ? 4 : (p.a_dtype == CORUTV_BF16 ? 2 : 1);
    const double a_bytes = (double)p.m * p.n * eb, sk = 4.0 * p.l * (double)(sz[i].len1 + sz[i].len2);
    for (int it = 0; it <= p.q; ++it) {
      B->pass_bytes[3 * it + kB_C1] += a_bytes + sk;
      B->pass_bytes[3 * it + kB_C2] += a_bytes + sk;
    }
    if (p.core == CORUTV_CORE_EXACT) B->pass_bytes[3 * (maxq + 1) + kB_CORE] += a_bytes + sk;
  }
  memcpy(hbase, T.probs.data(), sizeof(BatchProb) * count);
  CUB(cudaMemcpyAsync(B->ws, B->host, B->table_bytes, cudaMemcpyHostToDevice, h->stream));
  B->count = count;
  B->lp = lp;
  B->lmax = lmax;
  B->maxq = maxq;
  B->key.assign(reinterpret_cast<const unsigned char*>(probs),
                reinterpret_cast<const unsigned char*>(probs) + sizeof(corutv_problem) * count);
  if (B->exec) {
    cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
  }
  return CORUTV_OK;
}

int orth_grouped(corutv_handle* h, const BatchState* B, int which, int it) {
  PhaseTimer tm(h, kPhOrth);
  const bool second = which == kG_ORTH2;
  const int passes = B->multi_pass[it] ? 3 : 1;
  for (int pass = 0; pass < passes; ++pass) {
    CUB(launch_gram_grouped(B->dprobs, second ? B->g2 : B->g1, second ? B->ng2 : B->ng1, B->red, B->nred, B->lp,
                            which, it, pass, h->stream));
    CUB(launch_cholinv_grouped(B->dprobs, B->count, B->lmax, which, it, pass, kSkipTol32, kShiftRel32, kTolRel32,
                               h->stream));
    CUB(launch_lmul_orth_grouped(B->dprobs, second ? B->lm2 : B->lm1, second ? B->nlm2 : B->nlm1, B->lp, which, it,
                                 pass, h->stream));
  }
  return CORUTV_OK;
}

// The whole batch, enqueued on the handle's stream.
int pass_grouped(corutv_handle* h, const BatchState* B, int which, int it) {
  const double bytes = B->pass_bytes[which == kB_CORE ? 3 * (B->maxq + 1) + kB_CORE : 3 * it + which];
  PhaseTimer tm(h, kPhPass, bytes);
  const bool first = which != kB_C2;
  CUB(launch_pass_simt_grouped(B->dprobs, first ? B->t1 : B->t2, first ? B->nt1 : B->nt2, B->lp, B->a_dtype,
                               which, it, h->stream));
  return CORUTV_OK;
}

int enqueue(corutv_handle* h, const BatchState* B) {
  cudaStream_t st = h->stream;
  CUB(cudaMemsetAsync(B->dstatus, 0, sizeof(DevStatus) * B->count, st));
  {
    PhaseTimer tm(h, kPhAsm);
    CUB(launch_stage_grouped(B->dprobs, B->s2, B->ns2, st));                           // S0
  }
  for (int it = 0; it <= B->maxq; ++it) {
    int rc = pass_grouped(h, B, kB_C1, it);                                              // S1
    if (!rc) rc = orth_grouped(h, B, kG_ORTH1, it);                                      // S2
    if (!rc) rc = pass_grouped(h, B, kB_C2, it);                                         // S3
    if (rc) return rc;
    if (B->any_sketch) CUB(launch_copy_sketch_grouped(B->dprobs, B->s2, B->ns2, it, st));
    rc = orth_grouped(h, B, kG_ORTH2, it);                                               // S4
    if (rc) return rc;
  }
  if (B->any_exact) {                                                                    // S5
    const int rc = pass_grouped(h, B, kB_CORE, 0);
    if (rc) return rc;
    PhaseTimer tm(h, kPhCore);
    CUB(launch_gram_grouped(B->dprobs, B->g1, B->ng1, B->red, B->nred, B->lp, kG_CORE_EXACT, 0, 0, st));
  }
  if (B->any_sketch) {
    PhaseTimer tm(h, kPhCore);
    CUB(launch_gram_grouped(B->dprobs, B->g2, B->ng2, B->red, B->nred, B->lp, kG_CORE_SKETCH, 0, 0, st));
  }
  {
    PhaseTimer tm(h, kPhQrcp);
    CUB(launch_qrcp_grouped(B->dprobs, B->count, st));                                  // S6
  }
  {
    PhaseTimer tm(h, kPhAsm);
    CUB(launch_assemble_grouped(B->dprobs, B->lm1, B->nlm1, B->s2, B->ns2, B->lp, st)); // S7
  }
  if (B->any_fro2) CUB(launch_fro2_grouped(B->dprobs, B->count, st));                   // S9
  return CORUTV_OK;
}

bool same_key(const BatchState* B, int count, const corutv_problem* probs) {
  return B->count == count && B->key.size() == sizeof(corutv_problem) * (size_t)count &&
         memcmp(B->key.data(), probs, B->key.size()) == 0;
}

}  // namespace

extern "C" {

int corutv_batch_workspace_size(int count, const corutv_problem* probs, size_t* bytes) {
  if (!bytes || !probs || count < 1) return CORUTV_ERR_INVALID_ARG;
  int lmax = 1;
  for (int i = 0; i < count; ++i) {
    const int rc = validate(probs[i]);
    if (rc) return rc;
    lmax = std::max(lmax, (int)probs[i].l);
  }
  const int lp = lp_for(lmax);
  Tables T;
  size_t per = 0, blocks = 0;
  for (int i = 0; i < count; ++i) {
    const ProbSizes z = prob_sizes(probs[i], lp);
    per += prob_bytes(z);
    blocks += cdiv(z.len1, kBatchPassBN) + cdiv(z.len2, kBatchPassBN) + z.gp1 + z.gp2 +
              cdiv((int64_t)4 * probs[i].l * probs[i].l, 256) + cdiv(z.len1, kBatchLmulBI) +
              cdiv(z.len2, kBatchLmulBI) + cdiv(z.len2, kBatchTile32);
  }
  *bytes = align_up(sizeof(BatchProb) * count) + 8 * kBAlign + sizeof(int2) * blocks +
           align_up(sizeof(DevStatus) * count) + per;
  return CORUTV_OK;
}

int corutv_solve_batched(corutv_handle* h, int count, const corutv_problem* probs, corutv_info* infos) {
  if (!h || !probs || count < 1) return CORUTV_ERR_INVALID_ARG;
  int a_dtype = probs[0].a_dtype;
  for (int i = 0; i < count; ++i) {
    const int rc = validate(probs[i]);
    if (rc) return rc;
    if (probs[i].a_dtype != a_dtype) return CORUTV_ERR_UNSUPPORTED;   // one storage dtype per batch
  }
  if (!h->batch) h->batch = new (std::nothrow) BatchState();
  if (!h->batch) return CORUTV_ERR_OOM;
  BatchState* B = h->batch;
  const int64_t l0 = launch_counter();
  if (!same_key(B, count, probs)) {
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return CORUTV_ERR_CUDA;
    B->key.clear();
    int rc = build(h, B, count, probs);
    if (rc) return rc;
    B->a_dtype = a_dtype;
    rc = enqueue(h, B);                           // first run of a problem set: direct launches
    if (rc) return rc;
    B->launches_per_run = launch_counter() - l0;
  } else if (B->exec && !h->tracing) {
    CUB(cudaGraphLaunch(B->exec, h->stream));
    launch_counter() += B->launches_per_run;
  } else if (h->tracing || h->stream == nullptr || h->stream == cudaStreamLegacy) {
    // traced runs record their own events; the legacy stream cannot be captured
    int rc = enqueue(h, B);
    if (rc) return rc;
  } else {
    // second run of the same set: capture the sequence once, then replay it
    cudaGraph_t g = nullptr;
    CUB(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    const int64_t c0 = launch_counter();
    const int rc = enqueue(h, B);
    const cudaError_t ce = cudaStreamEndCapture(h->stream, &g);
    launch_counter() = c0;
    if (rc || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return rc ? rc : CORUTV_ERR_CUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&B->exec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      B->exec = nullptr;
      cudaGetLastError();
      return CORUTV_ERR_CUDA;
    }
    CUB(cudaGraphLaunch(B->exec, h->stream));
    launch_counter() += B->launches_per_run;
  }
  h->launches += launch_counter() - l0;
  if (h->tracing) h->acc.solves += count;
  if (infos) return corutv_batch_info_wait(h, count, infos);
  return CORUTV_OK;
}

int corutv_batch_info_wait(corutv_handle* h, int count, corutv_info* infos) {
  if (!h || !infos) return CORUTV_ERR_INVALID_ARG;
  BatchState* B = h->batch;
  if (!B || B->count != count || B->key.empty()) return CORUTV_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return CORUTV_ERR_CUDA;
  std::vector<DevStatus> st(count);
  if (cudaMemcpy(st.data(), B->dstatus, sizeof(DevStatus) * count, cudaMemcpyDeviceToHost) != cudaSuccess)
    return CORUTV_ERR_CUDA;
  for (int i = 0; i < count; ++i) {
    corutv_info& o = infos[i];
    memset(&o, 0, sizeof(o));
    o.status = (st[i].flags & kStatTimeout) ? CORUTV_ERR_TIMEOUT : CORUTV_OK;
    o.passes_over_A = B->passes[i];
    o.chol_fallbacks = st[i].chol_fallbacks;
    o.chol_shift_rel = kShiftRel32;
    o.fro2_A = B->want_fro2[i] ? st[i].fro2_A : NAN;
    o.fro2_T = st[i].fro2_T;
    o.fro2_Tk = st[i].fro2_Tk;
  }
  return CORUTV_OK;
}

}  // extern "C"
