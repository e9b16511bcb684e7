// Batched CoR-UTV solves (corutv_solve_batched): the schedule of one solve
// (Alg. 2 / Alg. 3, stabilised range finding) with every step a grouped launch
// over all problems of the batch.  The host builds, once per problem set, a
// device table of per-problem descriptors (BatchProb), block -> (problem,
// local block) maps for each kind of grouped launch and, for FP32 batches the
// tensor cores can read, one table per grouped TF32 pass (GPassProb) with the
// problems' tensor maps; repeated calls with the same problem set replay a
// CUDA graph of the whole sequence.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <stdlib.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/corutv.h"
#include "common.cuh"
#include "handle.h"
#include "internal.h"
#include "tc_common.cuh"

namespace corutv {

// one grouped TF32 pass (its problem table lives in the device tables)
struct PassTable {
  int which = 0, it = 0;
  size_t off_gp = 0, off_rmap = 0;
  int np = 0, nround = 0;
  int64_t iters = 0, tiles = 0;
  int lmax = 1;
  bool fro = false;
  bool keep_a = false;                // the C1 table of a fused group: A stays in L2 for the W launch
  double bytes = 0.0;
  GPassProb* d_gp = nullptr;
  int2* d_rmap = nullptr;
};

// one grouped kind::f16 pass (BF16 / FP8 problems): its problem table, the CTAs' runs of work
// units, and the block maps of the sketch operand's split and of the ordered split-K reduction
struct LpTable {
  int which = 0, it = 0;
  size_t off_gp = 0, off_cta = 0, off_smap = 0, off_rmap = 0;
  int np = 0, G = 0, nsplit = 0, nred = 0, lmax = 1;
  bool fro = false;
  bool keep_a = false;                // the C1 table of a fused group: A stays in L2 for the W launch
  double bytes = 0.0;                 // algorithmic bytes of the pass
  GLpProb* d_gp = nullptr;
  int* d_cta = nullptr;
  int2* d_smap = nullptr;
  int2* d_rmap = nullptr;
};

// Shapes of a batched plan that the autotuner may change (defaults: the fixed plan).
struct BatchTune {
  int gram_cols = kBatchGramCols;     // columns per Gram partial block
  int64_t split_k = kBatchSplitK;     // K range of one split of the CUDA-core passes
  int tc_order = 0;                   // tensor-core pass tables: 0 problems as given, 1 largest K first
};

enum MapKind { kMapT1 = 0, kMapT2, kMapG1, kMapG2, kMapRed, kMapLm1, kMapLm2, kMapS2, kMapQ, kNumMaps };

struct BatchState {
  std::vector<unsigned char> key;     // bytes of the problem array the tables were built for
  BatchTune tune;                     // shapes the tables were built with
  bool tuned = false, tune_from_cache = false;
  double tuned_ms = 0.0, default_ms = 0.0;
  std::vector<std::pair<std::string, BatchTune>> tuned_keys;   // this handle's searches, by key
  void* ws = nullptr;                 // device: tables + per-problem buffers (owned)
  size_t ws_bytes = 0;
  void* host = nullptr;               // pinned staging of the tables
  size_t host_bytes = 0;
  size_t table_bytes = 0;
  BatchProb* dprobs = nullptr;
  DevStatus* dstatus = nullptr;
  DevStatus* bstatus = nullptr;       // batch-wide (timeouts of the grouped tensor-core passes)
  float* partials = nullptr;
  int* kcount = nullptr;              // split counters of the SIMT passes (all problems)
  size_t kcount_bytes = 0;
  int count = 0;
  std::vector<int> passes;            // passes over A per problem
  std::vector<int> want_fro2;
  // grouped-launch maps (device) and their block counts, per sketch-size class (problems
  // with l <= 32, <= 64, <= 128 run the 32-, 64- and 128-row kernel variants); kinds:
  // kMapT1/T2 SIMT pass tiles, kMapG1/G2 Gram partials, kMapRed Gram reduction, kMapLm1/Lm2
  // lmul tiles, kMapS2 32-column tiles of the second sketch (class-independent: class 0), kMapQ
  // one block per problem (QRCP)
  int2* map[3][kNumMaps] = {};
  int nmap[3][kNumMaps] = {};
  int lp = 32, lmax = 1, maxq = 0, a_dtype = CORUTV_F32;
  bool any_exact = false, any_sketch = false, any_fro2 = false;
  bool tc = false;                    // FP32 batch: passes on the tensor cores (grouped TF32)
  std::vector<PassTable> ptabs;       // index 2 * it + which (C1, C2), then the core pass
  bool lpt = false;                   // BF16 / FP8 batch: some problems' passes on the grouped kind::f16 kernel
  std::vector<LpTable> ltabs;
  // table indices (into ptabs or ltabs) per power step: the non-fused problems' C1 and C2, the
  // fused problems' (C1, W) groups; then the exact core (-1: no table)
  std::vector<int> t_c1, t_c2;
  std::vector<std::vector<std::pair<int, int>>> t_groups;
  int t_core = -1;
  bool any_fuse = false;
  std::vector<int> hbm_passes;        // passes per problem that stream A from HBM
  std::vector<char> multi_pass;       // per power step: some problem runs more than one CholeskyQR pass
  std::vector<double> pass_bytes;     // SIMT passes: algorithmic bytes, [3 * it + which]
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

constexpr int kClassLP[3] = {32, 64, 128};
// A of one group of fused problems: small enough to stay in L2 (126 MB) between its C1 and W launches
constexpr double kFuseGroupBytes = 80.0 * (1 << 20);
// autotuner candidates (the first of each list is the largest plan: the workspace query sizes for it)
constexpr int kTuneGramCols[4] = {256, 512, 1024, 2048};
constexpr int64_t kTuneSplitK[3] = {1024, 2048, 4096};
int lclass(int l) { return l <= 32 ? 0 : (l <= 64 ? 1 : 2); }
bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int validate(const corutv_problem& p) {
  if (p.fuse_power != 0 && p.fuse_power != 1) return CORUTV_ERR_INVALID_ARG;
  for (int64_t r : p.reserved)
    if (r) return CORUTV_ERR_INVALID_ARG;
  if (p.a_dtype == CORUTV_F64) return CORUTV_ERR_UNSUPPORTED;
  if (p.a_dtype < CORUTV_F32 || p.a_dtype > CORUTV_FP8_E4M3) return CORUTV_ERR_INVALID_ARG;
  if (p.mma < CORUTV_MMA_AUTO || p.mma > CORUTV_MMA_BF16X2) return CORUTV_ERR_INVALID_ARG;
  if (p.mma != CORUTV_MMA_AUTO && p.mma != CORUTV_MMA_SIMT && !(p.mma == CORUTV_MMA_TF32 && p.a_dtype == CORUTV_F32))
    return CORUTV_ERR_UNSUPPORTED;
  if (p.side != CORUTV_SIDE_RIGHT && p.side != CORUTV_SIDE_LEFT) return CORUTV_ERR_INVALID_ARG;
  if (p.core != CORUTV_CORE_EXACT && p.core != CORUTV_CORE_SKETCH) return CORUTV_ERR_INVALID_ARG;
  if (p.orth == CORUTV_ORTH_LITERAL) return CORUTV_ERR_UNSUPPORTED;
  if (p.orth != CORUTV_ORTH_STABILISED && p.orth != CORUTV_ORTH_STRICT) return CORUTV_ERR_INVALID_ARG;
  if (p.m <= 0 || p.n <= 0) return CORUTV_ERR_SHAPE;
  if (p.k < 1 || p.k > p.l) return CORUTV_ERR_INVALID_ARG;      // 1 <= k <= l (Sec. III)
  if (p.q < 0) return CORUTV_ERR_INVALID_ARG;
  if (p.l >= std::min(p.m, p.n) || p.l > kMaxL) return CORUTV_ERR_SHAPE;   // l < min(m, n) (Sec. III)
  if (!p.A || !p.Phi || !p.U || !p.T || !p.V || !p.perm) return CORUTV_ERR_INVALID_ARG;
  if (p.a_dtype == CORUTV_FP8_E4M3 && !p.a_tile_scales) return CORUTV_ERR_INVALID_ARG;
  if (p.lda < p.n || p.ldphi < p.l || p.ldu < p.l || p.ldt < p.l || p.ldv < p.l) return CORUTV_ERR_SHAPE;
  if (p.mma == CORUTV_MMA_TF32 && !(aligned16(p.A) && (p.lda * 4) % 16 == 0)) return CORUTV_ERR_ALIGN;
  return CORUTV_OK;
}

// TF32 tensor-core passes for the whole batch: FP32 A whose rows TMA can address,
// no problem asking for SIMT.
bool batch_uses_tc(int count, const corutv_problem* probs) {
  for (int i = 0; i < count; ++i) {
    const corutv_problem& p = probs[i];
    if (p.a_dtype != CORUTV_F32 || p.mma == CORUTV_MMA_SIMT) return false;
    if (!(aligned16(p.A) && (p.lda * 4) % 16 == 0)) return false;
  }
  return true;
}

// Grouped kind::f16 passes for one BF16 / FP8 problem: rows TMA can address, no SIMT request.
// Decided per problem, so a problem's pass engine (and its result) does not depend on its batch.
bool f16_ok(const corutv_problem& p) {
  if (p.a_dtype != CORUTV_BF16 && p.a_dtype != CORUTV_FP8_E4M3) return false;
  if (p.mma != CORUTV_MMA_AUTO) return false;
  const int eb = p.a_dtype == CORUTV_BF16 ? 2 : 1;
  return aligned16(p.A) && (p.lda * eb) % 16 == 0;
}

enum PassEngine : char { kEngSimt = 0, kEngTf32 = 1, kEngF16 = 2 };

void engines(int count, const corutv_problem* probs, std::vector<char>& eng) {
  const bool tf32 = batch_uses_tc(count, probs);
  eng.assign(count, kEngSimt);
  for (int i = 0; i < count; ++i)
    eng[i] = tf32 ? kEngTf32 : (f16_ok(probs[i]) ? kEngF16 : kEngSimt);
}

// Sizes of one problem's buffers (FP32 sketches and factors, FP64 l x l blocks).
struct ProbSizes {
  int64_t len1, len2, ld1, ld2, ld3, tiles1, tiles2;
  int gp1, gp2, nf, ks1, ks2, ntiles;
  size_t sk1, sk2, sk3, xr, gparts, ll8, ll4, defic, fparts, status, kparts;
};

ProbSizes prob_sizes(const corutv_problem& p, int lp, char eng, const BatchTune& tune) {
  ProbSizes z{};
  const bool right = p.side == CORUTV_SIDE_RIGHT;
  z.len1 = right ? p.m : p.n;
  z.len2 = right ? p.n : p.m;
  z.ld1 = ld_for(z.len1);
  z.ld2 = ld_for(z.len2);
  z.ld3 = std::max(z.ld1, z.ld2);
  z.gp1 = (int)std::max<int64_t>(1, cdiv(z.len1, tune.gram_cols));
  z.gp2 = (int)std::max<int64_t>(1, cdiv(z.len2, tune.gram_cols));
  z.tiles1 = cdiv(z.len1, kBatchPassBN);
  z.tiles2 = cdiv(z.len2, kBatchPassBN);
  // SIMT passes: C1 and the core reduce over len2, C2 over len1
  z.ks1 = batch_ksplit(z.len2, tune.split_k);
  z.ks2 = batch_ksplit(z.len1, tune.split_k);
  z.ntiles = (int)std::max(z.tiles1, z.tiles2);
  z.nf = (int)(z.tiles1 * z.ks1);
  z.sk1 = sizeof(float) * p.l * z.ld1;
  z.sk2 = sizeof(float) * p.l * z.ld2;
  z.sk3 = sizeof(float) * p.l * z.ld3;
  z.xr = eng != kEngSimt ? z.sk3 : 0;       // TF32 operand, or its two BF16 parts
  z.gparts = sizeof(float) * (size_t)std::max(z.gp1, z.gp2) * lp * lp;
  z.ll8 = sizeof(double) * p.l * p.l;
  z.ll4 = sizeof(float) * p.l * p.l;
  z.defic = sizeof(int) * p.l;
  z.fparts = sizeof(double) * z.nf;
  z.status = sizeof(DevStatus);
  z.kparts = sizeof(float) * (size_t)p.l *
             std::max<int64_t>(z.ks1 > 1 ? z.ks1 * z.len1 : 0, z.ks2 > 1 ? z.ks2 * z.len2 : 0);
  if (eng == kEngF16) {
    // grouped kind::f16 units: C1 / core reduce over len2 into len1 positions, C2 the other way;
    // partials [split][l][ld], one sum(a^2) per unit of the first pass
    const int s1 = lp_unit_nsplit(z.len2), s2 = lp_unit_nsplit(z.len1);
    const size_t kp = sizeof(float) * (size_t)p.l *
                      std::max<int64_t>(s1 > 1 ? s1 * z.ld1 : 0, s2 > 1 ? s2 * z.ld2 : 0);
    z.kparts = std::max(z.kparts, kp);
    z.nf = (int)std::max<int64_t>(z.nf, cdiv(z.len1, kLpUnitBN) * s1);
    z.fparts = sizeof(double) * z.nf;
  }
  return z;
}

size_t prob_bytes(const ProbSizes& z) {
  return align_up(z.sk1) + align_up(z.sk2) + align_up(z.sk3) + align_up(z.xr) + align_up(z.gparts) +
         3 * align_up(z.ll8) + 2 * align_up(z.ll4) + align_up(z.defic) + align_up(z.fparts) + align_up(z.status) +
         align_up(z.kparts);
}

int lp_for(int lmax) { return lmax <= 32 ? 32 : (lmax <= 64 ? 64 : 128); }

void add_blocks(std::vector<int2>& v, int p, int64_t n) {
  for (int64_t b = 0; b < n; ++b) v.push_back(make_int2(p, (int)b));
}

#define CUB(x)                                                                         \
  do {                                                                                 \
    cudaError_t e_ = (x);                                                              \
    if (e_ != cudaSuccess) {                                                           \
      fprintf(stderr, "corutv: %s (%s:%d)\n", cudaGetErrorString(e_), __FILE__, __LINE__); \
      return CORUTV_ERR_CUDA;                                                          \
    }                                                                                  \
  } while (0)

// Host-side plan: every table and its byte offset in the uploaded tables region.
struct Plan {
  int count = 0, lp = 32, lmax = 1, maxq = 0;
  bool tc = false, lpt = false;
  std::vector<char> eng;              // pass engine per problem
  std::vector<char> fuse;             // problem fuses its power steps (tensor-core engines)
  std::vector<int> t_c1, t_c2;
  std::vector<std::vector<std::pair<int, int>>> t_groups;
  int t_core = -1;
  std::vector<ProbSizes> sz;
  std::vector<int2> maps[3][kNumMaps];   // per class and MapKind
  size_t off_maps[3][kNumMaps] = {};
  std::vector<PassTable> ptabs;
  std::vector<std::vector<int>> pt_probs;     // problems of each pass table
  std::vector<std::vector<int2>> pt_rmaps;
  std::vector<std::vector<int64_t>> pt_fro;   // fro slots per problem of the table (0: none)
  std::vector<LpTable> ltabs;                 // grouped kind::f16 tables
  std::vector<std::vector<int>> lt_probs;     // problems of each table
  std::vector<std::vector<int>> lt_cta;       // first unit of each CTA (G + 1 entries)
  std::vector<std::vector<int2>> lt_smap, lt_rmap;
  size_t off_tmaps = 0, off_fro = 0, table_bytes = 0, total_fro = 0;
  size_t off_status = 0, off_bstatus = 0, off_partials = 0, off_probs = 0, need = 0;
  size_t off_kcount = 0, kcount_bytes = 0;    // split counters of the SIMT passes, all problems
};

void make_plan(Plan& L, int count, const corutv_problem* probs, int sms, const BatchTune& tune) {
  L.count = count;
  for (int i = 0; i < count; ++i) {
    L.lmax = std::max(L.lmax, (int)probs[i].l);
    L.maxq = std::max(L.maxq, (int)probs[i].q);
  }
  L.lp = lp_for(L.lmax);
  L.tc = batch_uses_tc(count, probs);
  engines(count, probs, L.eng);
  L.sz.resize(count);
  for (int i = 0; i < count; ++i) {
    const corutv_problem& p = probs[i];
    const ProbSizes& z = L.sz[i] = prob_sizes(p, kClassLP[lclass(p.l)], L.eng[i], tune);
    std::vector<int2>* mc = L.maps[lclass(p.l)];
    L.lpt |= L.eng[i] == kEngF16;
    if (L.eng[i] == kEngSimt) {                 // CUDA-core pass blocks
      add_blocks(mc[kMapT1], i, z.tiles1 * z.ks1);
      add_blocks(mc[kMapT2], i, z.tiles2 * z.ks2);
    }
    L.kcount_bytes += sizeof(int) * z.ntiles;
    add_blocks(mc[kMapG1], i, z.gp1);
    add_blocks(mc[kMapG2], i, z.gp2);
    add_blocks(mc[kMapRed], i, cdiv((int64_t)p.l * p.l, 32));
    add_blocks(mc[kMapLm1], i, cdiv(z.len1, kBatchLmulBI));
    add_blocks(mc[kMapLm2], i, cdiv(z.len2, kBatchLmulBI));
    add_blocks(L.maps[0][kMapS2], i, cdiv(z.len2, kBatchTile32));
    add_blocks(mc[kMapQ], i, 1);
  }
  size_t off = align_up(sizeof(BatchProb) * count);
  for (int c = 0; c < 3; ++c)
    for (int k = 0; k < kNumMaps; ++k) {
      L.off_maps[c][k] = off;
      off += align_up(sizeof(int2) * std::max<size_t>(1, L.maps[c][k].size()));
    }
  // Pass tables (tensor-core engines).  Per power step: one table of the C1 and one of the C2
  // products of the problems that do not fuse their power steps; for the ones that do, L2-sized
  // groups, each a C1 table and a W = op2(A) C1 table launched back to back.  Then the exact core.
  auto make_ptab = [&](int which, int it, std::vector<int> members) -> int {
    PassTable T;
    T.which = which;
    T.it = it;
    std::vector<int2> rmap;
    if (tune.tc_order == 1) {
      // largest reduction first (ties: larger output, then the given order)
      auto kk = [&](int i) { return T.which == kB_C2 ? L.sz[i].len1 : L.sz[i].len2; };
      auto ll = [&](int i) { return T.which == kB_C2 ? L.sz[i].len2 : L.sz[i].len1; };
      std::stable_sort(members.begin(), members.end(), [&](int a, int b) {
        return kk(a) != kk(b) ? kk(a) > kk(b) : ll(a) > ll(b);
      });
    }
    for (size_t u = 0; u < members.size(); ++u) {
      const int i = members[u];
      const corutv_problem& p = probs[i];
      const ProbSizes& z = L.sz[i];
      const int64_t len = T.which == kB_C2 ? z.len2 : z.len1, K = T.which == kB_C2 ? z.len1 : z.len2;
      T.iters += tc_grouped_tiles(len) * tc_grouped_kblocks(K);
      T.tiles += tc_grouped_tiles(len);
      T.lmax = std::max(T.lmax, (int)p.l);
      T.bytes += (double)p.m * p.n * 4 + 4.0 * p.l * (double)(len + K);
      add_blocks(rmap, (int)u, cdiv(K, 128));
    }
    T.np = (int)members.size();
    T.nround = (int)rmap.size();
    std::vector<int64_t> fro(members.size(), 0);
    if (T.which == kB_C1 && T.it == 0 && T.np > 0) {
      const int64_t G = std::min<int64_t>(T.iters, sms);
      int64_t base = 0;
      for (size_t u = 0; u < members.size(); ++u) {
        const int i = members[u];
        const ProbSizes& z = L.sz[i];
        const int64_t iters = tc_grouped_tiles(z.len1) * tc_grouped_kblocks(z.len2);
        if (probs[i].want_fro2) {
          fro[u] = 4 * (tc_grouped_owner(base + iters - 1, T.iters, G) - tc_grouped_owner(base, T.iters, G) + 1);
          T.fro = true;
          L.total_fro += (size_t)fro[u];
        }
        base += iters;
      }
    }
    T.off_gp = off;
    off += align_up(sizeof(GPassProb) * std::max(1, T.np));
    T.off_rmap = off;
    off += align_up(sizeof(int2) * std::max(1, T.nround));
    L.ptabs.push_back(T);
    L.pt_probs.push_back(members);
    L.pt_rmaps.push_back(rmap);
    L.pt_fro.push_back(fro);
    return (int)L.ptabs.size() - 1;
  };
  auto make_ltab = [&](int which, int it, std::vector<int> members) -> int {
    LpTable T;
    T.which = which;
    T.it = it;
    auto kk = [&](int i) { return T.which == kB_C2 ? L.sz[i].len1 : L.sz[i].len2; };
    auto ll = [&](int i) { return T.which == kB_C2 ? L.sz[i].len2 : L.sz[i].len1; };
    if (tune.tc_order == 1)
      std::stable_sort(members.begin(), members.end(), [&](int a, int b) {
        return kk(a) != kk(b) ? kk(a) > kk(b) : ll(a) > ll(b);
      });
    // units in table order, weighted by k-blocks (+1 for the epilogue's tile write)
    std::vector<int> w;
    std::vector<int2> smap, rmap;
    for (size_t u = 0; u < members.size(); ++u) {
      const int i = members[u];
      const corutv_problem& p = probs[i];
      const int64_t len = ll(i), K = kk(i);
      const int64_t tiles = cdiv(len, kLpUnitBN), KB = lp_unit_kblocks(K), kbc = lp_unit_kbc(K);
      const int S = lp_unit_nsplit(K);
      for (int s2 = 0; s2 < S; ++s2)
        for (int64_t t2 = 0; t2 < tiles; ++t2) w.push_back((int)(std::min(KB, (s2 + 1) * kbc) - s2 * kbc) + 1);
      add_blocks(smap, (int)u, cdiv(K, 256));
      if (S > 1) add_blocks(rmap, (int)u, tiles);
      T.lmax = std::max(T.lmax, (int)p.l);
      T.fro |= T.which == kB_C1 && T.it == 0 && p.want_fro2;
      const int eb = p.a_dtype == CORUTV_BF16 ? 2 : 1;
      T.bytes += (double)p.m * p.n * eb + 4.0 * p.l * (double)(len + K);
    }
    const int64_t U = (int64_t)w.size();
    T.np = (int)members.size();
    T.G = (int)std::min<int64_t>(U, sms);
    std::vector<int> first(T.G + 1, (int)U);
    if (T.G > 0) {
      // CTA c runs units [first[c], first[c + 1]): first[c] = first unit whose prefix weight
      // reaches c / G of the total
      double total = 0.0, acc = 0.0;
      for (int x : w) total += x;
      int c = 1;
      first[0] = 0;
      for (int64_t u = 0; u < U; ++u) {
        while (c < T.G && acc >= total * c / T.G) first[c++] = (int)u;
        acc += w[u];
      }
    }
    T.nsplit = (int)smap.size();
    T.nred = (int)rmap.size();
    T.off_gp = off;
    off += align_up(sizeof(GLpProb) * std::max(1, T.np));
    T.off_cta = off;
    off += align_up(sizeof(int) * first.size());
    T.off_smap = off;
    off += align_up(sizeof(int2) * std::max<size_t>(1, smap.size()));
    T.off_rmap = off;
    off += align_up(sizeof(int2) * std::max<size_t>(1, rmap.size()));
    L.ltabs.push_back(T);
    L.lt_probs.push_back(members);
    L.lt_cta.push_back(first);
    L.lt_smap.push_back(smap);
    L.lt_rmap.push_back(rmap);
    return (int)L.ltabs.size() - 1;
  };
  L.fuse.assign(count, 0);
  L.t_c1.assign(L.maxq + 1, -1);
  L.t_c2.assign(L.maxq + 1, -1);
  L.t_groups.assign(L.maxq + 1, {});
  if (L.tc || L.lpt) {
    auto on_tc = [&](int i) { return L.tc || L.eng[i] == kEngF16; };
    for (int i = 0; i < count; ++i) L.fuse[i] = probs[i].fuse_power && on_tc(i) ? 1 : 0;
    auto add = [&](int which, int it, const std::vector<int>& members) {
      return L.tc ? make_ptab(which, it, members) : make_ltab(which, it, members);
    };
    for (int it = 0; it <= L.maxq; ++it) {
      std::vector<int> plain, fused;
      for (int i = 0; i < count; ++i)
        if (on_tc(i) && it <= probs[i].q) (L.fuse[i] ? fused : plain).push_back(i);
      L.t_c1[it] = add(kB_C1, it, plain);
      L.t_c2[it] = add(kB_C2, it, plain);
      // groups of at most kFuseGroupBytes of A (a larger problem alone), in the given order
      std::vector<int> g;
      double gb = 0.0;
      auto flush = [&]() {
        if (g.empty()) return;
        const int c1 = add(kB_C1, it, g);
        if (L.tc) L.ptabs[c1].keep_a = true;
        else L.ltabs[c1].keep_a = true;
        L.t_groups[it].push_back(std::make_pair(c1, add(kB_C2, it, g)));
        g.clear();
        gb = 0.0;
      };
      for (int i : fused) {
        const corutv_problem& p = probs[i];
        const double ab = (double)p.m * p.n * (p.a_dtype == CORUTV_F32 ? 4 : (p.a_dtype == CORUTV_BF16 ? 2 : 1));
        if (!g.empty() && gb + ab > kFuseGroupBytes) flush();
        g.push_back(i);
        gb += ab;
      }
      flush();
    }
    std::vector<int> core;
    for (int i = 0; i < count; ++i)
      if (on_tc(i) && probs[i].core == CORUTV_CORE_EXACT) core.push_back(i);
    L.t_core = add(kB_CORE, 0, core);
    L.off_tmaps = off;                              // 4 (TF32) or 6 (kind::f16) tensor maps per problem
    off += align_up(sizeof(CUtensorMap) * (L.tc ? 4 : 6) * (size_t)count);
  }
  L.table_bytes = off;                              // uploaded part
  L.off_fro = off;
  off += align_up(sizeof(double) * std::max<size_t>(1, L.total_fro));
  L.off_status = off;
  off += align_up(sizeof(DevStatus) * count);
  L.off_bstatus = off;
  off += align_up(sizeof(DevStatus));
  L.off_partials = off;
  if (L.tc) off += align_up(tc_grouped_partial_bytes(sms));
  L.off_kcount = off;
  off += align_up(std::max<size_t>(sizeof(int), L.kcount_bytes));
  L.off_probs = off;
  for (int i = 0; i < count; ++i) off += prob_bytes(L.sz[i]);
  L.need = off;
}

// Build tables and buffers for a new problem set (the stream is idle).
int build(corutv_handle* h, BatchState* B, int count, const corutv_problem* probs, const BatchTune& tune) {
  Plan L;
  make_plan(L, count, probs, h->sms, tune);
  if (!B->ws || B->ws_bytes < L.need) {
    if (B->ws) cudaFree(B->ws);
    B->ws = nullptr;
    B->ws_bytes = 0;
    if (cudaMalloc(&B->ws, L.need) != cudaSuccess) {
      cudaGetLastError();
      return CORUTV_ERR_OOM;
    }
    B->ws_bytes = L.need;
  }
  if (!B->host || B->host_bytes < L.table_bytes) {
    if (B->host) cudaFreeHost(B->host);
    B->host = nullptr;
    B->host_bytes = 0;
    if (cudaMallocHost(&B->host, L.table_bytes) != cudaSuccess) {
      cudaGetLastError();
      return CORUTV_ERR_OOM;
    }
    B->host_bytes = L.table_bytes;
  }
  char* d = static_cast<char*>(B->ws);
  char* hb = static_cast<char*>(B->host);
  memset(hb, 0, L.table_bytes);
  B->dprobs = reinterpret_cast<BatchProb*>(d);
  for (int c = 0; c < 3; ++c)
    for (int k = 0; k < kNumMaps; ++k) {
      B->map[c][k] = reinterpret_cast<int2*>(d + L.off_maps[c][k]);
      B->nmap[c][k] = (int)L.maps[c][k].size();
      if (!L.maps[c][k].empty())
        memcpy(hb + L.off_maps[c][k], L.maps[c][k].data(), sizeof(int2) * L.maps[c][k].size());
    }
  B->dstatus = reinterpret_cast<DevStatus*>(d + L.off_status);
  B->bstatus = reinterpret_cast<DevStatus*>(d + L.off_bstatus);
  B->partials = L.tc ? reinterpret_cast<float*>(d + L.off_partials) : nullptr;
  B->kcount = reinterpret_cast<int*>(d + L.off_kcount);
  B->kcount_bytes = std::max<size_t>(sizeof(int), L.kcount_bytes);
  size_t kc_off = 0;
  B->passes.assign(count, 0);
  B->hbm_passes.assign(count, 0);
  B->any_fuse = false;
  B->want_fro2.assign(count, 0);
  B->multi_pass.assign(L.maxq + 1, 0);
  B->any_exact = B->any_sketch = B->any_fro2 = false;
  std::vector<BatchProb> P(count);
  size_t off = L.off_probs;
  for (int i = 0; i < count; ++i) {
    const corutv_problem& p = probs[i];
    const ProbSizes& z = L.sz[i];
    BatchProb& Q = P[i];
    memset(&Q, 0, sizeof(Q));
    Q.A = p.A;
    Q.lda = p.lda;
    Q.scales = p.a_tile_scales;
    Q.sld = cdiv(p.n, 128);
    Q.Phi = static_cast<const float*>(p.Phi);
    Q.ldphi = p.ldphi;
    Q.U = static_cast<float*>(p.U);
    Q.ldu = p.ldu;
    Q.T = p.T;
    Q.ldt = p.ldt;
    Q.V = static_cast<float*>(p.V);
    Q.ldv = p.ldv;
    Q.perm = p.perm;
    Q.m = p.m;
    Q.n = p.n;
    Q.len1 = z.len1;
    Q.len2 = z.len2;
    Q.l = p.l;
    Q.k = p.k;
    Q.q = p.q;
    Q.side = p.side;
    Q.core = p.core;
    Q.orth = p.orth;
    Q.want_fro2 = p.want_fro2 ? 1 : 0;
    Q.fuse = L.fuse[i];
    const bool right = p.side == CORUTV_SIDE_RIGHT;
    Q.dir1 = right ? CORUTV_DIR_AX : CORUTV_DIR_ATY;
    Q.dir2 = right ? CORUTV_DIR_ATY : CORUTV_DIR_AX;
    Q.ld1 = z.ld1;
    Q.ld2 = z.ld2;
    Q.ld3 = z.ld3;
    Q.gp1 = z.gp1;
    Q.gp2 = z.gp2;
    Q.nfparts = z.nf;
    Q.status = B->dstatus + i;
    Q.ks1 = z.ks1;
    Q.ks2 = z.ks2;
    Q.kcount = B->kcount + kc_off;
    kc_off += z.ntiles;
    auto take = [&](size_t bytes) {
      char* r = d + off;
      off += align_up(bytes);
      return r;
    };
    Q.P1 = reinterpret_cast<float*>(take(z.sk1));
    Q.P2 = reinterpret_cast<float*>(take(z.sk2));
    Q.P3 = reinterpret_cast<float*>(take(z.sk3));
    float* Xr = reinterpret_cast<float*>(take(z.xr));
    Q.gparts = reinterpret_cast<float*>(take(z.gparts));
    Q.G = reinterpret_cast<float*>(take(z.ll8));
    Q.D = reinterpret_cast<float*>(take(z.ll8));
    Q.Qt = reinterpret_cast<float*>(take(z.ll8));
    Q.R = reinterpret_cast<float*>(take(z.ll4));
    Q.Rinv = reinterpret_cast<float*>(take(z.ll4));
    Q.defic = reinterpret_cast<int*>(take(z.defic));
    Q.fparts = reinterpret_cast<double*>(take(z.fparts));
    take(z.status);
    Q.kparts = z.kparts ? reinterpret_cast<float*>(take(z.kparts)) : nullptr;
    if (L.tc) {
      // tensor maps: A rows (dir AX), A columns (dir ATY), Xr over len1 and over len2 columns
      CUtensorMap* tm = reinterpret_cast<CUtensorMap*>(hb + L.off_tmaps) + 4 * i;
      bool ok = make_map_2d(&tm[0], p.A, p.m, p.n, p.lda, 4, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 32, 256, true) &&
                make_map_2d(&tm[1], p.A, p.m, p.n, p.lda, 4, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 32, 32, true) &&
                make_map_2d(&tm[2], Xr, p.l, z.len1, z.ld3, 4, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 32, 128, true) &&
                make_map_2d(&tm[3], Xr, p.l, z.len2, z.ld3, 4, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 32, 128, true);
      if (!ok) return CORUTV_ERR_CUDA;
    }
    if (L.eng[i] == kEngF16) {
      // tensor maps: A tiles for A X and for A^T Y, the BF16 parts (Xh, Xl) of the sketch operand
      // over len1 and over len2 columns; Xh and Xl share the Xr buffer (l rows of ld3 each)
      CUtensorMap* tm = reinterpret_cast<CUtensorMap*>(hb + L.off_tmaps) + 6 * i;
      char* Xh = reinterpret_cast<char*>(Xr);
      char* Xl = Xh + 2 * (size_t)p.l * z.ld3;
      const auto bf = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
      bool ok;
      if (p.a_dtype == CORUTV_FP8_E4M3)       // raw bytes, no swizzle: 64 x 256 and 256 x 64 boxes
        ok = make_map_2d(&tm[0], p.A, p.m, p.n, p.lda, 1, CU_TENSOR_MAP_DATA_TYPE_UINT8, 64, 256, false) &&
             make_map_2d(&tm[1], p.A, p.m, p.n, p.lda, 1, CU_TENSOR_MAP_DATA_TYPE_UINT8, 256, 64, false);
      else
        ok = make_map_2d(&tm[0], p.A, p.m, p.n, p.lda, 2, bf, 64, 256, true) &&
             make_map_2d(&tm[1], p.A, p.m, p.n, p.lda, 2, bf, 64, 64, true);
      ok = ok && make_map_2d(&tm[2], Xh, p.l, z.len1, z.ld3, 2, bf, 64, 128, true) &&
           make_map_2d(&tm[3], Xl, p.l, z.len1, z.ld3, 2, bf, 64, 128, true) &&
           make_map_2d(&tm[4], Xh, p.l, z.len2, z.ld3, 2, bf, 64, 128, true) &&
           make_map_2d(&tm[5], Xl, p.l, z.len2, z.ld3, 2, bf, 64, 128, true);
      if (!ok) return CORUTV_ERR_CUDA;
    }
    B->passes[i] = 2 * (p.q + 1) + (p.core == CORUTV_CORE_EXACT ? 1 : 0);
    // fused power steps: the W launch of each step re-reads A from L2
    B->hbm_passes[i] = B->passes[i] - (L.fuse[i] ? p.q + 1 : 0);
    B->any_fuse |= L.fuse[i] != 0;
    B->want_fro2[i] = Q.want_fro2;
    B->any_exact |= p.core == CORUTV_CORE_EXACT;
    B->any_sketch |= p.core == CORUTV_CORE_SKETCH;
    B->any_fro2 |= Q.want_fro2 != 0;
    for (int it = 0; it <= p.q; ++it)
      if (it == p.q || p.orth == CORUTV_ORTH_STRICT) B->multi_pass[it] = 1;
    (void)Xr;   // the pass tables find it right after P3 (carve order above)
  }
  // pass tables (TF32 tensor cores)
  B->tc = L.tc;
  B->ptabs = L.ptabs;
  B->t_c1 = L.t_c1;
  B->t_c2 = L.t_c2;
  B->t_groups = L.t_groups;
  B->t_core = L.t_core;
  if (L.tc) {
    const CUtensorMap* dmaps = reinterpret_cast<const CUtensorMap*>(d + L.off_tmaps);
    double* fro_base = reinterpret_cast<double*>(d + L.off_fro);
    size_t fro_used = 0;
    for (size_t t = 0; t < L.ptabs.size(); ++t) {
      PassTable& T = B->ptabs[t];
      T.d_gp = reinterpret_cast<GPassProb*>(d + T.off_gp);
      T.d_rmap = reinterpret_cast<int2*>(d + T.off_rmap);
      if (!L.pt_rmaps[t].empty())
        memcpy(hb + T.off_rmap, L.pt_rmaps[t].data(), sizeof(int2) * L.pt_rmaps[t].size());
      GPassProb* gpv = reinterpret_cast<GPassProb*>(hb + T.off_gp);
      const int64_t G = std::min<int64_t>(T.iters, h->sms);
      int64_t ibase = 0, tbase = 0;
      for (int u = 0; u < T.np; ++u) {
        const int i = L.pt_probs[t][u];
        const BatchProb& Q = P[i];
        const ProbSizes& z = L.sz[i];
        GPassProb& g = gpv[u];
        const bool second = T.which == kB_C2;
        const int dir = second ? Q.dir2 : Q.dir1;
        g.mapA = dmaps + 4 * i + (dir == CORUTV_DIR_AX ? 0 : 1);
        g.mapX = dmaps + 4 * i + (second ? 2 : 3);
        g.Ct = T.which == kB_C1 ? Q.P1 : (second ? Q.P2 : Q.P3);
        g.ldc = T.which == kB_C1 ? Q.ld1 : (second ? Q.ld2 : Q.ld3);
        g.X = second ? Q.P1 : Q.P2;
        g.ldx = second ? Q.ld1 : Q.ld2;
        // Xr sits right after P3 (see the carve order above)
        g.Xr = reinterpret_cast<float*>(reinterpret_cast<char*>(Q.P3) + align_up(z.sk3));
        g.ldr = z.ld3;
        g.len = second ? z.len2 : z.len1;
        g.K = second ? z.len1 : z.len2;
        g.KB = tc_grouped_kblocks(g.K);
        g.tiles = tc_grouped_tiles(g.len);
        g.iter_base = ibase;
        g.tile_base = tbase;
        g.owner_first = tc_grouped_owner(ibase, T.iters, G);
        g.l = Q.l;
        g.dir = dir;
        g.fro = nullptr;
        if (L.pt_fro[t][u] > 0) {
          g.fro = fro_base + fro_used;
          P[i].fparts = g.fro;
          P[i].nfparts = (int)L.pt_fro[t][u];
          fro_used += (size_t)L.pt_fro[t][u];
        }
        ibase += g.tiles * g.KB;
        tbase += g.tiles;
      }
    }
  }
  // grouped kind::f16 tables
  B->lpt = L.lpt;
  B->ltabs = L.ltabs;
  if (L.lpt) {
    const CUtensorMap* dmaps = reinterpret_cast<const CUtensorMap*>(d + L.off_tmaps);
    for (size_t t = 0; t < L.ltabs.size(); ++t) {
      LpTable& T = B->ltabs[t];
      T.d_gp = reinterpret_cast<GLpProb*>(d + T.off_gp);
      T.d_cta = reinterpret_cast<int*>(d + T.off_cta);
      T.d_smap = reinterpret_cast<int2*>(d + T.off_smap);
      T.d_rmap = reinterpret_cast<int2*>(d + T.off_rmap);
      memcpy(hb + T.off_cta, L.lt_cta[t].data(), sizeof(int) * L.lt_cta[t].size());
      if (!L.lt_smap[t].empty()) memcpy(hb + T.off_smap, L.lt_smap[t].data(), sizeof(int2) * L.lt_smap[t].size());
      if (!L.lt_rmap[t].empty()) memcpy(hb + T.off_rmap, L.lt_rmap[t].data(), sizeof(int2) * L.lt_rmap[t].size());
      GLpProb* gpv = reinterpret_cast<GLpProb*>(hb + T.off_gp);
      int64_t ubase = 0;
      for (int u = 0; u < T.np; ++u) {
        const int i = L.lt_probs[t][u];
        const corutv_problem& p = probs[i];
        const BatchProb& Q = P[i];
        const ProbSizes& z = L.sz[i];
        GLpProb& g = gpv[u];
        const bool second = T.which == kB_C2;
        const int dir = second ? Q.dir2 : Q.dir1;
        g.mapA = dmaps + 6 * i + (dir == CORUTV_DIR_AX ? 0 : 1);
        g.mapXh = dmaps + 6 * i + (second ? 2 : 4);
        g.mapXl = dmaps + 6 * i + (second ? 3 : 5);
        g.Ct = T.which == kB_C1 ? Q.P1 : (second ? Q.P2 : Q.P3);
        g.ldc = T.which == kB_C1 ? Q.ld1 : (second ? Q.ld2 : Q.ld3);
        g.kparts = Q.kparts;
        g.ldk = second ? z.ld2 : z.ld1;
        g.X = second ? Q.P1 : Q.P2;
        g.ldx = second ? Q.ld1 : Q.ld2;
        // Xh / Xl sit right after P3 (see the carve order above)
        g.Xh = reinterpret_cast<char*>(Q.P3) + align_up(z.sk3);
        g.Xl = static_cast<char*>(g.Xh) + 2 * (size_t)p.l * z.ld3;
        g.ldxs = z.ld3;
        g.scales = p.a_tile_scales;
        g.sld = cdiv(p.n, 128);
        g.srows = cdiv(p.m, 128);
        g.scols = cdiv(p.n, 128);
        g.len = second ? z.len2 : z.len1;
        g.K = second ? z.len1 : z.len2;
        g.KB = lp_unit_kblocks(g.K);
        g.kbc = lp_unit_kbc(g.K);
        g.S = lp_unit_nsplit(g.K);
        g.tiles = cdiv(g.len, kLpUnitBN);
        g.units = g.tiles * g.S;
        g.unit_base = ubase;
        g.l = p.l;
        g.dir = dir;
        g.fro = nullptr;
        if (T.which == kB_C1 && T.it == 0 && p.want_fro2) {
          g.fro = Q.fparts;
          P[i].nfparts = (int)g.units;
        }
        ubase += g.units;
      }
    }
  }
  // SIMT passes: algorithmic bytes of every grouped pass, index 3 * it + which
  B->pass_bytes.assign(3 * (L.maxq + 2), 0.0);
  for (int i = 0; i < count; ++i) {
    const corutv_problem& p = probs[i];
    const int eb = p.a_dtype == CORUTV_F32 ? 4 : (p.a_dtype == CORUTV_BF16 ? 2 : 1);
    const double a_bytes = (double)p.m * p.n * eb, sk = 4.0 * p.l * (double)(L.sz[i].len1 + L.sz[i].len2);
    for (int it = 0; it <= p.q && !L.fuse[i]; ++it) {      // fused problems: their group tables count
      B->pass_bytes[3 * it + kB_C1] += a_bytes + sk;
      B->pass_bytes[3 * it + kB_C2] += a_bytes + sk;
    }
    if (p.core == CORUTV_CORE_EXACT) B->pass_bytes[3 * (L.maxq + 1) + kB_CORE] += a_bytes + sk;
  }
  memcpy(hb, P.data(), sizeof(BatchProb) * count);
  B->table_bytes = L.table_bytes;
  CUB(cudaMemcpyAsync(B->ws, B->host, L.table_bytes, cudaMemcpyHostToDevice, h->stream));
  B->count = count;
  B->lp = L.lp;
  B->lmax = L.lmax;
  B->maxq = L.maxq;
  B->key.assign(reinterpret_cast<const unsigned char*>(probs),
                reinterpret_cast<const unsigned char*>(probs) + sizeof(corutv_problem) * count);
  B->tune = tune;
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
    for (int c = 0; c < 3; ++c)
      CUB(launch_gram_grouped(B->dprobs, B->map[c][second ? kMapG2 : kMapG1], B->nmap[c][second ? kMapG2 : kMapG1],
                              B->map[c][kMapRed], B->nmap[c][kMapRed], kClassLP[c], which, it, pass, h->stream));
    CUB(launch_cholinv_grouped(B->dprobs, B->count, B->lmax, which, it, pass, kSkipTol32, kShiftRel32, kTolRel32,
                               h->stream));
    for (int c = 0; c < 3; ++c)
      CUB(launch_lmul_orth_grouped(B->dprobs, B->map[c][second ? kMapLm2 : kMapLm1],
                                   B->nmap[c][second ? kMapLm2 : kMapLm1], kClassLP[c], which, it, pass, h->stream));
    // fused power steps: the same R^-1 applied to W = op2(A) C1 (in P2), so after the last pass
    // P2 = W R1^-1 = op2(A) Q1, the sketch C2 of the step
    if (!second && B->any_fuse)
      for (int c = 0; c < 3; ++c)
        CUB(launch_lmul_orth_grouped(B->dprobs, B->map[c][kMapLm2], B->nmap[c][kMapLm2], kClassLP[c], kG_ORTH1_W,
                                     it, pass, h->stream));
  }
  return CORUTV_OK;
}

int gram_core_grouped(corutv_handle* h, const BatchState* B, int which) {
  const int k = which == kG_CORE_EXACT ? kMapG1 : kMapG2;
  for (int c = 0; c < 3; ++c)
    CUB(launch_gram_grouped(B->dprobs, B->map[c][k], B->nmap[c][k], B->map[c][kMapRed], B->nmap[c][kMapRed],
                            kClassLP[c], which, 0, 0, h->stream));
  return CORUTV_OK;
}

// one tensor-core pass table (index into ptabs / ltabs; -1: none); km (tracing, may be null):
// events around the pass kernel alone
int launch_table(corutv_handle* h, const BatchState* B, int t, KernelMark* km = nullptr) {
  if (t < 0) return CORUTV_OK;
  if (B->tc) {
    const PassTable& T = B->ptabs[t];
    if (T.np == 0) return CORUTV_OK;
    CUB(launch_pass_tc_grouped(T.d_gp, T.np, T.iters, T.tiles, T.lmax, T.d_rmap, T.nround, B->partials, T.fro,
                               h->sms, B->bstatus, T.keep_a, h->stream, km));
    return CORUTV_OK;
  }
  const LpTable& T = B->ltabs[t];
  if (T.np == 0) return CORUTV_OK;
  CUB(launch_pass_lp_grouped(T.d_gp, T.np, B->a_dtype == CORUTV_FP8_E4M3, T.fro, T.d_cta, T.G, T.d_smap,
                             T.nsplit, T.d_rmap, T.nred, T.lmax, B->bstatus, T.keep_a, h->stream, km));
  return CORUTV_OK;
}

// Tracing of a pass phase that is one table launch: a second event pair around its pass
// kernel alone, recorded as a pass-kernel phase once both events were recorded.
struct TableMark {
  corutv_handle* h;
  double bytes;
  KernelMark km;
  TableMark(corutv_handle* h_, double by) : h(h_), bytes(by) {
    if (h->tracing) {
      km.a = ev_get(h);
      km.b = ev_get(h);
    }
  }
  KernelMark* get() { return km.a ? &km : nullptr; }
  ~TableMark() {
    if (!km.a) return;
    if (km.state == 2) {
      h->recs.push_back(TraceRec{kPhPassKernel, km.a, km.b, bytes});
    } else {
      h->ev_pool.push_back(km.a);
      h->ev_pool.push_back(km.b);
    }
  }
};

// the same as one traced pass phase
int run_table(corutv_handle* h, const BatchState* B, int t) {
  if (t < 0) return CORUTV_OK;
  const bool empty = B->tc ? B->ptabs[t].np == 0 : B->ltabs[t].np == 0;
  if (empty) return CORUTV_OK;
  const double bytes = B->tc ? B->ptabs[t].bytes : B->ltabs[t].bytes;
  PhaseTimer tm(h, kPhPass, bytes);
  TableMark mk(h, bytes);
  return launch_table(h, B, t, mk.get());
}

// the pass `which` of power step `it` for the problems that do not fuse their power steps
int pass_grouped(corutv_handle* h, const BatchState* B, int which, int it) {
  const int t = which == kB_CORE ? B->t_core : (which == kB_C1 ? B->t_c1[it] : B->t_c2[it]);
  if (B->tc) return run_table(h, B, t);
  const double bytes = B->pass_bytes[which == kB_CORE ? 3 * (B->maxq + 1) + kB_CORE : 3 * it + which];
  PhaseTimer tm(h, kPhPass, bytes);
  const int k = which != kB_C2 ? kMapT1 : kMapT2;
  // the kernel-only record when the table's kernel is the phase's only pass kernel
  bool simt_none = true;
  for (int c = 0; c < 3; ++c) simt_none = simt_none && B->nmap[c][k] == 0;
  TableMark mk(h, bytes);
  if (B->lpt) {
    const int rc = launch_table(h, B, t, simt_none ? mk.get() : nullptr);
    if (rc) return rc;
  }
  for (int c = 0; c < 3; ++c)
    CUB(launch_pass_simt_grouped(B->dprobs, B->map[c][k], B->nmap[c][k], kClassLP[c], B->a_dtype, which, it,
                                 h->stream));
  return CORUTV_OK;
}

// The whole batch, enqueued on the handle's stream; steps S0 .. S9 as in a single solve (corutv_abi.cu).
int enqueue(corutv_handle* h, const BatchState* B) {
  cudaStream_t st = h->stream;
  CUB(cudaMemsetAsync(B->dstatus, 0, sizeof(DevStatus) * B->count, st));
  CUB(cudaMemsetAsync(B->kcount, 0, B->kcount_bytes, st));
  CUB(cudaMemsetAsync(B->bstatus, 0, sizeof(DevStatus), st));
  {
    PhaseTimer tm(h, kPhAsm);
    CUB(launch_stage_grouped(B->dprobs, B->map[0][kMapS2], B->nmap[0][kMapS2], st));    // S0
  }
  for (int it = 0; it <= B->maxq; ++it) {
    int rc = CORUTV_OK;
    // fused power steps: per L2-sized group, C1 = op1(A) X and then W = op2(A) C1 while A is in L2
    for (const auto& g : B->t_groups[it]) {
      if (!rc) rc = run_table(h, B, g.first);
      if (!rc) rc = run_table(h, B, g.second);
    }
    if (!rc) rc = pass_grouped(h, B, kB_C1, it);                                         // S1
    if (!rc) rc = orth_grouped(h, B, kG_ORTH1, it);                                      // S2
    if (!rc) rc = pass_grouped(h, B, kB_C2, it);                                         // S3
    if (rc) return rc;
    if (B->any_sketch) CUB(launch_copy_sketch_grouped(B->dprobs, B->map[0][kMapS2], B->nmap[0][kMapS2], it, st));
    rc = orth_grouped(h, B, kG_ORTH2, it);                                               // S4
    if (rc) return rc;
  }
  if (B->any_exact) {                                                                    // S5
    const int rc = pass_grouped(h, B, kB_CORE, 0);
    if (rc) return rc;
    PhaseTimer tm(h, kPhCore);
    const int rc2 = gram_core_grouped(h, B, kG_CORE_EXACT);
    if (rc2) return rc2;
  }
  if (B->any_sketch) {
    PhaseTimer tm(h, kPhCore);
    const int rc = gram_core_grouped(h, B, kG_CORE_SKETCH);
    if (rc) return rc;
  }
  {
    PhaseTimer tm(h, kPhQrcp);
    for (int c = 0; c < 3; ++c)                                                         // S6
      CUB(launch_qrcp_grouped(B->dprobs, B->map[c][kMapQ], B->nmap[c][kMapQ], kClassLP[c], st));
  }
  {
    PhaseTimer tm(h, kPhAsm);
    for (int c = 0; c < 3; ++c)                                                         // S7
      CUB(launch_assemble_grouped(B->dprobs, B->map[c][kMapLm1], B->nmap[c][kMapLm1], B->map[0][kMapS2],
                                  c == 0 ? B->nmap[0][kMapS2] : 0, kClassLP[c], st));
  }
  if (B->any_fro2) CUB(launch_fro2_grouped(B->dprobs, B->count, st));                   // S9
  return CORUTV_OK;
}

// ------------------------------------------------------------------ autotuner
// Cache key: storage dtype, pass engine, sketch-size class of the largest l, and power-of-two
// buckets of the mean m, the mean n and the count, plus the largest q.
int bucket_log2(double x) { return x <= 1.0 ? 0 : (int)floor(log2(x) + 0.5); }

std::string tune_key(int count, const corutv_problem* probs, bool tc) {
  double sm = 0.0, sn = 0.0;
  int lmax = 1, qmax = 0, fused = 0;
  for (int i = 0; i < count; ++i) {
    sm += (double)probs[i].m;
    sn += (double)probs[i].n;
    lmax = std::max(lmax, (int)probs[i].l);
    qmax = std::max(qmax, (int)probs[i].q);
    fused |= probs[i].fuse_power;
  }
  char buf[160];
  snprintf(buf, sizeof(buf), "dtype%d/%s/lclass%d/m%d/n%d/count%d/q%d%s", (int)probs[0].a_dtype,
           tc ? "tc" : "simt", lclass(lmax), bucket_log2(sm / count), bucket_log2(sn / count),
           bucket_log2((double)count), qmax, fused ? "/fused" : "");
  return std::string(buf);
}

// The cache is a JSON object with one entry object per line:
//   {"corutv_autotune": 1, "entries": [
//   {"key": "...", "gram_cols": 512, "split_k": 2048, "tc_order": 0, "tuned_ms": 17.2, "default_ms": 17.6},
//   ...
//   ]}
bool json_int(const std::string& line, const char* name, int64_t* out) {
  const std::string pat = std::string("\"") + name + "\":";
  const size_t at = line.find(pat);
  if (at == std::string::npos) return false;
  *out = strtoll(line.c_str() + at + pat.size(), nullptr, 10);
  return true;
}

std::string line_key(const std::string& line) {
  const std::string pat = "\"key\": \"";
  const size_t at = line.find(pat);
  if (at == std::string::npos) return std::string();
  const size_t end = line.find('"', at + pat.size());
  return end == std::string::npos ? std::string() : line.substr(at + pat.size(), end - at - pat.size());
}

std::vector<std::string> cache_entries(const std::string& path) {
  std::vector<std::string> v;
  FILE* f = fopen(path.c_str(), "r");
  if (!f) return v;
  char buf[1024];
  while (fgets(buf, sizeof(buf), f)) {
    std::string line(buf);
    if (!line_key(line).empty()) {
      while (!line.empty() && (line.back() == '\n' || line.back() == ',' || line.back() == '\r')) line.pop_back();
      v.push_back(line);
    }
  }
  fclose(f);
  return v;
}

bool cache_lookup(const std::string& path, const std::string& key, BatchTune* t) {
  for (const std::string& line : cache_entries(path)) {
    if (line_key(line) != key) continue;
    int64_t gc = 0, sk = 0, order = 0;
    if (!json_int(line, "gram_cols", &gc) || !json_int(line, "split_k", &sk) || !json_int(line, "tc_order", &order))
      return false;
    bool ok_gc = false, ok_sk = false;
    for (int c : kTuneGramCols) ok_gc |= c == gc;
    for (int64_t c : kTuneSplitK) ok_sk |= c == sk;
    if (!ok_gc || !ok_sk || (order != 0 && order != 1)) return false;   // not a shape this build offers
    t->gram_cols = (int)gc;
    t->split_k = sk;
    t->tc_order = (int)order;
    return true;
  }
  return false;
}

void cache_store(const std::string& path, const std::string& key, const BatchTune& t, double tuned_ms,
                 double default_ms) {
  std::vector<std::string> v = cache_entries(path);
  v.erase(std::remove_if(v.begin(), v.end(), [&](const std::string& x) { return line_key(x) == key; }), v.end());
  char buf[512];
  snprintf(buf, sizeof(buf),
           "{\"key\": \"%s\", \"gram_cols\": %d, \"split_k\": %lld, \"tc_order\": %d, \"tuned_ms\": %.4f, "
           "\"default_ms\": %.4f}",
           key.c_str(), t.gram_cols, (long long)t.split_k, t.tc_order, tuned_ms, default_ms);
  v.push_back(buf);
  const std::string tmp = path + ".tmp";
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return;                                  // an unwritable cache only costs a later search
  fprintf(f, "{\"corutv_autotune\": 1, \"entries\": [\n");
  for (size_t i = 0; i < v.size(); ++i) fprintf(f, "%s%s\n", v[i].c_str(), i + 1 < v.size() ? "," : "");
  fprintf(f, "]}\n");
  fclose(f);
  rename(tmp.c_str(), path.c_str());
}

// Whole-batch time of the plan built with shapes t: one warm run, then the faster of two timed runs.
int time_plan(corutv_handle* h, BatchState* B, int count, const corutv_problem* probs, const BatchTune& t,
              double* ms) {
  int rc = build(h, B, count, probs, t);
  if (rc) return rc;
  rc = enqueue(h, B);
  if (rc) return rc;
  cudaEvent_t e0, e1;
  CUB(cudaEventCreate(&e0));
  CUB(cudaEventCreate(&e1));
  double best = 1e30;
  for (int r = 0; r < 2 && !rc; ++r) {
    CUB(cudaEventRecord(e0, h->stream));
    rc = enqueue(h, B);
    CUB(cudaEventRecord(e1, h->stream));
    CUB(cudaEventSynchronize(e1));
    float f = 0.f;
    CUB(cudaEventElapsedTime(&f, e0, e1));
    best = std::min(best, (double)f);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = best;
  return rc;
}

// Coordinate search over the plan's shapes, timing whole batches (outside any capture: the
// first call of a problem set).  The cache answers first when it holds the key.
int autotune(corutv_handle* h, BatchState* B, int count, const corutv_problem* probs, BatchTune* out) {
  std::vector<char> eng;
  engines(count, probs, eng);
  bool tc = false, simt = false;               // some problems on tensor-core tables / on CUDA cores
  for (char e : eng) {
    tc |= e != kEngSimt;
    simt |= e == kEngSimt;
  }
  const std::string key = tune_key(count, probs, tc);
  BatchTune best;
  for (const auto& kv : B->tuned_keys) {
    if (kv.first != key) continue;
    *out = kv.second;                             // searched before on this handle
    B->tuned = true;
    B->tune_from_cache = true;
    B->tuned_ms = B->default_ms = 0.0;
    return CORUTV_OK;
  }
  if (!h->tune_cache.empty() && cache_lookup(h->tune_cache, key, &best)) {
    *out = best;
    B->tuned = true;
    B->tune_from_cache = true;
    B->tuned_ms = B->default_ms = 0.0;
    return CORUTV_OK;
  }
  const bool was_tracing = h->tracing;
  h->tracing = false;
  double best_ms = 0.0;
  int rc = time_plan(h, B, count, probs, best, &best_ms);
  const double default_ms = best_ms;
  auto try_shape = [&](const BatchTune& cand) {
    if (rc) return;
    double ms = 0.0;
    rc = time_plan(h, B, count, probs, cand, &ms);
    if (!rc && ms < best_ms) {
      best_ms = ms;
      best = cand;
    }
  };
  if (tc) {
    BatchTune c = best;
    c.tc_order = 1;
    try_shape(c);
  }
  for (int gc : kTuneGramCols) {
    if (gc == best.gram_cols) continue;
    BatchTune c = best;
    c.gram_cols = gc;
    try_shape(c);
  }
  if (simt) {
    for (int64_t sk : kTuneSplitK) {
      if (sk == best.split_k) continue;
      BatchTune c = best;
      c.split_k = sk;
      try_shape(c);
    }
  }
  h->tracing = was_tracing;
  if (rc) return rc;
  *out = best;
  B->tuned = true;
  B->tune_from_cache = false;
  B->tuned_ms = best_ms;
  B->default_ms = default_ms;
  B->tuned_keys.emplace_back(key, best);
  if (!h->tune_cache.empty()) cache_store(h->tune_cache, key, best, best_ms, default_ms);
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
  for (int i = 0; i < count; ++i) {
    const int rc = validate(probs[i]);
    if (rc) return rc;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess) {
    cudaGetLastError();
    sms = 160;                                    // no device: an upper bound for the plan
  }
  // the largest plan the autotuner can choose (more Gram partials and K splits than the defaults)
  BatchTune big;
  big.gram_cols = kTuneGramCols[0];
  big.split_k = kTuneSplitK[0];
  Plan L, L2;
  make_plan(L, count, probs, sms, BatchTune{});
  make_plan(L2, count, probs, sms, big);
  *bytes = std::max(L.need, L2.need);
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
  int64_t l0 = launch_counter();
  if (!same_key(B, count, probs)) {
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return CORUTV_ERR_CUDA;
    B->key.clear();
    BatchTune tune;
    B->tuned = B->tune_from_cache = false;
    B->tuned_ms = B->default_ms = 0.0;
    if (h->autotune) {
      B->a_dtype = a_dtype;
      int rc = autotune(h, B, count, probs, &tune);
      if (rc) return rc;
      B->key.clear();
      l0 = launch_counter();                      // the search's runs are not this call's launches
    }
    int rc = build(h, B, count, probs, tune);
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

int corutv_set_autotune(corutv_handle* h, int mode, const char* cache_path) {
  if (!h || (mode != 0 && mode != 1)) return CORUTV_ERR_INVALID_ARG;
  h->autotune = mode;
  if (cache_path) {
    h->tune_cache = cache_path;
  } else {
    const char* env = getenv("CORUTV_AUTOTUNE_CACHE");
    h->tune_cache = env ? env : "";
  }
  if (h->batch) {
    // the next batched call builds a new plan with (or without) tuned shapes
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return CORUTV_ERR_CUDA;
    h->batch->key.clear();
  }
  return CORUTV_OK;
}

int corutv_batch_tuning_read(corutv_handle* h, corutv_batch_tuning* out) {
  if (!h || !out) return CORUTV_ERR_INVALID_ARG;
  memset(out, 0, sizeof(*out));
  const BatchState* B = h->batch;
  if (!B || B->key.empty()) return CORUTV_ERR_INVALID_ARG;
  out->tuned = B->tuned ? 1 : 0;
  out->from_cache = B->tune_from_cache ? 1 : 0;
  out->gram_cols = B->tune.gram_cols;
  out->split_k = (int32_t)B->tune.split_k;
  out->tc_order = B->tune.tc_order;
  out->tuned_ms = B->tuned_ms;
  out->default_ms = B->default_ms;
  return CORUTV_OK;
}

int corutv_batch_info_wait(corutv_handle* h, int count, corutv_info* infos) {
  if (!h || !infos) return CORUTV_ERR_INVALID_ARG;
  BatchState* B = h->batch;
  if (!B || B->count != count || B->key.empty()) return CORUTV_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return CORUTV_ERR_CUDA;
  std::vector<DevStatus> st(count);
  DevStatus bst{};
  if (cudaMemcpy(st.data(), B->dstatus, sizeof(DevStatus) * count, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&bst, B->bstatus, sizeof(DevStatus), cudaMemcpyDeviceToHost) != cudaSuccess)
    return CORUTV_ERR_CUDA;
  for (int i = 0; i < count; ++i) {
    corutv_info& o = infos[i];
    memset(&o, 0, sizeof(o));
    o.status = ((st[i].flags | bst.flags) & kStatTimeout) ? CORUTV_ERR_TIMEOUT : CORUTV_OK;
    o.passes_over_A = B->passes[i];
    o.hbm_passes_over_A = B->hbm_passes[i];
    o.chol_fallbacks = st[i].chol_fallbacks;
    o.chol_shift_rel = kShiftRel32;
    o.fro2_A = B->want_fro2[i] ? st[i].fro2_A : NAN;
    o.fro2_T = st[i].fro2_T;
    o.fro2_Tk = st[i].fro2_Tk;
  }
  return CORUTV_OK;
}

}  // extern "C"
