// Shared device/host helpers of libcorutv (no method arithmetic lives here).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace corutv {

constexpr int kMaxL = 128;        // largest sample size l on the FP32 path (one MMA M tile)
constexpr int kMaxL64 = 128;      // largest l on the FP64 path

// Device status word bits (Handle::status, written by kernels, read by corutv_info_wait).
enum : int { kStatTimeout = 1 };

// Device-side status block (one per handle, in the workspace).
struct DevStatus {
  int flags;            // kStat* bits
  int chol_fallbacks;   // dependent sketch columns replaced
  int timeouts;         // bounded waits that expired
  int orth_skip;        // 1: the last CholeskyQR pass found Q^T Q = I and was skipped
  double fro2_A;
  double fro2_T;
  double fro2_Tk;
};

// ---------------------------------------------------------------------------
// Stream-K split of a (tiles x kb) iteration space over G workers: worker c
// owns the contiguous iterations [start(c), start(c+1)).  A tile covered by a
// single worker is written directly; otherwise every worker writes its
// partial tile into slot 2c (its first tile) or 2c+1 (its last tile) and the
// ordered reduction sums the slots of the tile in worker order, so the result
// does not depend on scheduling.
struct StreamK {
  int64_t tiles, kb, total, G;
  __host__ __device__ StreamK(int64_t tiles_, int64_t kb_, int64_t G_)
      : tiles(tiles_), kb(kb_), total(tiles_ * kb_), G(G_) {}
  __host__ __device__ int64_t start(int64_t c) const { return (c * total) / G; }
  // worker owning iteration x (largest c with start(c) <= x)
  __host__ __device__ int64_t owner(int64_t x) const {
    int64_t c = ((x + 1) * G + total - 1) / total - 1;
    if (c < 0) c = 0;
    if (c > G - 1) c = G - 1;
    return c;
  }
  __host__ __device__ int64_t first_tile(int64_t c) const { return start(c) / kb; }
  __host__ __device__ int slot(int64_t c, int64_t t) const {
    return (int)(2 * c + (first_tile(c) == t ? 0 : 1));
  }
};

__host__ __device__ inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
__host__ __device__ inline int64_t cdiv(int64_t x, int64_t a) { return (x + a - 1) / a; }
__host__ __device__ inline int64_t cdiv_d(int64_t x, int64_t a) { return (x + a - 1) / a; }

// bounded-wait budget for device spins (nanoseconds of %globaltimer)
constexpr unsigned long long kWaitBudgetNs = 2000000000ull;

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Programmatic dependent launch for the chains of small kernels between the passes (Gram
// partials -> reduction -> Cholesky -> Q = C R^-1 -> next Gram).  A kernel launched with
// launch_pdl may start while its predecessor on the stream is still running: pdl_enter, its
// first statement, waits until that predecessor has completed and its writes are visible (a no-op
// for an ordinary launch), then lets the next kernel begin launching, so the launch latency of
// each link overlaps the previous kernel instead of following it.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

#define CU_RET(x)                          \
  do {                                     \
    const cudaError_t e_ = (x);            \
    if (e_ != cudaSuccess) return e_;      \
  } while (0)

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace corutv
