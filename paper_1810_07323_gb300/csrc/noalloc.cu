// corutv_gram_noalloc: the Gram product of corutv_gram for callers that must
// not allocate device memory after start-up -- for example a latency-bound
// loop in which cudaMalloc could synchronise the device, or a process whose
// device memory is entirely handed to another allocator (a framework's
// caching pool), where an extra cudaMalloc may fail or fragment that pool.
//
// The per-CTA partial products live in a fixed, file-scope device array
// instead of a handle workspace.  The array (kNoAllocScratchBytes) exists on a
// GPU once the library's device code is loaded there -- under lazy module
// loading (the default since CUDA 12.2) that happens at the first kernel launch
// or symbol lookup of this library on that device -- and stays until the
// context is destroyed or the process exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/corutv.h"
#include "common.cuh"
#include "internal.h"

namespace corutv {
namespace {

constexpr size_t kNoAllocScratchBytes = CORUTV_NOALLOC_SCRATCH_BYTES;
constexpr int kNoAllocParts = 32;   // partial blocks: 32 x 128 x 128 FP64 = 4 MiB
static_assert((size_t)kNoAllocParts * kMaxL * kMaxL * sizeof(double) <= kNoAllocScratchBytes,
              "scratch too small for the partial blocks");

// Shared by every call on a device: calls whose kernels overlap on the GPU race.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};

// The driver's current context (null if it cannot be queried).
CUcontext current_context() {
  static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
  static bool looked = false;
  if (!looked) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
    looked = true;
  }
  CUcontext c = nullptr;
  if (fn && fn(&c) != CUDA_SUCCESS) c = nullptr;
  return c;
}

// Device address of the scratch array on the current device.  In host code
// the symbol is only a host-side stand-in, so the address is looked up with
// the device current and cached per device together with the context it
// belongs to; a new context on that device (after cudaDeviceReset, say) gets a
// fresh lookup, so a stale address is never handed to a kernel.
int scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CORUTV_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return CORUTV_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  // the runtime makes the device's primary context current on its first call
  // above; query the context after that
  const CUcontext ctx = current_context();
  if (!g_scratch_ptr[dev] || !ctx || ctx != g_scratch_ctx[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      g_scratch_ptr[dev] = nullptr;
      return CORUTV_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
    g_scratch_ctx[dev] = ctx;
  }
  *out = g_scratch_ptr[dev];
  return CORUTV_OK;
}

}  // namespace
}  // namespace corutv

using namespace corutv;

extern "C" int corutv_gram_noalloc(void* stream, int dtype, const void* Xt, int64_t ldx, const void* Yt,
                                   int64_t ldy, int64_t len, int32_t l, double* G) {
  if (!Xt || !Yt || !G) return CORUTV_ERR_INVALID_ARG;
  if (dtype != CORUTV_F32 && dtype != CORUTV_F64) return CORUTV_ERR_INVALID_ARG;
  // the scratch holds kNoAllocParts partial blocks of at most 128 x 128: larger l is rejected
  if (l < 1 || l > kMaxL) return CORUTV_ERR_SHAPE;
  if (len < 1 || ldx < len || ldy < len) return CORUTV_ERR_SHAPE;
  void* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != CORUTV_OK) return rc;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return CORUTV_ERR_CUDA;
  int parts = gram_parts(len, sms);
  if (parts > kNoAllocParts) parts = kNoAllocParts;
  // every partial block is written in full by its CTA before the reduction reads it,
  // so nothing in the scratch has to be cleared between calls
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t err;
  if (dtype == CORUTV_F64)
    err = launch_gram<double, double>(static_cast<const double*>(Xt), ldx, static_cast<const double*>(Yt), ldy, len, l,
                              static_cast<double*>(scratch), parts, G, l, st);
  else
    err = launch_gram<float, double>(static_cast<const float*>(Xt), ldx, static_cast<const float*>(Yt), ldy, len, l,
                             static_cast<float*>(scratch), parts, G, l, st);
  return err == cudaSuccess ? CORUTV_OK : CORUTV_ERR_CUDA;
}
