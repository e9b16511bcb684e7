// The handle behind corutv_handle* (shared by the C-ABI translation units).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/corutv.h"
#include "common.cuh"

namespace corutv {
struct BatchState;                  // batched-solve plan, workspace and graph cache (batched.cu)
void batch_state_free(BatchState* b);
}  // namespace corutv

enum Phase { kPhPass = 0, kPhOrth, kPhCore, kPhQrcp, kPhAsm, kPhFro2, kPhCorr, kPhQuant, kPhPassKernel, kNumPh };

struct TraceRec {
  int phase;
  cudaEvent_t a, b;
  double bytes;
};

// Ring of device buffers through which corutv_solve_host streams a host-resident A, one
// row chunk at a time, on a copy stream that runs ahead of the passes.
struct HostRing {
  static constexpr int kBufs = 3;
  cudaStream_t copy = nullptr;                     // host -> device copies
  cudaEvent_t filled[kBufs] = {}, freed[kBufs] = {};
  cudaEvent_t start = nullptr;                     // the solve's work may begin (ring free)
  void* mem = nullptr;                             // ring buffers, ATY accumulator, per-chunk ||A||^2
  size_t bytes = 0;
};

struct corutv_handle {
  cudaStream_t stream = nullptr;
  bool tracing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<TraceRec> recs;
  corutv_trace acc{};
  int64_t launches = 0;
  int device = 0;
  int sms = 0;
  void* ws = nullptr;          // workspace base (owned if own_ws)
  size_t ws_bytes = 0;
  bool own_ws = false;
  corutv::DevStatus* status = nullptr; // inside the workspace
  corutv_params last{};
  int last_passes = 0;
  double last_shift = 0.0;
  bool have_last = false;
  corutv::BatchState* batch = nullptr;
  void* rpca_ws = nullptr;      // factors of the ALM-CoRUTV iterations (rpca.cu), lazily allocated
  size_t rpca_ws_bytes = 0;
  HostRing ring;
  void* resid_ws = nullptr;     // vectors of the spectral readout (resid.cu), lazily allocated
  size_t resid_ws_bytes = 0;
  int autotune = 0;             // batched solves: 1 = search (or read from the cache) the plan's shapes
  std::string tune_cache;       // JSON cache of tuned shapes ("" = none)
};

void rpca_free(corutv_handle* h);
namespace corutv {
void resid_free(corutv_handle* h);
}
void ring_free(corutv_handle* h);


inline cudaEvent_t ev_get(corutv_handle* h) {
  if (!h->ev_pool.empty()) {
    cudaEvent_t e = h->ev_pool.back();
    h->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// RAII phase timer: records an event pair on the handle's stream when tracing.
struct PhaseTimer {
  corutv_handle* h;
  int phase;
  double bytes;
  cudaEvent_t a = nullptr;
  PhaseTimer(corutv_handle* h_, int ph, double by = 0.0) : h(h_), phase(ph), bytes(by) {
    if (h->tracing) {
      a = ev_get(h);
      cudaEventRecord(a, h->stream);
    }
  }
  ~PhaseTimer() {
    if (h->tracing && a) {
      cudaEvent_t b = ev_get(h);
      cudaEventRecord(b, h->stream);
      h->recs.push_back(TraceRec{phase, a, b, bytes});
    }
  }
};
