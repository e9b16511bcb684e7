// Serving: a request queue in front of corutv_solve_batched.  Each request is
// one CoR-UTV solve (a corutv_problem).  A worker thread forms batches from the
// pending requests (one storage dtype per batch, at most max_slots requests,
// admitted while their HBM footprint -- A as stored plus the batch workspace
// the request needs -- fits the budget) and runs them on two handles with two
// streams in turn, so the next batch is formed and enqueued while the previous
// one runs.  Submit never blocks; poll reports PENDING until a request's batch
// has finished.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/corutv.h"
#include "handle.h"

namespace {

enum ReqState { kPending = 0, kRunning = 1, kDone = 2 };

struct Req {
  uint64_t ticket;
  corutv_problem prob;
  size_t footprint;
};

struct Result {
  int state = kPending;
  int status = CORUTV_PENDING;
  corutv_info info{};
};

struct Inflight {
  std::vector<uint64_t> tickets;
  std::vector<corutv_problem> probs;
  cudaEvent_t done = nullptr;
  bool busy = false;
};

size_t elem_size(int dt) { return dt == CORUTV_F64 ? 8 : (dt == CORUTV_F32 ? 4 : (dt == CORUTV_BF16 ? 2 : 1)); }

}  // namespace

struct corutv_server {
  int device = 0;
  size_t budget = 0;
  int max_slots = 1;
  size_t queue_cap = 1;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req> pending;
  std::unordered_map<uint64_t, Result> results;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  corutv_handle* h[2] = {nullptr, nullptr};
  cudaStream_t st[2] = {nullptr, nullptr};
  Inflight fl[2];
  int64_t batches = 0, solved = 0;
  int64_t launches = 0;     // library kernels the batches launched (direct or in replayed graphs)
};

namespace {

void finish(corutv_server* s, Inflight& f, int rc_run) {
  std::vector<corutv_info> infos(f.tickets.size());
  int rc = rc_run;
  if (rc == CORUTV_OK) {
    const int slot = (int)(&f - s->fl);
    rc = corutv_batch_info_wait(s->h[slot], (int)f.tickets.size(), infos.data());
  }
  std::lock_guard<std::mutex> lk(s->mu);
  for (size_t i = 0; i < f.tickets.size(); ++i) {
    Result& r = s->results[f.tickets[i]];
    r.state = kDone;
    r.status = rc == CORUTV_OK ? infos[i].status : rc;
    if (rc == CORUTV_OK) r.info = infos[i];
  }
  s->solved += (int64_t)f.tickets.size();
  f.tickets.clear();
  f.probs.clear();
  f.busy = false;
}

// Take the next batch from the queue: same dtype as the oldest request, at most
// max_slots, while the footprints fit the budget.  Requests that alone exceed the
// budget fail with ERR_OOM.
void form_batch(corutv_server* s, Inflight& f) {
  std::lock_guard<std::mutex> lk(s->mu);
  size_t used = 0;
  int dt = -1;
  for (auto it = s->pending.begin(); it != s->pending.end() && (int)f.tickets.size() < s->max_slots;) {
    if (it->footprint > s->budget) {
      Result& r = s->results[it->ticket];
      r.state = kDone;
      r.status = CORUTV_ERR_OOM;
      it = s->pending.erase(it);
      continue;
    }
    if (dt < 0) dt = it->prob.a_dtype;
    if (it->prob.a_dtype != dt || used + it->footprint > s->budget) {
      ++it;
      continue;
    }
    used += it->footprint;
    f.tickets.push_back(it->ticket);
    f.probs.push_back(it->prob);
    s->results[it->ticket].state = kRunning;
    it = s->pending.erase(it);
  }
}

void worker_main(corutv_server* s) {
  cudaSetDevice(s->device);
  int turn = 0;
  while (true) {
    bool progressed = false;
    // completions
    for (int i = 0; i < 2; ++i) {
      Inflight& f = s->fl[i];
      if (f.busy && cudaEventQuery(f.done) != cudaErrorNotReady) {
        finish(s, f, CORUTV_OK);
        progressed = true;
      }
    }
    // launch on a free slot
    Inflight& f = s->fl[turn];
    if (!f.busy) {
      form_batch(s, f);
      if (!f.tickets.empty()) {
        const int64_t l0 = s->h[turn]->launches;
        const int rc = corutv_solve_batched(s->h[turn], (int)f.probs.size(), f.probs.data(), nullptr);
        if (rc != CORUTV_OK) {
          finish(s, f, rc);
        } else {
          cudaEventRecord(f.done, s->st[turn]);
          f.busy = true;
          std::lock_guard<std::mutex> lk(s->mu);
          s->batches += 1;
          s->launches += s->h[turn]->launches - l0;
        }
        turn ^= 1;
        progressed = true;
      }
    }
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->stop && s->pending.empty() && !s->fl[0].busy && !s->fl[1].busy) break;
    if (!progressed) {
      if (s->fl[0].busy || s->fl[1].busy)
        s->cv.wait_for(lk, std::chrono::microseconds(20));   // a batch is running: check again soon
      else
        s->cv.wait_for(lk, std::chrono::milliseconds(50), [s] { return s->stop || !s->pending.empty(); });
    }
  }
}

int validate_for_server(const corutv_problem* p, size_t* footprint) {
  size_t ws = 0;
  const int rc = corutv_batch_workspace_size(1, p, &ws);
  if (rc) return rc;
  *footprint = (size_t)p->m * (size_t)p->lda * elem_size(p->a_dtype) + ws;
  return CORUTV_OK;
}

}  // namespace

extern "C" {

int corutv_server_create(corutv_server** out, int device, size_t hbm_budget, int max_slots, int queue_capacity) {
  if (!out || max_slots < 1 || queue_capacity < 1 || hbm_budget == 0) return CORUTV_ERR_INVALID_ARG;
  *out = nullptr;
  corutv_server* s = new (std::nothrow) corutv_server();
  if (!s) return CORUTV_ERR_OOM;
  s->device = device;
  s->budget = hbm_budget;
  s->max_slots = max_slots;
  s->queue_cap = (size_t)queue_capacity;
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) {
    delete s;
    return CORUTV_ERR_CUDA;
  }
  int rc = CORUTV_OK;
  for (int i = 0; i < 2 && rc == CORUTV_OK; ++i) {
    if (cudaStreamCreateWithFlags(&s->st[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->fl[i].done, cudaEventDisableTiming) != cudaSuccess)
      rc = CORUTV_ERR_CUDA;
    else
      rc = corutv_create(&s->h[i], s->st[i]);
  }
  cudaSetDevice(prev);
  if (rc != CORUTV_OK) {
    for (int i = 0; i < 2; ++i) {
      if (s->h[i]) corutv_destroy(s->h[i]);
      if (s->fl[i].done) cudaEventDestroy(s->fl[i].done);
      if (s->st[i]) cudaStreamDestroy(s->st[i]);
    }
    delete s;
    return rc;
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return CORUTV_OK;
}

int corutv_server_submit(corutv_server* s, const corutv_problem* p, uint64_t* ticket) {
  if (!s || !p || !ticket) return CORUTV_ERR_INVALID_ARG;
  size_t fp = 0;
  const int rc = validate_for_server(p, &fp);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return CORUTV_ERR_INVALID_ARG;
    if (s->pending.size() >= s->queue_cap) return CORUTV_ERR_BUSY;
    const uint64_t t = s->next_ticket++;
    s->pending.push_back(Req{t, *p, fp});
    s->results.emplace(t, Result{});
    *ticket = t;
  }
  s->cv.notify_one();
  return CORUTV_OK;
}

int corutv_server_poll(corutv_server* s, uint64_t ticket, corutv_info* info) {
  if (!s) return CORUTV_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->results.find(ticket);
  if (it == s->results.end()) return CORUTV_ERR_INVALID_ARG;
  if (it->second.state != kDone) return CORUTV_PENDING;
  const int status = it->second.status;
  if (info) *info = it->second.info;
  s->results.erase(it);
  return status;
}

int corutv_server_stats(corutv_server* s, int64_t* batches, int64_t* solved, int64_t* pending) {
  if (!s) return CORUTV_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (batches) *batches = s->batches;
  if (solved) *solved = s->solved;
  if (pending) *pending = (int64_t)s->pending.size();
  return CORUTV_OK;
}

int corutv_server_launches(corutv_server* s, int64_t* launches) {
  if (!s || !launches) return CORUTV_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  *launches = s->launches;
  return CORUTV_OK;
}

int corutv_server_destroy(corutv_server* s) {
  if (!s) return CORUTV_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (int i = 0; i < 2; ++i) {
    if (s->h[i]) corutv_destroy(s->h[i]);
    if (s->fl[i].done) cudaEventDestroy(s->fl[i].done);
    if (s->st[i]) cudaStreamDestroy(s->st[i]);
  }
  delete s;
  return CORUTV_OK;
}

}  // extern "C"
