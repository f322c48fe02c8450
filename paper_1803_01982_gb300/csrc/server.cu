// server.cu -- a truncated-SVD request server: admission under a device
// memory budget, continuous batching over concurrent streams, latency per
// request.
//
// The server owns one device arena of budget bytes, carved first-fit into
// the workspaces of admitted requests, and S slots (one stream each).  The
// caller owns each request's A and outputs (device memory).  A scheduler
// thread of the server loops:
//   - reap: a slot whose completion event has fired is marked done, its
//     report copied out and its workspace returned to the arena;
//   - admit: queued requests, in arrival order, start as soon as a slot is
//     free and the arena has room for their workspace, so requests that
//     arrive while others run are admitted as resources free up and their
//     kernels overlap on the device (different streams).
// Plans are cached by (m, n, k, p, mode).  A request whose workspace exceeds
// the whole budget is refused at submission (FFSRQR_STATUS_WORKSPACE).
// Latency = completion seen by the scheduler - submission (host steady clock).
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "../../include/ffsrqr.h"

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Req {
  ffsrqr_request_t r;
  ffsrqr_plan_t plan = nullptr;
  size_t need = 0, off = 0;
  int state = 0;  // 0 queued, 1 running, 2 done, 3 failed
  int rc = 0;
  int slot = -1;
  double t_submit = 0, t_done = 0;
  ffsrqr_info_t info{};
};

// First-fit allocator over [0, size) with coalescing of free ranges.
struct Arena {
  std::map<size_t, size_t> free_;  // offset -> length
  explicit Arena(size_t size = 0) {
    if (size) free_[0] = size;
  }
  bool alloc(size_t len, size_t *off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= len) {
        *off = it->first;
        const size_t rest = it->second - len, at = it->first + len;
        free_.erase(it);
        if (rest) free_[at] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t len) {
    auto it = free_.emplace(off, len).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct ffsrqr_server_s {
  int device = 0;
  size_t budget = 0;
  unsigned char *arena_base = nullptr;
  Arena arena;
  int slots = 0;
  std::vector<cudaStream_t> st;
  std::vector<cudaEvent_t> done_ev;
  std::vector<int64_t> slot_req;  // ticket running in the slot, -1 if free
  ffsrqr_info_t *slot_info = nullptr;  // pinned, one per slot
  ffsrqr_opts_t opts{};
  bool has_opts = false;
  std::map<std::tuple<int64_t, int64_t, int, int, int>, std::pair<ffsrqr_plan_t, size_t>> plans;
  std::unordered_map<int64_t, Req> reqs;
  std::deque<int64_t> queue;
  int64_t next_ticket = 1;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::thread worker;
  int64_t admitted = 0, completed = 0;
};

namespace {

// Caller holds s->mu.
int plan_for(ffsrqr_server_s *s, const ffsrqr_request_t &r, ffsrqr_plan_t *plan, size_t *need) {
  const auto key = std::make_tuple(r.m, r.n, r.k, r.p, r.mode);
  auto it = s->plans.find(key);
  if (it == s->plans.end()) {
    ffsrqr_plan_t p = nullptr;
    size_t w = 0;
    const int rc = ffsrqr_plan(&p, r.m, r.n, r.k, r.p, r.mode, s->has_opts ? &s->opts : nullptr, &w);
    if (rc) return rc;
    it = s->plans.emplace(key, std::make_pair(p, align256(w))).first;
  }
  *plan = it->second.first;
  *need = it->second.second;
  return 0;
}

void scheduler(ffsrqr_server_s *s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lock(s->mu);
  while (!s->stop) {
    bool progress = false;
    // reap finished slots
    for (int k = 0; k < s->slots; ++k) {
      const int64_t t = s->slot_req[k];
      if (t < 0) continue;
      const cudaError_t q = cudaEventQuery(s->done_ev[k]);
      if (q == cudaErrorNotReady) continue;
      Req &rq = s->reqs[t];
      rq.t_done = now_s();
      rq.info = s->slot_info[k];
      rq.state = (q == cudaSuccess) ? 2 : 3;
      if (q != cudaSuccess) rq.rc = FFSRQR_STATUS_CUDA;
      s->arena.release(rq.off, rq.need);
      s->slot_req[k] = -1;
      ++s->completed;
      progress = true;
    }
    // admit queued requests in arrival order
    while (!s->queue.empty()) {
      int slot = -1;
      for (int k = 0; k < s->slots; ++k)
        if (s->slot_req[k] < 0) {
          slot = k;
          break;
        }
      if (slot < 0) break;
      const int64_t t = s->queue.front();
      Req &rq = s->reqs[t];
      size_t off = 0;
      if (!s->arena.alloc(rq.need, &off)) break;  // wait for memory (no overtaking)
      s->queue.pop_front();
      rq.off = off;
      rq.slot = slot;
      const ffsrqr_request_t &r = rq.r;
      const int rc = ffsrqr_run(rq.plan, r.A, r.lda, r.seed, r.U, r.ldu, r.S, r.V, r.ldv, r.piv,
                                s->arena_base + off, s->st[slot], s->slot_info + slot);
      if (rc || cudaEventRecord(s->done_ev[slot], s->st[slot]) != cudaSuccess) {
        rq.state = 3;
        rq.rc = rc ? rc : FFSRQR_STATUS_CUDA;
        rq.t_done = now_s();
        // let the stream drain before the workspace can be reused
        cudaStreamSynchronize(s->st[slot]);
        s->arena.release(off, rq.need);
        ++s->completed;
      } else {
        rq.state = 1;
        s->slot_req[slot] = t;
        ++s->admitted;
      }
      progress = true;
    }
    if (progress) s->cv.notify_all();
    // poll again soon; submissions wake the thread at once
    s->cv.wait_for(lock, std::chrono::microseconds(20));
  }
}

}  // namespace

extern "C" {

int ffsrqr_server_create(ffsrqr_server_t *server, size_t budget_bytes, int32_t slots, const ffsrqr_opts_t *opts) {
  if (!server) return -1;
  *server = nullptr;
  if (budget_bytes < 4096) return -2;
  if (slots < 1 || slots > 64) return -3;
  ffsrqr_server_s *s = new (std::nothrow) ffsrqr_server_s();
  if (!s) return FFSRQR_STATUS_WORKSPACE;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return FFSRQR_STATUS_CUDA;
  }
  s->budget = budget_bytes & ~(size_t)255;
  if (cudaMalloc(&s->arena_base, s->budget) != cudaSuccess) {
    delete s;
    return FFSRQR_STATUS_WORKSPACE;
  }
  s->arena = Arena(s->budget);
  s->slots = slots;
  s->st.assign(slots, nullptr);
  s->done_ev.assign(slots, nullptr);
  s->slot_req.assign(slots, -1);
  bool ok = cudaHostAlloc(&s->slot_info, sizeof(ffsrqr_info_t) * slots, cudaHostAllocDefault) == cudaSuccess;
  for (int k = 0; k < slots && ok; ++k) {
    ok = cudaStreamCreateWithFlags(&s->st[k], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&s->done_ev[k], cudaEventDisableTiming) == cudaSuccess;
  }
  if (opts) {
    s->opts = *opts;
    s->has_opts = true;
  }
  if (!ok) {
    ffsrqr_server_destroy(s);
    return FFSRQR_STATUS_CUDA;
  }
  s->worker = std::thread(scheduler, s);
  *server = s;
  return 0;
}

int ffsrqr_server_submit(ffsrqr_server_t s, const ffsrqr_request_t *req, int64_t *ticket) {
  if (!s) return -1;
  if (!req || !req->A || !req->U || !req->S || !req->V || !req->piv) return -2;
  if (!ticket) return -3;
  std::lock_guard<std::mutex> lock(s->mu);
  Req rq;
  rq.r = *req;
  const int rc = plan_for(s, *req, &rq.plan, &rq.need);
  if (rc) return rc;
  if (rq.need > s->budget) return FFSRQR_STATUS_WORKSPACE;  // can never be admitted
  rq.t_submit = now_s();
  const int64_t t = s->next_ticket++;
  s->reqs.emplace(t, rq);
  s->queue.push_back(t);
  *ticket = t;
  s->cv.notify_all();
  return 0;
}

int ffsrqr_server_poll(ffsrqr_server_t s, int64_t ticket, ffsrqr_info_t *info, double *latency_s) {
  if (!s) return -1;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return -2;
  const Req &rq = it->second;
  if (rq.state < 2) return 1;
  if (info) *info = rq.info;
  if (latency_s) *latency_s = rq.t_done - rq.t_submit;
  const int rc = (rq.state == 2) ? 0 : (rq.rc ? rq.rc : FFSRQR_STATUS_CUDA);
  s->reqs.erase(it);  // a final status is reported once
  return rc;
}

int ffsrqr_server_wait(ffsrqr_server_t s, int64_t ticket, ffsrqr_info_t *info, double *latency_s) {
  if (!s) return -1;
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return -2;
  s->cv.wait(lock, [&] { return it->second.state >= 2 || s->stop; });
  const Req &rq = it->second;
  if (rq.state < 2) return FFSRQR_STATUS_CUDA;
  if (info) *info = rq.info;
  if (latency_s) *latency_s = rq.t_done - rq.t_submit;
  const int rc = (rq.state == 2) ? 0 : (rq.rc ? rq.rc : FFSRQR_STATUS_CUDA);
  s->reqs.erase(it);  // a final status is reported once
  return rc;
}

int ffsrqr_server_stats(ffsrqr_server_t s, int64_t *admitted, int64_t *completed, int64_t *queued,
                        size_t *arena_free) {
  if (!s) return -1;
  std::lock_guard<std::mutex> lock(s->mu);
  if (admitted) *admitted = s->admitted;
  if (completed) *completed = s->completed;
  if (queued) *queued = (int64_t)s->queue.size();
  if (arena_free) {
    size_t f = 0;
    for (const auto &kv : s->arena.free_) f += kv.second;
    *arena_free = f;
  }
  return 0;
}

int ffsrqr_server_destroy(ffsrqr_server_t s) {
  if (!s) return -1;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (int k = 0; k < s->slots; ++k) {
    if (s->st[k]) {
      cudaStreamSynchronize(s->st[k]);
      cudaStreamDestroy(s->st[k]);
    }
    if (s->done_ev[k]) cudaEventDestroy(s->done_ev[k]);
  }
  for (auto &kv : s->plans) ffsrqr_destroy(kv.second.first);
  if (s->slot_info) cudaFreeHost(s->slot_info);
  if (s->arena_base) cudaFree(s->arena_base);
  delete s;
  return 0;
}

}  // extern "C"
