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
//
// Same-phase batching (ffsrqr_server_set_phase_batch): the requests admitted
// in one pass of the scheduler whose small SVD can be batched (single
// precision, SRQR depth k) run their pipelines up to the small SVD on their
// slot streams, a group stream waits for all of them and takes their small
// SVDs in one launch per cluster size, and each slot stream waits for that
// before the rest of its pipeline.  Results are bitwise those of a request
// run alone.  ffsrqr_server_pause holds admission, so that requests
// submitted meanwhile are admitted (and batched) together.
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

// phase-batched runs (ffsrqr.cu)
bool ffq_phase_batchable(ffsrqr_plan_t P);
int ffq_run_pre(ffsrqr_plan_t P, const void *A, int64_t lda, uint64_t seed, int32_t *piv, void *workspace,
                cudaStream_t st);
int ffq_run_post(ffsrqr_plan_t P, const void *A, int64_t lda, void *U, int64_t ldu, void *V, int64_t ldv,
                 int32_t *piv, void *workspace, cudaStream_t st, ffsrqr_info_t *info);
int ffq_small_svd_batched(const ffsrqr_plan_t *plans, void *const *workspaces, void *const *S, int count,
                          cudaStream_t st, int *launches);

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
  std::vector<cudaEvent_t> pre_ev;  // per slot: its request's part before the small SVD
  cudaStream_t grp = nullptr;       // batched small SVDs
  cudaEvent_t grp_ev = nullptr;
  bool phase_batch = false, paused = false;
  int64_t grp_launches = 0, grp_requests = 0;
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

// A request that failed to start: let its stream drain before its
// workspace can be reused.  Caller holds s->mu.
void fail_start(ffsrqr_server_s *s, int64_t t, int rc) {
  Req &rq = s->reqs[t];
  rq.state = 3;
  rq.rc = rc ? rc : FFSRQR_STATUS_CUDA;
  rq.t_done = now_s();
  cudaStreamSynchronize(s->st[rq.slot]);
  s->arena.release(rq.off, rq.need);
  s->slot_req[rq.slot] = -1;
  ++s->completed;
}

// Start the admitted requests (slots and workspaces reserved).  Caller holds
// s->mu.
void start(ffsrqr_server_s *s, const std::vector<int64_t> &adm) {
  // a group needs two batchable requests; a single one runs as usual
  int nb = 0;
  if (s->phase_batch)
    for (int64_t t : adm) nb += ffq_phase_batchable(s->reqs[t].plan) ? 1 : 0;
  std::vector<int64_t> grp;
  for (int64_t t : adm) {
    Req &rq = s->reqs[t];
    if (nb >= 2 && ffq_phase_batchable(rq.plan)) {
      grp.push_back(t);
      continue;
    }
    const ffsrqr_request_t &r = rq.r;
    const int slot = rq.slot;
    const int rc = ffsrqr_run(rq.plan, r.A, r.lda, r.seed, r.U, r.ldu, r.S, r.V, r.ldv, r.piv,
                              s->arena_base + rq.off, s->st[slot], s->slot_info + slot);
    if (rc || cudaEventRecord(s->done_ev[slot], s->st[slot]) != cudaSuccess) {
      fail_start(s, t, rc);
    } else {
      rq.state = 1;
      ++s->admitted;
    }
  }
  if (grp.empty()) return;
  // same-phase batch: parts before the small SVD, one batched small SVD per
  // cluster size on the group stream, then the rest
  int rc = 0;
  std::vector<ffsrqr_plan_t> plans;
  std::vector<void *> wss, Ss;
  for (int64_t t : grp) {
    Req &rq = s->reqs[t];
    const ffsrqr_request_t &r = rq.r;
    void *ws = s->arena_base + rq.off;
    if (!rc) rc = ffq_run_pre(rq.plan, r.A, r.lda, r.seed, r.piv, ws, s->st[rq.slot]);
    if (!rc && cudaEventRecord(s->pre_ev[rq.slot], s->st[rq.slot]) != cudaSuccess) rc = FFSRQR_STATUS_CUDA;
    if (!rc && cudaStreamWaitEvent(s->grp, s->pre_ev[rq.slot], 0) != cudaSuccess) rc = FFSRQR_STATUS_CUDA;
    plans.push_back(rq.plan);
    wss.push_back(ws);
    Ss.push_back(r.S);
  }
  int nl = 0;
  if (!rc) rc = ffq_small_svd_batched(plans.data(), wss.data(), Ss.data(), (int)plans.size(), s->grp, &nl);
  if (!rc && cudaEventRecord(s->grp_ev, s->grp) != cudaSuccess) rc = FFSRQR_STATUS_CUDA;
  for (size_t e = 0; e < grp.size(); ++e) {
    Req &rq = s->reqs[grp[e]];
    const ffsrqr_request_t &r = rq.r;
    const int slot = rq.slot;
    int rr = rc;
    if (!rr && cudaStreamWaitEvent(s->st[slot], s->grp_ev, 0) != cudaSuccess) rr = FFSRQR_STATUS_CUDA;
    if (!rr)
      rr = ffq_run_post(rq.plan, r.A, r.lda, r.U, r.ldu, r.V, r.ldv, r.piv, wss[e], s->st[slot],
                        s->slot_info + slot);
    if (!rr && cudaEventRecord(s->done_ev[slot], s->st[slot]) != cudaSuccess) rr = FFSRQR_STATUS_CUDA;
    if (rr) {
      if (!rc) cudaStreamSynchronize(s->grp);
      fail_start(s, grp[e], rr);
    } else {
      rq.state = 1;
      ++s->admitted;
    }
  }
  if (!rc) {
    s->grp_launches += nl;
    s->grp_requests += (int64_t)grp.size();
  }
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
    // admit queued requests in arrival order: first take slots and memory,
    // then start them (together, when same-phase batching is on)
    std::vector<int64_t> adm;
    while (!s->paused && !s->queue.empty()) {
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
      s->slot_req[slot] = t;  // reserved; reset below if the start fails
      adm.push_back(t);
    }
    if (!adm.empty()) {
      start(s, adm);
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
  s->pre_ev.assign(slots, nullptr);
  s->slot_req.assign(slots, -1);
  bool ok = cudaHostAlloc(&s->slot_info, sizeof(ffsrqr_info_t) * slots, cudaHostAllocDefault) == cudaSuccess;
  for (int k = 0; k < slots && ok; ++k) {
    ok = cudaStreamCreateWithFlags(&s->st[k], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&s->done_ev[k], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&s->pre_ev[k], cudaEventDisableTiming) == cudaSuccess;
  }
  ok = ok && cudaStreamCreateWithFlags(&s->grp, cudaStreamNonBlocking) == cudaSuccess &&
       cudaEventCreateWithFlags(&s->grp_ev, cudaEventDisableTiming) == cudaSuccess;
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

int ffsrqr_server_set_phase_batch(ffsrqr_server_t s, int32_t on) {
  if (!s) return -1;
  if (on != 0 && on != 1) return -2;
  std::lock_guard<std::mutex> lock(s->mu);
  s->phase_batch = (on == 1);
  return 0;
}

int ffsrqr_server_pause(ffsrqr_server_t s, int32_t paused) {
  if (!s) return -1;
  if (paused != 0 && paused != 1) return -2;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->paused = (paused == 1);
  }
  s->cv.notify_all();
  return 0;
}

int ffsrqr_server_phase_stats(ffsrqr_server_t s, int64_t *small_svd_launches, int64_t *grouped_requests) {
  if (!s) return -1;
  std::lock_guard<std::mutex> lock(s->mu);
  if (small_svd_launches) *small_svd_launches = s->grp_launches;
  if (grouped_requests) *grouped_requests = s->grp_requests;
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
    if (s->pre_ev[k]) cudaEventDestroy(s->pre_ev[k]);
  }
  if (s->grp) {
    cudaStreamSynchronize(s->grp);
    cudaStreamDestroy(s->grp);
  }
  if (s->grp_ev) cudaEventDestroy(s->grp_ev);
  for (auto &kv : s->plans) ffsrqr_destroy(kv.second.first);
  if (s->slot_info) cudaFreeHost(s->slot_info);
  if (s->arena_base) cudaFree(s->arena_base);
  delete s;
  return 0;
}

}  // extern "C"
