// batch.cu -- many Flip-Flop SRQR problems of uneven sizes as one CUDA graph
// launch, with an autotuner for the number of concurrent streams.
//
// A batch owns one plan per problem (host metadata only) and one workspace
// layout: problem i's workspace is the slice [off_i, off_i + ws_i) of the
// caller's buffer.  ffsrqr_batch_run captures, on first use or when the
// problem pointers change, the whole pipeline of every problem into one graph:
// a capture stream of the batch (the caller's stream may be the legacy stream,
// which cannot be captured) forks into S internal streams, problem i (problems
// ordered by decreasing m*n) goes to stream i mod S, and the streams join back.
// The graph is instantiated once and launched on the caller's stream, one
// cudaGraphLaunch per run, so a batch of hundreds of small problems costs one host launch and the
// device overlaps the small problems' latency-bound phases across streams.
// Phase-batched graphs (ffsrqr_batch_set_phased): the streams run every
// problem up to its small SVD, join, one launch per cluster size takes the
// small SVDs of all single-precision problems together, and the streams fork
// again for the rest of each pipeline (results bitwise those of the plain
// graph).  ffsrqr_batch_tune times the graph for S in {1, 2, 4, 8}, plain and
// phase-batched, and keeps the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/ffsrqr.h"

void ffq_set_last_error(const char *what, cudaError_t e);  // ffsrqr.cu
// phase-batched runs (ffsrqr.cu)
bool ffq_phase_batchable(ffsrqr_plan_t P);
int ffq_run_pre(ffsrqr_plan_t P, const void *A, int64_t lda, uint64_t seed, int32_t *piv, void *workspace,
                cudaStream_t st);
int ffq_run_post(ffsrqr_plan_t P, const void *A, int64_t lda, void *U, int64_t ldu, void *V, int64_t ldv,
                 int32_t *piv, void *workspace, cudaStream_t st, ffsrqr_info_t *info);
int ffq_small_svd_batched(const ffsrqr_plan_t *plans, void *const *workspaces, void *const *S, int count,
                          cudaStream_t st, int *launches);

namespace {

// Records the CUDA error text (ffsrqr_last_cuda_error) and maps it to the
// library status.
int cuda_fail(const char *what, cudaError_t e) {
  ffq_set_last_error(what, e);
  return FFSRQR_STATUS_CUDA;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct ffsrqr_batch_s {
  int count = 0;
  int mode = 0;
  std::vector<ffsrqr_plan_t> plans;
  std::vector<size_t> off, ws;
  std::vector<int> order;  // problems by decreasing m * n
  size_t total = 0;
  int streams = 4;
  std::vector<cudaStream_t> st;
  cudaStream_t cap = nullptr;  // capture origin (the caller's stream may be the legacy stream)
  cudaEvent_t fork = nullptr, fork2 = nullptr;
  std::vector<cudaEvent_t> join;
  int phased = 0;           // phase-batched graph
  int svd_launches = -1;    // batched small-SVD launches in the captured graph (-1: none)
  cudaGraphExec_t exec = nullptr;
  std::vector<ffsrqr_problem_t> key;  // problems the graph was captured with
  void *key_ws = nullptr;
  ffsrqr_info_t *key_info = nullptr;
  int key_streams = 0;
  int key_phased = 0;
};

namespace {

void drop_graph(ffsrqr_batch_s *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->key.clear();
}

bool same_problems(const ffsrqr_batch_s *b, const ffsrqr_problem_t *probs, void *ws, ffsrqr_info_t *infos) {
  if (!b->exec || b->key_ws != ws || b->key_info != infos || b->key_streams != b->streams ||
      b->key_phased != b->phased)
    return false;
  return std::memcmp(b->key.data(), probs, sizeof(ffsrqr_problem_t) * b->count) == 0;
}

int ensure_streams(ffsrqr_batch_s *b) {
  while ((int)b->st.size() < b->streams) {
    cudaStream_t s;
    cudaEvent_t e;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return FFSRQR_STATUS_CUDA;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      cudaStreamDestroy(s);
      return FFSRQR_STATUS_CUDA;
    }
    b->st.push_back(s);
    b->join.push_back(e);
  }
  return 0;
}

// Capture every problem's ffsrqr_run into one graph, from the batch's own
// capture stream forked into its S streams.
int capture(ffsrqr_batch_s *b, const ffsrqr_problem_t *probs, void *workspace, ffsrqr_info_t *infos) {
  int rc;
  if ((rc = ensure_streams(b))) return rc;
  drop_graph(b);
  const int S = b->streams;
  cudaStream_t stream = b->cap;
  cudaError_t ce;
  if ((ce = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
    return cuda_fail("cudaStreamBeginCapture", ce);
  int err = 0;
  if ((ce = cudaEventRecord(b->fork, stream)) != cudaSuccess) err = cuda_fail("cudaEventRecord(fork)", ce);
  for (int s = 0; s < S && !err; ++s)
    if ((ce = cudaStreamWaitEvent(b->st[s], b->fork, 0)) != cudaSuccess) err = cuda_fail("cudaStreamWaitEvent", ce);
  auto join_all = [&]() {
    for (int s = 0; s < S && !err; ++s) {
      if ((ce = cudaEventRecord(b->join[s], b->st[s])) != cudaSuccess ||
          (ce = cudaStreamWaitEvent(stream, b->join[s], 0)) != cudaSuccess)
        err = cuda_fail("join", ce);
    }
  };
  std::vector<ffsrqr_plan_t> bp;  // phase-batched problems, in stream order
  std::vector<void *> bws, bS;
  std::vector<int> bidx;
  for (int j = 0; j < b->count && !err; ++j) {
    const int i = b->order[j];
    const ffsrqr_problem_t &q = probs[i];
    unsigned char *ws = reinterpret_cast<unsigned char *>(workspace) + b->off[i];
    int r;
    if (b->phased && ffq_phase_batchable(b->plans[i])) {
      r = ffq_run_pre(b->plans[i], q.A, q.lda, q.seed, q.piv, ws, b->st[j % S]);
      bp.push_back(b->plans[i]);
      bws.push_back(ws);
      bS.push_back(q.S);
      bidx.push_back(j);
    } else {
      r = ffsrqr_run(b->plans[i], q.A, q.lda, q.seed, q.U, q.ldu, q.S, q.V, q.ldv, q.piv, ws, b->st[j % S],
                     infos ? infos + i : nullptr);
    }
    if (r) err = r;
  }
  join_all();
  b->svd_launches = -1;
  if (!err && !bp.empty()) {
    int nl = 0;
    const int r = ffq_small_svd_batched(bp.data(), bws.data(), bS.data(), (int)bp.size(), stream, &nl);
    if (r) err = r;
    b->svd_launches = nl;
    if (!err && (ce = cudaEventRecord(b->fork2, stream)) != cudaSuccess) err = cuda_fail("cudaEventRecord(fork2)", ce);
    for (int s = 0; s < S && !err; ++s)
      if ((ce = cudaStreamWaitEvent(b->st[s], b->fork2, 0)) != cudaSuccess) err = cuda_fail("cudaStreamWaitEvent", ce);
    for (size_t e = 0; e < bidx.size() && !err; ++e) {
      const int j = bidx[e], i = b->order[j];
      const ffsrqr_problem_t &q = probs[i];
      const int r2 = ffq_run_post(b->plans[i], q.A, q.lda, q.U, q.ldu, q.V, q.ldv, q.piv, bws[e], b->st[j % S],
                                  infos ? infos + i : nullptr);
      if (r2) err = r2;
    }
    join_all();
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(stream, &graph);
  if (err || ec != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    return err ? err : cuda_fail("cudaStreamEndCapture", ec);
  }
  const cudaError_t ei = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    b->exec = nullptr;
    return cuda_fail("cudaGraphInstantiate", ei);
  }
  b->key.assign(probs, probs + b->count);
  b->key_ws = workspace;
  b->key_info = infos;
  b->key_streams = S;
  b->key_phased = b->phased;
  return 0;
}

}  // namespace

extern "C" {

int ffsrqr_batch_create(ffsrqr_batch_t *batch, int32_t count, const int64_t *m, const int64_t *n,
                        const int32_t *k, const int32_t *p, int32_t mode, const ffsrqr_opts_t *opts,
                        int32_t streams, size_t *workspace_bytes) {
  if (!batch) return -1;
  *batch = nullptr;
  if (count < 1) return -2;
  if (!m || !n || !k || !p) return -3;
  if (streams < 1 || streams > 64) return -8;
  if (!workspace_bytes) return -9;
  ffsrqr_batch_s *b = new (std::nothrow) ffsrqr_batch_s();
  if (!b) return FFSRQR_STATUS_WORKSPACE;
  b->count = count;
  b->mode = mode;
  b->streams = streams;
  b->plans.assign(count, nullptr);
  b->off.assign(count, 0);
  b->ws.assign(count, 0);
  for (int i = 0; i < count; ++i) {
    size_t w = 0;
    const int rc = ffsrqr_plan(&b->plans[i], m[i], n[i], k[i], p[i], mode, opts, &w);
    if (rc) {
      ffsrqr_batch_destroy(b);
      return rc;
    }
    b->off[i] = b->total;
    b->ws[i] = w;
    b->total = align256(b->total + w);
  }
  b->order.resize(count);
  std::iota(b->order.begin(), b->order.end(), 0);
  std::stable_sort(b->order.begin(), b->order.end(),
                   [&](int x, int y) { return (double)m[x] * n[x] > (double)m[y] * n[y]; });
  cudaError_t ce;
  if ((ce = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess ||
      (ce = cudaEventCreateWithFlags(&b->fork2, cudaEventDisableTiming)) != cudaSuccess ||
      (ce = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)) != cudaSuccess) {
    ffsrqr_batch_destroy(b);
    return cuda_fail("batch set-up", ce);
  }
  *workspace_bytes = b->total;
  *batch = b;
  return 0;
}

int ffsrqr_batch_run(ffsrqr_batch_t b, const ffsrqr_problem_t *probs, void *workspace, void *stream,
                     ffsrqr_info_t *infos) {
  if (!b) return -1;
  if (!probs) return -2;
  if (!workspace || ((uintptr_t)workspace & 255u)) return -3;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (!same_problems(b, probs, workspace, infos)) {
    const int rc = capture(b, probs, workspace, infos);
    if (rc) return rc;
  }
  const cudaError_t e = cudaGraphLaunch(b->exec, st);
  return (e == cudaSuccess) ? 0 : cuda_fail("cudaGraphLaunch", e);
}

int ffsrqr_batch_tune(ffsrqr_batch_t b, const ffsrqr_problem_t *probs, void *workspace, void *stream,
                      ffsrqr_info_t *infos, int32_t *chosen, float *ms_best) {
  if (!b) return -1;
  if (!probs) return -2;
  if (!workspace || ((uintptr_t)workspace & 255u)) return -3;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return FFSRQR_STATUS_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return FFSRQR_STATUS_CUDA;
  }
  int best = b->streams, best_phased = b->phased;
  float best_ms = -1.f;
  int rc = 0;
  const int cand[4] = {1, 2, 4, 8};
  for (int c = 0; c < 8 && !rc; ++c) {
    b->streams = cand[c % 4];
    b->phased = c / 4;
    if ((rc = ffsrqr_batch_run(b, probs, workspace, stream, infos))) break;  // capture + warm-up
    if (cudaEventRecord(e0, st) != cudaSuccess) {
      rc = FFSRQR_STATUS_CUDA;
      break;
    }
    for (int r = 0; r < 3 && !rc; ++r) rc = ffsrqr_batch_run(b, probs, workspace, stream, infos);
    if (rc) break;
    float t = 0.f;
    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
      rc = FFSRQR_STATUS_CUDA;
      break;
    }
    t /= 3.f;
    if (best_ms < 0.f || t < best_ms) {
      best_ms = t;
      best = cand[c % 4];
      best_phased = c / 4;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->streams = best;
  b->phased = best_phased;
  drop_graph(b);
  if (rc) return rc;
  if (chosen) *chosen = best;
  if (ms_best) *ms_best = best_ms;
  return 0;
}

int ffsrqr_batch_streams(ffsrqr_batch_t b) { return b ? b->streams : -1; }

int ffsrqr_batch_set_phased(ffsrqr_batch_t b, int32_t phased) {
  if (!b) return -1;
  if (phased != 0 && phased != 1) return -2;
  b->phased = phased;
  return 0;
}

int ffsrqr_batch_phased(ffsrqr_batch_t b) { return b ? b->phased : -1; }

int ffsrqr_batch_small_svd_launches(ffsrqr_batch_t b) { return (b && b->exec) ? b->svd_launches : -1; }

int ffsrqr_batch_workspace_offset(ffsrqr_batch_t b, int32_t i, size_t *offset, ffsrqr_plan_t *plan) {
  if (!b) return -1;
  if (i < 0 || i >= b->count) return -2;
  if (offset) *offset = b->off[i];
  if (plan) *plan = b->plans[i];
  return 0;
}

int ffsrqr_batch_destroy(ffsrqr_batch_t b) {
  if (!b) return -1;
  drop_graph(b);
  for (size_t s = 0; s < b->st.size(); ++s) {
    cudaStreamDestroy(b->st[s]);
    cudaEventDestroy(b->join[s]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->fork2) cudaEventDestroy(b->fork2);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (ffsrqr_plan_t pl : b->plans)
    if (pl) ffsrqr_destroy(pl);
  delete b;
  return 0;
}

}  // extern "C"
