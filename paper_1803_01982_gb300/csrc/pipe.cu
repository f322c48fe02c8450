// pipe.cu -- problems with host-resident A and outputs, with the copies
// overlapped with the computation.
//
// Two device buffer sets (A, U, S, V, piv).  Problem i uses set b = i % 2:
//   H2D stream: waits until run i-2 (the last user of set b's A) is done,
//               copies A_i into set b, records in[b];
//   stream:     waits in[b] and until the outputs of problem i-2 have been
//               copied out of set b, runs ffsrqr_run, records run[b];
//   D2H stream: waits run[b], copies U, S, V, piv to the host, records out[b].
// The H2D copy of problem i+1 is enqueued before the D2H copy of problem i,
// on another stream, so it does not queue behind the run it overlaps.
#include <cuda_runtime.h>

#include <new>

#include "../../include/ffsrqr.h"

void ffq_set_last_error(const char *what, cudaError_t e);  // ffsrqr.cu

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int cuda_fail(const char *what, cudaError_t e) {
  ffq_set_last_error(what, e);
  return FFSRQR_STATUS_CUDA;
}

}  // namespace

struct ffsrqr_pipe_s {
  ffsrqr_plan_t plan = nullptr;
  int64_t m = 0, n = 0;
  int k = 0;
  size_t elem = 4;
  int64_t lda = 0;  // device row stride of A (elements, multiple of 4)
  size_t off_a[2], off_u[2], off_s[2], off_v[2], off_piv[2], total = 0;
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_run[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
  cudaEvent_t ev_start = nullptr, ev_done = nullptr;
};

extern "C" {

int ffsrqr_pipe_destroy(ffsrqr_pipe_t q) {
  if (!q) return -1;
  if (q->h2d) cudaStreamSynchronize(q->h2d);
  if (q->d2h) cudaStreamSynchronize(q->d2h);
  for (int b = 0; b < 2; ++b) {
    if (q->ev_in[b]) cudaEventDestroy(q->ev_in[b]);
    if (q->ev_run[b]) cudaEventDestroy(q->ev_run[b]);
    if (q->ev_out[b]) cudaEventDestroy(q->ev_out[b]);
  }
  if (q->ev_start) cudaEventDestroy(q->ev_start);
  if (q->ev_done) cudaEventDestroy(q->ev_done);
  if (q->h2d) cudaStreamDestroy(q->h2d);
  if (q->d2h) cudaStreamDestroy(q->d2h);
  delete q;
  return 0;
}

int ffsrqr_pipe_create(ffsrqr_pipe_t *pipe, ffsrqr_plan_t plan, size_t *device_bytes) {
  if (!pipe) return -1;
  *pipe = nullptr;
  if (!plan) return -2;
  if (!device_bytes) return -3;
  ffsrqr_pipe_s *q = new (std::nothrow) ffsrqr_pipe_s();
  if (!q) return FFSRQR_STATUS_WORKSPACE;
  int32_t k = 0, mode = 0;
  ffsrqr_plan_shape(plan, &q->m, &q->n, &k, nullptr, &mode);
  q->plan = plan;
  q->k = k;
  q->elem = (mode == FFSRQR_FP64) ? 8 : 4;
  q->lda = (q->n + 3) / 4 * 4;
  size_t off = 0;
  for (int b = 0; b < 2; ++b) {
    q->off_a[b] = off;
    off = align256(off + (size_t)q->m * q->lda * q->elem);
    q->off_u[b] = off;
    off = align256(off + (size_t)q->m * k * q->elem);
    q->off_s[b] = off;
    off = align256(off + (size_t)k * q->elem);
    q->off_v[b] = off;
    off = align256(off + (size_t)q->n * k * q->elem);
    q->off_piv[b] = off;
    off = align256(off + (size_t)q->n * sizeof(int32_t));
  }
  q->total = off;
  bool ok = cudaStreamCreateWithFlags(&q->h2d, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&q->d2h, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&q->ev_start, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&q->ev_done, cudaEventDisableTiming) == cudaSuccess;
  for (int b = 0; b < 2 && ok; ++b)
    ok = cudaEventCreateWithFlags(&q->ev_in[b], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&q->ev_run[b], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&q->ev_out[b], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    ffsrqr_pipe_destroy(q);
    return cuda_fail("pipe set-up", cudaGetLastError());
  }
  *device_bytes = q->total;
  *pipe = q;
  return 0;
}

int ffsrqr_pipe_run(ffsrqr_pipe_t q, const ffsrqr_host_problem_t *probs, int32_t count, void *device_mem,
                    void *workspace, void *stream, ffsrqr_info_t *infos) {
  if (!q) return -1;
  if (!probs) return -2;
  if (!device_mem || ((uintptr_t)device_mem & 255u)) return -3;
  if (count < 0) return -4;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  unsigned char *mem = reinterpret_cast<unsigned char *>(device_mem);
  const size_t E = q->elem;
  const int64_t m = q->m, n = q->n, k = q->k;
  for (int i = 0; i < count; ++i) {  // nothing is enqueued for an invalid batch
    const ffsrqr_host_problem_t &pr = probs[i];
    if (!pr.A || pr.lda < n || !pr.U || !pr.S || !pr.V || !pr.piv || pr.ldu < k || pr.ldv < k) return -2;
  }
  cudaError_t e;
  // the side streams start after the work already on the caller's stream
  if ((e = cudaEventRecord(q->ev_start, st)) != cudaSuccess) return cuda_fail("cudaEventRecord", e);
  if ((e = cudaStreamWaitEvent(q->h2d, q->ev_start, 0)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(q->d2h, q->ev_start, 0)) != cudaSuccess)
    return cuda_fail("cudaStreamWaitEvent", e);
  auto h2d = [&](int i) -> int {
    const int b = i & 1;
    const ffsrqr_host_problem_t &pr = probs[i];
    if (i >= 2 && (e = cudaStreamWaitEvent(q->h2d, q->ev_run[b], 0)) != cudaSuccess)
      return cuda_fail("cudaStreamWaitEvent", e);
    if ((e = cudaMemcpy2DAsync(mem + q->off_a[b], q->lda * E, pr.A, pr.lda * E, n * E, m, cudaMemcpyHostToDevice,
                               q->h2d)) != cudaSuccess)
      return cuda_fail("cudaMemcpy2DAsync (A)", e);
    if ((e = cudaEventRecord(q->ev_in[b], q->h2d)) != cudaSuccess) return cuda_fail("cudaEventRecord", e);
    return 0;
  };
  int rc = 0;
  if (count > 0 && (rc = h2d(0))) return rc;
  for (int i = 0; i < count; ++i) {
    const int b = i & 1;
    const ffsrqr_host_problem_t &pr = probs[i];
    if (i + 1 < count && (rc = h2d(i + 1))) return rc;
    if ((e = cudaStreamWaitEvent(st, q->ev_in[b], 0)) != cudaSuccess) return cuda_fail("cudaStreamWaitEvent", e);
    if (i >= 2 && (e = cudaStreamWaitEvent(st, q->ev_out[b], 0)) != cudaSuccess)
      return cuda_fail("cudaStreamWaitEvent", e);
    if ((rc = ffsrqr_run(q->plan, mem + q->off_a[b], q->lda, pr.seed, mem + q->off_u[b], k, mem + q->off_s[b],
                         mem + q->off_v[b], k, reinterpret_cast<int32_t *>(mem + q->off_piv[b]), workspace, st,
                         infos ? infos + i : nullptr)))
      return rc;
    if ((e = cudaEventRecord(q->ev_run[b], st)) != cudaSuccess) return cuda_fail("cudaEventRecord", e);
    if ((e = cudaStreamWaitEvent(q->d2h, q->ev_run[b], 0)) != cudaSuccess ||
        (e = cudaMemcpy2DAsync(pr.U, pr.ldu * E, mem + q->off_u[b], k * E, k * E, m, cudaMemcpyDeviceToHost,
                               q->d2h)) != cudaSuccess ||
        (e = cudaMemcpyAsync(pr.S, mem + q->off_s[b], k * E, cudaMemcpyDeviceToHost, q->d2h)) != cudaSuccess ||
        (e = cudaMemcpy2DAsync(pr.V, pr.ldv * E, mem + q->off_v[b], k * E, k * E, n, cudaMemcpyDeviceToHost,
                               q->d2h)) != cudaSuccess ||
        (e = cudaMemcpyAsync(pr.piv, mem + q->off_piv[b], n * sizeof(int32_t), cudaMemcpyDeviceToHost, q->d2h)) !=
            cudaSuccess ||
        (e = cudaEventRecord(q->ev_out[b], q->d2h)) != cudaSuccess)
      return cuda_fail("output copy", e);
  }
  // the caller's stream waits for the last copies in both directions
  if ((e = cudaEventRecord(q->ev_done, q->d2h)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(st, q->ev_done, 0)) != cudaSuccess ||
      (e = cudaEventRecord(q->ev_done, q->h2d)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(st, q->ev_done, 0)) != cudaSuccess)
    return cuda_fail("join", e);
  return 0;
}

}  // extern "C"
