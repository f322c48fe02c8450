// qrcp_static.cu -- ffsrqr_qrcp_static: the partial QRCP of a sketch (Alg. 1
// applied to B, as inside ffsrqr_run) with every scratch buffer in a
// fixed-size device array of this library, so the call allocates nothing.
//
// It serves callers that cannot allocate device memory at the point of the
// call: a process whose device memory is already handed to its own memory
// pool (or a serving loop that has committed its budget), where a new
// cudaMalloc could fail or would have to wait for memory held elsewhere.
// Such a caller keeps the sketch and the outputs in memory it already owns.
//
// The scratch is one static __device__ array (QS_BYTES, below 1 MiB) that
// every device loading the library holds until the process exits.  In host
// code its name only stands for it: the device address is looked up with
// cudaGetSymbolAddress, with the calling device current, on every call (a
// host-side lookup; the first call on a device also loads the module, so make
// it before any stream capture).  Every call zeroes the part that must start
// at zero (the control words: grid-barrier counter, status) and the
// per-column selection flags with cudaMemsetAsync on its stream.  Because all
// calls on one device share the array, calls whose executions overlap (on
// different streams without an ordering between them) race: serialise them
// on one stream or with events.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/ffsrqr.h"
#include "common.cuh"
#include "qrcp.cuh"

using namespace ffq;

namespace {

constexpr int64_t QS_MAX_N = 65536;  // columns of the sketch
constexpr int64_t QS_MAX_LDS = 256;  // leading dimension of B^T (>= s)
constexpr int QS_MAX_GRID = 256;     // blocks of the cooperative QRCP
constexpr size_t QS_CTL = 256;       // CTL_WORDS control words, zeroed per call
constexpr size_t QS_CVAL = QS_CTL;
constexpr size_t QS_CIDX = QS_CVAL + sizeof(float) * 4 * QS_MAX_GRID;  // bests and bounds, two buffers
constexpr size_t QS_CCOL = QS_CIDX + sizeof(int) * 2 * QS_MAX_GRID;
constexpr size_t QS_SEL = QS_CCOL + sizeof(float) * 2 * QS_MAX_GRID * QS_MAX_LDS;
constexpr size_t QS_BYTES = QS_SEL + sizeof(int) * QS_MAX_N;  // 792,832 bytes
static_assert(QS_CTL >= CTL_WORDS * sizeof(int), "control words");

static __device__ __align__(256) unsigned char g_qrcp_scratch[QS_BYTES];

// Rows of S11 flipped so that its diagonal is non-negative (left
// multiplication by a sign matrix), as the planned path does; one warp per
// row reads the diagonal before any lane writes the row.
__global__ void qs_posdiag_kernel(float *__restrict__ R, int k) {
  const int lane = threadIdx.x & 31;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < k; i += (gridDim.x * blockDim.x) >> 5) {
    const bool neg = R[(int64_t)i * k + i] < 0.f;
    __syncwarp();
    if (neg)
      for (int j = lane; j < k; j += 32) R[(int64_t)i * k + j] = -R[(int64_t)i * k + j];
  }
}

}  // namespace

extern "C" int ffsrqr_qrcp_static(const float *Bt, int64_t n, int32_t s, int64_t lds, int32_t k,
                                  int32_t *piv, float *S11, int32_t *status, void *stream) {
  if (!Bt) return -1;
  if (n < 1) return -2;
  if (s < 1) return -3;
  if (lds < s) return -4;
  if (k < 1 || k > s || k > n) return -5;
  if (!piv) return -6;
  if (!S11) return -7;
  if (n > QS_MAX_N || lds > QS_MAX_LDS) return FFSRQR_STATUS_UNSUPPORTED;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, nsm = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FFSRQR_STATUS_CUDA;
  // the scratch's address on the current device (never cached: a context that
  // was reset and re-created would leave a cached address stale)
  unsigned char *base = nullptr;
  {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_qrcp_scratch) != cudaSuccess || !p) return FFSRQR_STATUS_CUDA;
    base = reinterpret_cast<unsigned char *>(p);
  }
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return FFSRQR_STATUS_CUDA;
  // slab per block in shared memory: the same sizing as the planned path
  const int spad = (int)round_up(s, 4);
  const int gmax = std::min(nsm, QS_MAX_GRID);
  int64_t grid = std::min<int64_t>(gmax, std::max<int64_t>(1, cdiv(n, 16)));
  int cols = 0;
  size_t smem = 0;
  for (;;) {
    cols = (int)cdiv(n, grid);
    smem = ((size_t)cols * spad + cols + spad + qrcp_pair_extra(spad)) * sizeof(float) + 16;
    if (smem + 2048 <= (size_t)optin) break;
    if (grid >= gmax) return FFSRQR_STATUS_UNSUPPORTED;
    grid = std::min<int64_t>(gmax, grid * 2);
  }
  if (smem_cap_max((const void *)qrcp_kernel<float>) != cudaSuccess) return FFSRQR_STATUS_CUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qrcp_kernel<float>, 512, smem) != cudaSuccess ||
      per_sm < 1)
    return FFSRQR_STATUS_UNSUPPORTED;
  int *ctl = reinterpret_cast<int *>(base);
  int *sel = reinterpret_cast<int *>(base + QS_SEL);
  if (cudaMemsetAsync(ctl, 0, QS_CTL, st) != cudaSuccess) return FFSRQR_STATUS_CUDA;
  if (cudaMemsetAsync(sel, 0, (size_t)n * sizeof(int), st) != cudaSuccess) return FFSRQR_STATUS_CUDA;
  QrcpArgs<float> qa;
  qa.Bt = Bt;
  qa.n = n;
  qa.s = s;
  qa.lds = (int)lds;
  qa.k = k;
  qa.piv = piv;
  qa.S11 = S11;
  qa.cand_val = reinterpret_cast<float *>(base + QS_CVAL);
  qa.cand_idx = reinterpret_cast<int *>(base + QS_CIDX);
  qa.cand_col = reinterpret_cast<float *>(base + QS_CCOL);
  qa.sel = sel;
  qa.ctl = ctl;
  qa.spin_limit = 2000000;
  qa.stall_step = -1;
  qa.cols_per_block = cols;
  qa.s_pad = spad;
  void *args[] = {&qa};
  if (cudaLaunchCooperativeKernel((void *)qrcp_kernel<float>, dim3((unsigned)grid), dim3(512), args, smem, st) !=
      cudaSuccess)
    return FFSRQR_STATUS_CUDA;
  qs_posdiag_kernel<<<(unsigned)cdiv((int64_t)k * 32, 256), 256, 0, st>>>(S11, k);
  if (cudaGetLastError() != cudaSuccess) return FFSRQR_STATUS_CUDA;
  if (status && cudaMemcpyAsync(status, ctl + CTL_STATUS, sizeof(int32_t), cudaMemcpyDeviceToDevice, st) !=
                    cudaSuccess)
    return FFSRQR_STATUS_CUDA;
  return 0;
}
