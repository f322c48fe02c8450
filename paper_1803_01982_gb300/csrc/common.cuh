// common.cuh -- shared device helpers for the Flip-Flop SRQR kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cfloat>
#include <math.h>

namespace ffq {

// Device-side status word layout (an int array in the workspace).
enum CtlSlot : int {
  CTL_STATUS = 0,      // FFSRQR_STATUS_* (max-combined)
  CTL_TIMEOUT = 1,     // 1 if a bounded wait expired
  CTL_SWAPS = 2,
  CTL_CAND = 3,        // original index of the current SRQR candidate
  CTL_IMAX = 4,        // leaving position of the current swap
  CTL_NEED_SWAP = 5,   // 1 while g2 > g and swaps < cap
  CTL_CAND_FIRST = 6,  // original index of the first SRQR candidate
  CTL_BARRIER0 = 8,    // grid-barrier counters (one per cooperative kernel)
  CTL_BARRIER1 = 9,
  CTL_BARRIER2 = 10,
  CTL_JACOBI_SWEEPS = 11,
  CTL_NONFINITE = 12,
  CTL_SERIES_SKIP = 13,   // 1 while the current second Cholesky-QR factor came from the expansion
  CTL_SERIES = 14,        // second Cholesky-QR sweeps that took the first-order expansion
  CTL_SERIES_EXACT = 15,  // second sweeps that took the exact factorization
  CTL_SWEEP_ROT0 = 16,  // rotations performed in Jacobi sweeps 0..15 (diagnostic)
  CTL_WIN_KEY = 32,     // 3 x uint64 (words 32..37): QRCP winner keys, one per step mod 3
  CTL_QRCP_BARRIERS = 38,  // grid barriers the single-precision QRCP took (diagnostic)
  CTL_WORDS = 40,
};

// Doubles kept beside the control words.
enum DSlot : int {
  D_G2_FIRST = 0,
  D_G2 = 1,
  D_ALPHA = 2,
  D_ALPHA_FIRST = 3,
  D_WORDS = 8,
};

constexpr int STATUS_OK = 0;
constexpr int STATUS_RANK_DEFICIENT = 1;
constexpr int STATUS_SWAP_CAP = 2;
constexpr int STATUS_TIMEOUT = 3;
constexpr int STATUS_NONFINITE = 4;

__device__ __forceinline__ void set_status(int *ctl, int code) { atomicMax(ctl + CTL_STATUS, code); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum; every thread gets the result.  red must hold >= 32 T.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T *red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T t = (threadIdx.x < nw) ? red[threadIdx.x] : T(0);
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  t = red[0];
  __syncthreads();
  return t;
}

template <typename T>
__host__ __device__ __forceinline__ T neg_inf();
template <>
__host__ __device__ __forceinline__ float neg_inf<float>() { return -INFINITY; }
template <>
__host__ __device__ __forceinline__ double neg_inf<double>() { return -HUGE_VAL; }

// Argmax over (value, original index) pairs: the larger value wins, ties go to
// the lowest original column index.  NaN never wins.
template <typename T>
__device__ __forceinline__ bool better(T v1, int i1, T v2, int i2) {
  if (v1 > v2) return true;
  if (v1 == v2) return i1 < i2;
  return !(v2 == v2) && (v1 == v1);  // v2 NaN, v1 not
}

template <typename T>
__device__ __forceinline__ void warp_argmax(T &v, int &i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T w = __shfl_xor_sync(0xffffffffu, v, o);
    int j = __shfl_xor_sync(0xffffffffu, i, o);
    if (better(w, j, v, i)) {
      v = w;
      i = j;
    }
  }
}

// Block-wide argmax; every thread gets the result. redv/redi hold >= 32 entries.
template <typename T>
__device__ __forceinline__ void block_argmax(T &v, int &i, T *redv, int *redi) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  warp_argmax(v, i);
  __syncthreads();
  if (lane == 0) {
    redv[wid] = v;
    redi[wid] = i;
  }
  __syncthreads();
  if (wid == 0) {
    T t = (lane < nw) ? redv[lane] : neg_inf<T>();
    int j = (lane < nw) ? redi[lane] : 0x7fffffff;
    warp_argmax(t, j);
    if (lane == 0) {
      redv[0] = t;
      redi[0] = j;
    }
  }
  __syncthreads();
  v = redv[0];
  i = redi[0];
  __syncthreads();
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Bounded grid barrier for a co-resident (cooperatively launched) grid.  The
// counter only grows: barrier number b (1-based) waits until it reaches
// b * gridDim.x.  A wait that exceeds spin_limit polls sets CTL_TIMEOUT and the
// status, and every block then returns false so the kernel can exit.
__device__ __forceinline__ bool grid_barrier(unsigned *ctr, unsigned target, int *ctl,
                                             long long spin_limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    // release: the block's writes (ordered before by bar.sync) become visible
    // to every block that acquires the counter value
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(ctr), "r"(1u) : "memory");
    int ok = 1;
    long long spins = 0;
    while (ld_acquire_u32(ctr) < target) {
      if ((++spins & 63) == 0 &&
          (*((volatile int *)(ctl + CTL_TIMEOUT)) != 0 || spins > spin_limit)) {
        ok = 0;
        atomicExch(ctl + CTL_TIMEOUT, 1);
        set_status(ctl, STATUS_TIMEOUT);
        break;
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Raise a kernel's dynamic shared-memory cap to the most the device allows for
// it (the opt-in maximum less the kernel's static shared memory).  Every
// caller sets this same value, so host threads that launch one kernel with
// different sizes never lower the cap under one another's launch.
inline cudaError_t smem_cap_max(const void *fn) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  return e;
}

__host__ __device__ __forceinline__ int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ __forceinline__ int64_t round_up(int64_t a, int64_t b) { return cdiv(a, b) * b; }

}  // namespace ffq
