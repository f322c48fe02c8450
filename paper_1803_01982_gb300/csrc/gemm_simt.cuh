// gemm_simt.cuh -- CUDA-core (FFMA / DFMA) GEMM used by the plain-FP32 and FP64
// modes and for the small dense products around the factorisation.
//
//   C(i, j) = sum_l X(i, l) Y(l, j),   0 <= i < M, 0 <= j < N, 0 <= l < K
//   X(i, l) = XM ? X[l*ldx + i] : X[i*ldx + l]      (XM: X stored K x M)
//   Y(l, j) = YN ? Y[l*ldy + j] : Y[j*ldy + l]      (YN: Y stored K x N)
//   C row-major, leading dimension ldc.
// Split-K: blockIdx.z takes K-slice [z*klen, (z+1)*klen); with more than one
// slice the kernel writes partial tiles to part[z][M][N] and splitk_reduce
// sums them in slice order (deterministic).
#pragma once

#include "common.cuh"

namespace ffq {

template <typename T, int BM, int BN, int BK, int TM, int TN, bool XM, bool YN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    gemm_simt_kernel(int M, int N, int K, const T *__restrict__ X, int64_t ldx,
                     const T *__restrict__ Y, int64_t ldy, T *__restrict__ C, int64_t ldc, int klen,
                     T *__restrict__ part, T alpha, T beta) {
  constexpr int NT = (BM / TM) * (BN / TN);
  __shared__ T Xs[BK][BM + 1];
  __shared__ T Ys[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kbeg = blockIdx.z * klen;
  const int kend = min(K, kbeg + klen);
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    // X tile: BM x BK
    for (int e = tid; e < BM * BK; e += NT) {
      int ii, kk;
      if (XM) {
        kk = e / BM;
        ii = e % BM;
      } else {
        ii = e / BK;
        kk = e % BK;
      }
      const int gi = m0 + ii, gk = k0 + kk;
      T v = T(0);
      if (gi < M && gk < kend) v = XM ? X[(int64_t)gk * ldx + gi] : X[(int64_t)gi * ldx + gk];
      Xs[kk][ii] = v;
    }
    // Y tile: BK x BN
    for (int e = tid; e < BN * BK; e += NT) {
      int jj, kk;
      if (YN) {
        kk = e / BN;
        jj = e % BN;
      } else {
        jj = e / BK;
        kk = e % BK;
      }
      const int gj = n0 + jj, gk = k0 + kk;
      T v = T(0);
      if (gj < N && gk < kend) v = YN ? Y[(int64_t)gk * ldy + gj] : Y[(int64_t)gj * ldy + gk];
      Ys[kk][jj] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = Xs[kk][ty + i * (BM / TM)];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Ys[kk][tx + j * (BN / TN)];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  const bool split = gridDim.z > 1;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gi = m0 + ty + i * (BM / TM);
    if (gi >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gj = n0 + tx + j * (BN / TN);
      if (gj >= N) continue;
      if (split) {
        part[((int64_t)blockIdx.z * M + gi) * N + gj] = acc[i][j];
      } else {
        T *c = C + (int64_t)gi * ldc + gj;
        *c = (beta == T(0)) ? alpha * acc[i][j] : alpha * acc[i][j] + beta * (*c);
      }
    }
  }
}

template <typename T>
__global__ void splitk_reduce_kernel(int M, int N, int splits, const T *__restrict__ part,
                                     T *__restrict__ C, int64_t ldc, T alpha, T beta) {
  const int64_t total = (int64_t)M * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    T s = T(0);
    for (int z = 0; z < splits; ++z) s += part[z * total + e];
    const int64_t i = e / N, j = e - i * N;
    T *c = C + i * ldc + j;
    *c = (beta == T(0)) ? alpha * s : alpha * s + beta * (*c);
  }
}

}  // namespace ffq
