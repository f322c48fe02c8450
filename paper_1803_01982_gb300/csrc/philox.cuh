// philox.cuh -- Gaussian sketch matrix Omega of Alg. 2 (TRQRCP), drawn on the
// device from the counter-based Philox4x32-10 generator (Salmon, Moraes, Dror
// & Shaw, SC'11) with the Box-Muller transform (Box & Muller, 1958).
//
// Stream definition: element e of stream `stream` under `seed` uses the Philox
// block with counter (q_lo, q_hi, stream, 0), q = e / 4, and key
// (seed_lo, seed_hi); outputs (x0, x1) give elements 4q, 4q+1 as
// r cos(2 pi u2), r sin(2 pi u2) with r = sqrt(-2 ln u1), u = (x + 1/2) 2^-32,
// and (x2, x3) give elements 4q+2, 4q+3 the same way.  Omega(i, j) is element
// i*m + j of stream 0.
#pragma once

#include "common.cuh"

namespace ffq {

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k0;
    const uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// ln(u) for u = (a + 1/2) 2^-32 without losing accuracy near u = 1: for
// a >= 2^31 use log1p(-(1-u)) with 1-u = (~a + 1/2) 2^-32 formed exactly.
__device__ __forceinline__ float log_uniform_f(uint32_t a) {
  if (a < 0x80000000u) return logf(fmaf((float)a, 0x1p-32f, 0x1p-33f));
  const uint32_t b = 0xFFFFFFFFu - a;
  return log1pf(-fmaf((float)b, 0x1p-32f, 0x1p-33f));
}
__device__ __forceinline__ double log_uniform_d(uint32_t a) {
  return log(((double)a + 0.5) * 0x1p-32);
}

// Box-Muller pair from two 32-bit words; FP32 evaluation with the CUDA
// library's logf/log1pf/sincospif (a few FP32 ulps from the FP64 definition).
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float &z0, float &z1) {
  const float rad = sqrtf(-2.0f * log_uniform_f(a));
  float sn, cs;
  sincospif(2.0f * fmaf((float)b, 0x1p-32f, 0x1p-33f), &sn, &cs);
  z0 = rad * cs;
  z1 = rad * sn;
}
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, double &z0, double &z1) {
  const double rad = sqrt(-2.0 * log_uniform_d(a));
  double sn, cs;
  sincospi(2.0 * (((double)b + 0.5) * 0x1p-32), &sn, &cs);
  z0 = rad * cs;
  z1 = rad * sn;
}

// Element e of Gaussian stream `stream` under `seed` (the definition above),
// one Philox block per call.
template <typename T>
__device__ __forceinline__ T gauss_elem(uint64_t seed, uint32_t stream, uint64_t e) {
  const uint64_t q = e >> 2;
  uint32_t c[4] = {(uint32_t)q, (uint32_t)(q >> 32), stream, 0u};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const bool hi = (e & 2u) != 0;
  T z0, z1;
  box_muller(hi ? c[2] : c[0], hi ? c[3] : c[1], z0, z1);
  return (e & 1u) ? z1 : z0;
}

// Omega (s x m), row-major with leading dimension ldm; one thread per Philox
// block (four consecutive stream elements).
template <typename T>
__global__ void omega_kernel(T *__restrict__ Om, int s, int64_t m, int64_t ldm, uint64_t seed) {
  const int64_t total = (int64_t)s * m;
  const int64_t nq = (total + 3) / 4;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq;
       q += (int64_t)gridDim.x * blockDim.x) {
    uint32_t c[4] = {(uint32_t)q, (uint32_t)((uint64_t)q >> 32), 0u, 0u};
    philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    T z[4];
    box_muller(c[0], c[1], z[0], z[1]);
    box_muller(c[2], c[3], z[2], z[3]);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int64_t e = 4 * q + r;
      if (e < total) {
        const int64_t i = e / m, j = e - i * m;
        Om[i * ldm + j] = z[r];
      }
    }
  }
}

// Raw Philox blocks for the known-answer / cross-implementation tests.
__global__ void philox_raw_kernel(const uint32_t *__restrict__ ctr_key, uint32_t *__restrict__ out,
                                  int count) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  uint32_t c[4] = {ctr_key[6 * t + 0], ctr_key[6 * t + 1], ctr_key[6 * t + 2], ctr_key[6 * t + 3]};
  philox4x32_10(c, ctr_key[6 * t + 4], ctr_key[6 * t + 5]);
  for (int r = 0; r < 4; ++r) out[4 * t + r] = c[r];
}

}  // namespace ffq
