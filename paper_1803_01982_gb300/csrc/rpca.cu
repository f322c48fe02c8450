// rpca.cu -- robust PCA by the inexact augmented Lagrange multiplier method
// (Alg. 7, Sec. 3.2) with Flip-Flop SRQR (Alg. 9) as the truncated SVD.
//
//   min ||X||_* + lambda ||E||_1  subject to  M = X + E
//
// Start: J = max(||M||_2, ||M||_max), Y = M / J, E = 0, mu = mu0.  Iteration:
//   U S V^T = Alg. 9 of Z = M - E + Y/mu at the predicted rank sv
//   X = U S_{1/mu}(S) V^T            (the svp singular values above 1/mu)
//   E = S_{lambda/mu}(M - X + Y/mu)  (entrywise soft shrinkage)
//   Y = Y + mu (M - X - E),  mu = min(rho mu, mu_bar)
// until ||M - X - E||_F < tol ||M||_F, or until the residual stalls below
// 100 tol (its rounding floor; the FP32 modes reach it near 1e-6 at 2000^2).
// One fused kernel does the E, Y and
// residual updates and already writes the next iteration's Z, so each
// iteration reads M, X, Y once and writes E, Y, Z once besides Alg. 9 and the
// rank-svp product X = U' V^T.  The host reads S and two scalars back per
// iteration: the predicted-rank rule and the stopping test need them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "../../include/ffsrqr.h"

void ffq_set_last_error(const char *what, cudaError_t e);  // ffsrqr.cu
int ffq_gemm_nt(ffsrqr_plan_t P, int64_t m, int64_t n, int r, const void *U, int64_t ldu, const void *V,
                int64_t ldv, void *X, int64_t ldx, void *workspace, cudaStream_t st, int *launches);  // ffsrqr.cu

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Reduction results of one kernel: sum of squares (double), count, and the
// bit pattern of a non-negative maximum (ordered like the value).
struct Stats {
  double sumsq;
  unsigned long long count;
  unsigned long long maxbits;
  double pad;
};

template <typename T>
__device__ __forceinline__ unsigned long long abs_bits(T v);
template <>
__device__ __forceinline__ unsigned long long abs_bits<float>(float v) {
  return (unsigned long long)__float_as_uint(fabsf(v));
}
template <>
__device__ __forceinline__ unsigned long long abs_bits<double>(double v) {
  return (unsigned long long)__double_as_longlong(fabs(v));
}

// Block reduction of (sumsq, count, maxbits) into st with one atomic each.
__device__ void block_reduce_stats(double ss, unsigned long long cnt, unsigned long long mx, Stats *st) {
  __shared__ double s_ss[32];
  __shared__ unsigned long long s_cnt[32], s_mx[32];
  for (int o = 16; o > 0; o >>= 1) {
    ss += __shfl_down_sync(0xffffffffu, ss, o);
    cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    const unsigned long long t = __shfl_down_sync(0xffffffffu, mx, o);
    mx = t > mx ? t : mx;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    s_ss[warp] = ss;
    s_cnt[warp] = cnt;
    s_mx[warp] = mx;
  }
  __syncthreads();
  if (warp == 0) {
    ss = lane < nw ? s_ss[lane] : 0.0;
    cnt = lane < nw ? s_cnt[lane] : 0ull;
    mx = lane < nw ? s_mx[lane] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      ss += __shfl_down_sync(0xffffffffu, ss, o);
      cnt += __shfl_down_sync(0xffffffffu, cnt, o);
      const unsigned long long t = __shfl_down_sync(0xffffffffu, mx, o);
      mx = t > mx ? t : mx;
    }
    if (lane == 0) {
      atomicAdd(&st->sumsq, ss);
      atomicAdd(&st->count, cnt);
      atomicMax(&st->maxbits, mx);
    }
  }
}

// ||M||_F^2 and max |M_ij|.
template <typename T>
__global__ void __launch_bounds__(256) norms_kernel(const T *__restrict__ M, int64_t ldm, int64_t m, int64_t n,
                                                   Stats *st) {
  double ss = 0.0;
  unsigned long long mx = 0ull;
  for (int64_t i = blockIdx.x; i < m; i += gridDim.x)
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
      const T v = M[i * ldm + j];
      ss += (double)v * (double)v;
      const unsigned long long b = abs_bits<T>(v);
      mx = b > mx ? b : mx;
    }
  block_reduce_stats(ss, 0ull, mx, st);
}

// E = 0, Y = M / J, Z = M + Y / mu.
template <typename T>
__global__ void __launch_bounds__(256) init_kernel(const T *__restrict__ M, int64_t ldm, T *__restrict__ E,
                                                  int64_t lde, T *__restrict__ Y, T *__restrict__ Z, int64_t ldz,
                                                  int64_t m, int64_t n, T inv_j, T inv_mu) {
  for (int64_t i = blockIdx.x; i < m; i += gridDim.x)
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
      const T mv = M[i * ldm + j];
      const T y = mv * inv_j;
      E[i * lde + j] = T(0);
      Y[i * ldz + j] = y;
      Z[i * ldz + j] = mv + y * inv_mu;
    }
}

// U(:, j) *= S_j - tau for j < r (the shrunk singular values).
template <typename T>
__global__ void __launch_bounds__(256) shrink_cols_kernel(T *__restrict__ U, int64_t ldu, int64_t m, int r,
                                                         const T *__restrict__ S, T tau) {
  const int64_t total = m * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / r;
    const int j = (int)(e - i * r);
    U[i * ldu + j] *= S[j] - tau;
  }
}

// One IALM update per entry: t = M - X + Y/mu, E = S_{lambda/mu}(t),
// R = M - X - E, Y += mu R, Z = M - E + Y/mu_next; sums R^2 and counts E != 0.
template <typename T>
__global__ void __launch_bounds__(256) ialm_update_kernel(const T *__restrict__ M, int64_t ldm,
                                                         const T *__restrict__ X, int64_t ldx, T *__restrict__ E,
                                                         int64_t lde, T *__restrict__ Y, T *__restrict__ Z,
                                                         int64_t ldz, int64_t m, int64_t n, T mu, T inv_mu,
                                                         T thr, T inv_mu_next, Stats *st) {
  double ss = 0.0;
  unsigned long long cnt = 0ull;
  for (int64_t i = blockIdx.x; i < m; i += gridDim.x)
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
      const T mv = M[i * ldm + j];
      const T xv = X[i * ldx + j];
      T y = Y[i * ldz + j];
      const T d = mv - xv;
      const T t = d + y * inv_mu;
      const T a = fabs(t) - thr;
      const T ev = a > T(0) ? copysign(a, t) : T(0);
      const T r = d - ev;
      y += mu * r;
      E[i * lde + j] = ev;
      Y[i * ldz + j] = y;
      Z[i * ldz + j] = mv - ev + y * inv_mu_next;
      ss += (double)r * (double)r;
      cnt += ev != T(0) ? 1ull : 0ull;
    }
  block_reduce_stats(ss, cnt, 0ull, st);
}

int cuda_fail(const char *what, cudaError_t e) {
  ffq_set_last_error(what, e);
  return FFSRQR_STATUS_CUDA;
}

}  // namespace

struct ffsrqr_rpca_s {
  int64_t m = 0, n = 0, ldz = 0;
  int mode = 0, kmax = 0, p = 0, sv0 = 0, max_iter = 0;
  size_t elem = 4;
  double lambda = 0, rho = 0, mu_bar_ratio = 0, tol = 0;
  ffsrqr_opts_t fopts{};
  size_t ws_ffsrqr = 0, off_y = 0, off_z = 0, off_u = 0, off_s = 0, off_v = 0, off_piv = 0, off_st = 0, total = 0;
  std::map<int, ffsrqr_plan_t> plans;  // Alg. 9 plans by rank, made on first use
  int num_sms = 0;
  int launches = 0;
};

namespace {

int get_plan(ffsrqr_rpca_s *R, int k, ffsrqr_plan_t *out) {
  auto it = R->plans.find(k);
  if (it != R->plans.end()) {
    *out = it->second;
    return 0;
  }
  ffsrqr_plan_t pl = nullptr;
  size_t w = 0;
  const int rc = ffsrqr_plan(&pl, R->m, R->n, k, R->p, R->mode, &R->fopts, &w);
  if (rc != 0) return rc;
  if (w > R->ws_ffsrqr) {
    ffsrqr_destroy(pl);
    return FFSRQR_STATUS_WORKSPACE;
  }
  R->plans[k] = pl;
  *out = pl;
  return 0;
}

template <typename T>
int rpca_impl(ffsrqr_rpca_s *R, const T *M, int64_t ldm, T *X, int64_t ldx, T *E, int64_t lde, uint64_t seed,
              unsigned char *ws, cudaStream_t st, ffsrqr_rpca_info_t *info) {
  const int64_t m = R->m, n = R->n, ldz = R->ldz;
  const int kmax = R->kmax;
  T *Y = reinterpret_cast<T *>(ws + R->off_y);
  T *Z = reinterpret_cast<T *>(ws + R->off_z);
  T *U = reinterpret_cast<T *>(ws + R->off_u);
  T *S = reinterpret_cast<T *>(ws + R->off_s);
  T *V = reinterpret_cast<T *>(ws + R->off_v);
  int32_t *piv = reinterpret_cast<int32_t *>(ws + R->off_piv);
  Stats *dst = reinterpret_cast<Stats *>(ws + R->off_st);
  // elementwise kernels: one row per block step, 256 threads across the row
  const unsigned grid = (unsigned)std::min<int64_t>(m, (int64_t)R->num_sms * 8);
  int launches = 0, rc = 0;
  cudaError_t e;
  Stats hs{};
  std::vector<T> hS(kmax);
  auto fetch_stats = [&]() -> int {
    if ((e = cudaMemcpyAsync(&hs, dst, sizeof(Stats), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return cuda_fail("rpca stats", e);
    return 0;
  };
  // ||M||_F, ||M||_max
  if ((e = cudaMemsetAsync(dst, 0, sizeof(Stats), st)) != cudaSuccess) return cuda_fail("memset", e);
  norms_kernel<T><<<grid, 256, 0, st>>>(M, ldm, m, n, dst);
  ++launches;
  if ((rc = fetch_stats())) return rc;
  const double normM = std::sqrt(hs.sumsq);
  double absmax;
  if (sizeof(T) == 4) {
    const unsigned int b = (unsigned int)hs.maxbits;
    float f;
    memcpy(&f, &b, 4);
    absmax = f;
  } else {
    memcpy(&absmax, &hs.maxbits, 8);
  }
  const double lam = R->lambda > 0 ? R->lambda : 1.0 / std::sqrt((double)std::max(m, n));
  // ||M||_2 from Alg. 9 at rank sv0 (not run on M = 0)
  int sv = std::min(R->sv0, kmax);
  ffsrqr_plan_t pl = nullptr;
  double norm2 = 0.0;
  if (normM > 0.0) {
    if ((rc = get_plan(R, sv, &pl))) return rc;
    if ((rc = ffsrqr_run(pl, M, ldm, seed, U, kmax, S, V, kmax, piv, ws, st, nullptr))) return rc;
    launches += ffsrqr_launch_count(pl);
    if ((e = cudaMemcpyAsync(hS.data(), S, sizeof(T), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return cuda_fail("rpca sigma_1", e);
    norm2 = (double)hS[0];
  }
  if (!(norm2 > 0.0)) {  // M = 0: X = E = 0 is the solution
    if ((e = cudaMemset2DAsync(X, ldx * sizeof(T), 0, n * sizeof(T), m, st)) != cudaSuccess ||
        (e = cudaMemset2DAsync(E, lde * sizeof(T), 0, n * sizeof(T), m, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return cuda_fail("rpca zero", e);
    if (info) *info = ffsrqr_rpca_info_t{0, 0, 0, 0, 0.0, 0, norm2, lam};
    R->launches = launches;
    return 0;
  }
  const double J = std::max(norm2, absmax);
  double mu = 1.25 / norm2;
  const double mu_bar = R->mu_bar_ratio * mu;
  init_kernel<T><<<grid, 256, 0, st>>>(M, ldm, E, lde, Y, Z, ldz, m, n, T(1.0 / J), T(1.0 / mu));
  ++launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail("rpca init", e);
  int it = 0, svp = 0, status = FFSRQR_STATUS_SWAP_CAP;
  double rel = 0.0;
  unsigned long long nnz = 0;
  for (it = 1; it <= R->max_iter; ++it) {
    if ((rc = get_plan(R, sv, &pl))) return rc;
    ffsrqr_info_t finfo{};
    if ((rc = ffsrqr_run(pl, Z, ldz, seed + (uint64_t)it, U, kmax, S, V, kmax, piv, ws, st, &finfo))) return rc;
    launches += ffsrqr_launch_count(pl);
    if ((e = cudaMemcpyAsync(hS.data(), S, (size_t)sv * sizeof(T), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return cuda_fail("rpca singular values", e);
    if (finfo.status == FFSRQR_STATUS_TIMEOUT || finfo.status == FFSRQR_STATUS_NONFINITE) return finfo.status;
    const double tau = 1.0 / mu;
    svp = 0;
    while (svp < sv && (double)hS[svp] > tau) ++svp;  // S is descending
    const int sv_next = svp < sv ? std::min(svp + 1, kmax)
                                 : std::min(svp + (int)std::lround(0.05 * (double)n), kmax);
    if (svp > 0) {
      shrink_cols_kernel<T><<<(unsigned)std::min<int64_t>((m * svp + 255) / 256, (int64_t)R->num_sms * 8), 256, 0,
                              st>>>(U, kmax, m, svp, S, T(tau));
      ++launches;
      int nl = 0;
      if ((rc = ffq_gemm_nt(pl, m, n, svp, U, kmax, V, kmax, X, ldx, ws, st, &nl))) return rc;
      launches += nl;
    } else if ((e = cudaMemset2DAsync(X, ldx * sizeof(T), 0, n * sizeof(T), m, st)) != cudaSuccess) {
      return cuda_fail("rpca X = 0", e);
    }
    const double mu_next = std::min(R->rho * mu, mu_bar);
    if ((e = cudaMemsetAsync(dst, 0, sizeof(Stats), st)) != cudaSuccess) return cuda_fail("memset", e);
    ialm_update_kernel<T><<<grid, 256, 0, st>>>(M, ldm, X, ldx, E, lde, Y, Z, ldz, m, n, T(mu), T(1.0 / mu),
                                                T(lam / mu), T(1.0 / mu_next), dst);
    ++launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail("rpca update", e);
    if ((rc = fetch_stats())) return rc;
    const double rel_prev = rel;
    rel = std::sqrt(hs.sumsq) / normM;
    nnz = hs.count;
    mu = mu_next;
    sv = sv_next;
    // converged: below tol, or stalled below 100 tol (the residual has reached
    // the rounding floor of the truncated SVD, about 1e-6 of ||M||_F in FP32 at
    // 2000 x 2000; iterating on lets noise singular values pass 1/mu)
    if (rel < R->tol || (it > 1 && rel < 100.0 * R->tol && rel > 0.9 * rel_prev)) {
      status = 0;
      break;
    }
  }
  if (it > R->max_iter) it = R->max_iter;
  if (info) *info = ffsrqr_rpca_info_t{status, it, svp, 0, rel, (int64_t)nnz, norm2, lam};
  R->launches = launches;
  return 0;
}

}  // namespace

extern "C" {

int ffsrqr_rpca_destroy(ffsrqr_rpca_t R) {
  if (!R) return -1;
  for (auto &kv : R->plans) ffsrqr_destroy(kv.second);
  delete R;
  return 0;
}

int ffsrqr_rpca_create(ffsrqr_rpca_t *out, int64_t m, int64_t n, const ffsrqr_rpca_opts_t *opts,
                       size_t *workspace_bytes) {
  if (!out) return -1;
  *out = nullptr;
  if (m < 2) return -2;
  if (n < 2) return -3;
  if (!workspace_bytes) return -5;
  ffsrqr_rpca_opts_t o{};
  if (opts) o = *opts;
  const int mode = opts ? o.mode : FFSRQR_MIXED;
  if (mode != FFSRQR_PLAIN_FP32 && mode != FFSRQR_MIXED && mode != FFSRQR_MIXED_BF16X3 && mode != FFSRQR_FP64) return -4;
  if (opts && (o.rho < 0 || o.tol < 0 || o.mu_bar_ratio < 0 || o.lambda < 0)) return -4;
  ffsrqr_rpca_s *R = new (std::nothrow) ffsrqr_rpca_s();
  if (!R) return FFSRQR_STATUS_WORKSPACE;
  R->m = m;
  R->n = n;
  R->mode = mode;
  R->elem = mode == FFSRQR_FP64 ? 8 : 4;
  R->p = (opts && o.p > 0) ? o.p : 10;
  R->sv0 = (opts && o.sv0 > 0) ? o.sv0 : 10;
  R->max_iter = (opts && o.max_iter > 0) ? o.max_iter : 100;
  R->lambda = (opts && o.lambda > 0) ? o.lambda : 0.0;
  R->rho = (opts && o.rho > 1) ? o.rho : 1.5;
  R->mu_bar_ratio = (opts && o.mu_bar_ratio > 0) ? o.mu_bar_ratio : 1e7;
  R->tol = (opts && o.tol > 0) ? o.tol : (mode == FFSRQR_FP64 ? 1e-7 : 1e-6);
  const int klimit = mode == FFSRQR_FP64 ? 160 : 224;
  int64_t km = std::min<int64_t>(std::min<int64_t>(n, m - R->p), klimit);
  if (opts && o.kmax > 0) km = std::min<int64_t>(km, o.kmax);
  if (km < 1) {
    delete R;
    return -4;
  }
  R->kmax = (int)km;
  R->fopts.g = 2.0;
  R->fopts.max_swaps = 4 * R->kmax;
  R->fopts.flags = 0;
  int dev = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&R->num_sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) {
    delete R;
    return cuda_fail("rpca device query", e);
  }
  // the largest Alg. 9 plan sizes the shared workspace
  ffsrqr_plan_t big = nullptr;
  int rc = ffsrqr_plan(&big, m, n, R->kmax, R->p, mode, &R->fopts, &R->ws_ffsrqr);
  if (rc != 0) {
    delete R;
    return rc < 0 ? -4 : rc;
  }
  R->plans[R->kmax] = big;
  R->ldz = (n + 3) / 4 * 4;
  const size_t E = R->elem;
  size_t off = align256(R->ws_ffsrqr);
  R->off_y = off;
  off = align256(off + (size_t)m * R->ldz * E);
  R->off_z = off;
  off = align256(off + (size_t)m * R->ldz * E);
  R->off_u = off;
  off = align256(off + (size_t)m * R->kmax * E);
  R->off_s = off;
  off = align256(off + (size_t)R->kmax * E);
  R->off_v = off;
  off = align256(off + (size_t)n * R->kmax * E);
  R->off_piv = off;
  off = align256(off + (size_t)n * sizeof(int32_t));
  R->off_st = off;
  off = align256(off + sizeof(Stats));
  R->total = off;
  *workspace_bytes = R->total;
  *out = R;
  return 0;
}

int ffsrqr_rpca_run(ffsrqr_rpca_t R, const void *M, int64_t ldm, void *X, int64_t ldx, void *E, int64_t lde,
                    uint64_t seed, void *workspace, void *stream, ffsrqr_rpca_info_t *info) {
  if (!R) return -1;
  if (!M) return -2;
  if (ldm < R->n) return -3;
  if (!X) return -4;
  if (ldx < R->n) return -5;
  if (!E) return -6;
  if (lde < R->n) return -7;
  if (!workspace || ((uintptr_t)workspace & 255u)) return -9;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  unsigned char *ws = static_cast<unsigned char *>(workspace);
  if (R->elem == 8)
    return rpca_impl<double>(R, (const double *)M, ldm, (double *)X, ldx, (double *)E, lde, seed, ws, st, info);
  return rpca_impl<float>(R, (const float *)M, ldm, (float *)X, ldx, (float *)E, lde, seed, ws, st, info);
}

int ffsrqr_rpca_launch_count(ffsrqr_rpca_t R) {
  if (!R) return -1;
  return R->launches;
}

}  // extern "C"
