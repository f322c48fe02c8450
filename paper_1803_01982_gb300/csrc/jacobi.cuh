// jacobi.cuh -- SVD of the small k x k factor M of tmp (Alg. 9) by
// one-sided (Hestenes) Jacobi, preconditioned by a QR factorisation, on a
// thread-block cluster.
//
//   M^T = Q R (Householder, no pivoting), X = R^T, X J = W diag(sigma):
//   pairs of columns of X (rows of R) are rotated until every pair is
//   orthogonal to within tol * ||x_p|| ||x_q||; J, started at I, accumulates
//   the rotations.  Then M^T = (Q J) diag(sigma) W^T, i.e. U = W normalised
//   and V = Q J.  The rows of R are graded like the singular values, which
//   makes the sweeps converge in about a third fewer sweeps than on M^T
//   itself (the QR preconditioning of one-sided Jacobi of Drmac and Veselic,
//   without the column pivoting, which gains nothing here).
//
// The QR runs in two single-block kernels: R and the reflectors first; Q is
// then formed alongside the sweeps (the caller runs it on a second stream)
// and V = Q J is one small product afterwards.
// The sweeps run on a cluster of C blocks (C = 2, 4 or 8).  The rows of the
// stacked matrix [X; J] (2 kp rows, kk columns) are split into C slabs, one
// per block, each held column-major in shared memory.  One round of the
// parallel round-robin ordering (kk/2 disjoint pairs, every pair meets once
// per sweep of kk - 1 rounds) is, in every block at once:
//   1. the LPP lanes of pair i (2 or 4; few lanes per pair keep the warps,
//      and the per-warp work of a round, few) load their slices of columns p
//      and q of the slab into registers and form the partial sums of
//      ||x_p||^2, ||x_q||^2 and x_p . x_q over the X rows of the slab;
//   2. the blocks holding X rows push their partials with st.async into a
//      slot [round parity][source block][pair] of every block's shared
//      memory, completing on that block's mbarrier of the round parity; the
//      other blocks push one 16-byte token to each X block.  A block sends its
//      round-r message only after it has read its round r-1 slots, and sends
//      round r+1 only after receiving every block's round-r message, so no slot
//      is overwritten before it is read;
//   3. every block waits (bounded) for its mbarrier phase: nxc * npair
//      partials, plus the tokens at the X blocks;
//   4. every block adds the received partials in block order, so all blocks
//      take bitwise the same rotation (cos, sin) and the same convergence
//      decisions; it rotates its registers and stores them back;
//   5. one block barrier (the next round pairs the columns differently).
// The slab of a block is 1/C of the matrix, so the shared-memory traffic of a
// round (one read and one write of the slab) shrinks with C; the exchange
// costs one one-way DSMEM latency per round, with no cluster barrier.
// After a sweep without rotations, sigma_c = ||x_c|| (one more exchange of
// partial norms), the columns are ranked by descending sigma and each block
// writes its rows of U (from X) and V (from J).  Every block runs the same
// sequence of cluster barriers (one per sweep, for block 0's broadcast end
// decision, and the final ones): the rounds of a sweep are fixed in number.
// An mbarrier wait that gives up (about a second) marks the block failed: it
// skips its later waits, block 0 then ends the sweeps, and the run reports
// STATUS_TIMEOUT.
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"

namespace ffq {

namespace cg = cooperative_groups;

constexpr int JAC_MAX_SWEEPS = 40;
constexpr int JAC_NVL = 8;      // 16-byte vectors per lane per column of a slab

// Round-robin pairing (circle method): kk players, player kk-1 fixed.
__device__ __forceinline__ void rr_pair(int t, int i, int kk, int &p, int &q) {
  const int n1 = kk - 1;  // 0 <= t < n1, 0 <= i < kk / 2
  if (i == 0) {
    p = t;
    q = n1;
  } else {
    p = t + i;
    if (p >= n1) p -= n1;
    q = t - i;
    if (q < 0) q += n1;
  }
  if (p > q) {
    const int x = p;
    p = q;
    q = x;
  }
}

// 16-byte vector of T (4 floats or 2 doubles) in shared memory.
template <typename T>
struct Vec16 {
  static constexpr int N = 16 / sizeof(T);
  T v[N];
};
template <typename T>
__device__ __forceinline__ Vec16<T> ld16(const T *p) {
  Vec16<T> r;
  if (sizeof(T) == 4) {
    const float4 x = *reinterpret_cast<const float4 *>(p);
    r.v[0] = x.x;
    r.v[1] = x.y;
    r.v[2] = x.z;
    r.v[3] = x.w;
  } else {
    const double2 x = *reinterpret_cast<const double2 *>(p);
    r.v[0] = x.x;
    r.v[1] = x.y;
  }
  return r;
}
template <typename T>
__device__ __forceinline__ void st16(T *p, const Vec16<T> &r) {
  if (sizeof(T) == 4) *reinterpret_cast<float4 *>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
  else *reinterpret_cast<double2 *>(p) = make_double2(r.v[0], r.v[1]);
}

// ---------------------------------------------------------------------------
// The preconditioning QR, M^T = Q R = H_0 H_1 ... H_{k-1} R.
//
// The matrix is held column by column, each column padded with zeros to kp
// rows (16-byte aligned).  Every reflector is applied from a full-length copy
// of v (zeros above row j, 1 at row j, zeros in the padding), so the updates
// run on 16-byte vectors from the vector holding row j on, without
// per-element tests: rows above j see v = 0 and stay as they are.
// ---------------------------------------------------------------------------
// dst_u := (I - tau v v^T) src_u for NC columns src_u = src + u ld (dst
// likewise) on the vectors q0 .. nq - 1; one warp.
template <typename T, int NC>
__device__ __forceinline__ void hh_apply_group(const T *v, T tau, int q0, int nq, const T *src, T *dst, int ld) {
  constexpr int VN = Vec16<T>::N;
  const int lane = threadIdx.x & 31;
  T w[NC];
  if constexpr (sizeof(T) == 4) {  // packed pairs (f32x2)
    float2 w2[NC];
#pragma unroll
    for (int u = 0; u < NC; ++u) w2[u] = make_float2(0.f, 0.f);
    for (int q = q0 + lane; q < nq; q += 32) {
      const float4 vv = *reinterpret_cast<const float4 *>(v + q * VN);
      const float2 vl = make_float2(vv.x, vv.y), vh = make_float2(vv.z, vv.w);
#pragma unroll
      for (int u = 0; u < NC; ++u) {
        const float4 xx = *reinterpret_cast<const float4 *>(src + u * ld + q * VN);
        w2[u] = __ffma2_rn(vh, make_float2(xx.z, xx.w), __ffma2_rn(vl, make_float2(xx.x, xx.y), w2[u]));
      }
    }
#pragma unroll
    for (int u = 0; u < NC; ++u) w[u] = w2[u].x + w2[u].y;
  } else {
#pragma unroll
    for (int u = 0; u < NC; ++u) w[u] = T(0);
    for (int q = q0 + lane; q < nq; q += 32) {
      const Vec16<T> vv = ld16(v + q * VN);
#pragma unroll
      for (int u = 0; u < NC; ++u) {
        const Vec16<T> xx = ld16(src + u * ld + q * VN);
#pragma unroll
        for (int e = 0; e < VN; ++e) w[u] = fma(vv.v[e], xx.v[e], w[u]);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int u = 0; u < NC; ++u) w[u] += __shfl_xor_sync(0xffffffffu, w[u], o);
  }
  if constexpr (sizeof(T) == 4) {
    float2 m2[NC];
#pragma unroll
    for (int u = 0; u < NC; ++u) m2[u] = make_float2(-tau * w[u], -tau * w[u]);
    for (int q = q0 + lane; q < nq; q += 32) {
      const float4 vv = *reinterpret_cast<const float4 *>(v + q * VN);
      const float2 vl = make_float2(vv.x, vv.y), vh = make_float2(vv.z, vv.w);
#pragma unroll
      for (int u = 0; u < NC; ++u) {
        const float4 xx = *reinterpret_cast<const float4 *>(src + u * ld + q * VN);
        const float2 rl = __ffma2_rn(m2[u], vl, make_float2(xx.x, xx.y));
        const float2 rh = __ffma2_rn(m2[u], vh, make_float2(xx.z, xx.w));
        *reinterpret_cast<float4 *>(dst + u * ld + q * VN) = make_float4(rl.x, rl.y, rh.x, rh.y);
      }
    }
  } else {
    for (int q = q0 + lane; q < nq; q += 32) {
      const Vec16<T> vv = ld16(v + q * VN);
#pragma unroll
      for (int u = 0; u < NC; ++u) {
        const Vec16<T> xx = ld16(src + u * ld + q * VN);
        Vec16<T> r;
#pragma unroll
        for (int e = 0; e < VN; ++e) r.v[e] = fma(-tau * w[u], vv.v[e], xx.v[e]);
        st16(dst + u * ld + q * VN, r);
      }
    }
  }
}

// In-place H applied to columns c0 .. c1 - 1 of A, split into contiguous
// runs among the warps first_warp ..; each run goes in groups of 4, 2, 1.
template <typename T>
__device__ __forceinline__ void hh_apply_cols(const T *v, T tau, int q0, int nq, T *A, int ld, int c0, int c1,
                                              int first_warp) {
  const int g = (int)(threadIdx.x >> 5) - first_warp, nw = (int)(blockDim.x >> 5) - first_warp;
  if (g < 0 || c1 <= c0) return;
  const int per = (c1 - c0 + nw - 1) / nw;
  int c = c0 + g * per;
  const int ce = min(c1, c + per);
  for (; c + 4 <= ce; c += 4) hh_apply_group<T, 4>(v, tau, q0, nq, A + (size_t)c * ld, A + (size_t)c * ld, ld);
  if (c + 2 <= ce) {
    hh_apply_group<T, 2>(v, tau, q0, nq, A + (size_t)c * ld, A + (size_t)c * ld, ld);
    c += 2;
  }
  if (c < ce) hh_apply_group<T, 1>(v, tau, q0, nq, A + (size_t)c * ld, A + (size_t)c * ld, ld);
}

// Reflector of column x (rows j .. k - 1): x(j) := beta, x(j+1:k) := v,
// vb and vg (global) := the full-length v (padded length kp); returns tau.
// One warp.
template <typename T>
__device__ __forceinline__ T hh_make(T *x, T *vb, T *__restrict__ vg, int j, int k, int kp) {
  const int lane = threadIdx.x & 31;
  T ss = T(0);
  for (int t = j + 1 + lane; t < k; t += 32) ss = fma(x[t], x[t], ss);
  ss = warp_sum(ss);
  const T alpha = x[j];
  T tau = T(0), beta = alpha, scal = T(0);
  if (ss > T(0)) {
    const T nx = sqrt(fma(alpha, alpha, ss));
    beta = (alpha >= T(0)) ? -nx : nx;
    tau = (beta - alpha) / beta;
    scal = T(1) / (alpha - beta);
  }
  for (int t = lane; t < kp; t += 32) {
    T y = T(0);
    if (t > j && t < k) {
      y = x[t] * scal;
      x[t] = y;
    }
    y = (t == j) ? T(1) : y;
    vb[t] = y;
    vg[t] = y;
  }
  __syncwarp();
  if (lane == 0) x[j] = beta;
  return tau;
}


// Rank 0: R of the columns of A (= M^T), one barrier per step.  During step j
// warp 0 applies H_j to column j + 1 and at once builds the next reflector
// from it (look-ahead) while the other warps apply H_j to columns j + 2 ..
// k - 1.  The reflectors go to qv[j * kp ..] and tau to qv[k * kp + j]; A is
// left holding X = R^T (column i of X = row i of R, zeros above the diagonal).
template <typename T>
__device__ void precond_qr_r(T *A, int k, int kp, T *vb0, T *vb1, T *tau, T *__restrict__ qv) {
  constexpr int VN = Vec16<T>::N;
  const int nq = kp / VN, ld = kp;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (wid == 0) {
    const T t0 = hh_make(A, vb0, qv, 0, k, kp);
    if (lane == 0) tau[0] = t0;
  }
  __syncthreads();
  for (int j = 0; j + 1 < k; ++j) {
    const T *v = (j & 1) ? vb1 : vb0;
    const T tj = tau[j];
    const int q0 = j / VN;
    if (wid == 0) {
      T *x = A + (size_t)(j + 1) * ld;
      if (tj != T(0)) hh_apply_group<T, 1>(v, tj, q0, nq, x, x, ld);
      __syncwarp();
      const T tn = hh_make(x, (j & 1) ? vb0 : vb1, qv + (size_t)(j + 1) * kp, j + 1, k, kp);
      if (lane == 0) tau[j + 1] = tn;
    } else if (tj != T(0)) {
      hh_apply_cols(v, tj, q0, nq, A, ld, j + 2, k, 1);
    }
    __syncthreads();
  }
  for (int j = threadIdx.x; j < k; j += blockDim.x) qv[(size_t)k * kp + j] = tau[j];
  // X = R^T in place: row i of R (A(i, c), c > i) moves to column i
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int i = e / k, c = e - i * k;
    if (i < c) {
      A[(size_t)i * ld + c] = A[(size_t)c * ld + i];
      A[(size_t)c * ld + i] = T(0);
    }
  }
  __syncthreads();
}

// Rank 1: Q = H_0 (H_1 (... H_{k-1} I)) into the columns of A from the
// reflectors in qv (global), one barrier per step.  During step j warp 0 forms
// column j of the result, H_j e_j, in a side buffer and fetches v_{j-1} for
// the next step; warp 1 forms column j + 1 from the side buffer of the
// previous step; the other warps apply H_j to columns j + 2 .. k - 1.
template <typename T>
__device__ void precond_qr_q(T *A, int k, int kp, T *vb0, T *vb1, T *hb0, T *hb1, T *tau,
                             const T *__restrict__ qv) {
  constexpr int VN = Vec16<T>::N;
  const int nq = kp / VN, ld = kp;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int j = threadIdx.x; j < k; j += blockDim.x) tau[j] = __ldcg(qv + (size_t)k * kp + j);
  if (wid == 0) {
    T *vn = ((k - 1) & 1) ? vb1 : vb0;
    for (int t = lane; t < kp; t += 32) vn[t] = __ldcg(qv + (size_t)(k - 1) * kp + t);
  }
  __syncthreads();
  for (int j = k - 1; j >= 0; --j) {
    const T *v = (j & 1) ? vb1 : vb0;
    const T tj = tau[j];
    const int q0 = j / VN;
    if (wid == 0) {
      T *hj = (j & 1) ? hb1 : hb0;
      for (int t = lane; t < kp; t += 32) hj[t] = ((t == j) ? T(1) : T(0)) - tj * v[t];
      if (j > 0) {
        T *vn = ((j - 1) & 1) ? vb1 : vb0;
        for (int t = lane; t < kp; t += 32) vn[t] = __ldcg(qv + (size_t)(j - 1) * kp + t);
      }
    } else if (wid == 1) {
      if (j + 1 < k)  // column j + 1 = H_j (H_{j+1} ... e_{j+1}), all rows
        hh_apply_group<T, 1>(v, tj, 0, nq, (j & 1) ? hb0 : hb1, A + (size_t)(j + 1) * ld, ld);
    } else if (tj != T(0)) {
      hh_apply_cols(v, tj, q0, nq, A, ld, j + 2, k, 2);
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < kp; t += blockDim.x) A[t] = hb0[t];  // column 0 = H_0 e_0
  __syncthreads();
}


// R of M^T and the reflectors: X = R^T to Xg (column-major, X(r, c) at
// Xg[c * k + r]), reflectors and tau to qv (k * kp + k).  One block.
template <typename T>
__global__ void __launch_bounds__(1024) precond_qr_r_kernel(const T *__restrict__ M, int k, T *__restrict__ Xg,
                                                             T *__restrict__ qv) {
  constexpr int VN = Vec16<T>::N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int kp = (k + VN - 1) / VN * VN;
  T *A = reinterpret_cast<T *>(smem_raw);  // k columns of kp
  T *vb0 = A + (size_t)k * kp, *vb1 = vb0 + kp, *tau = vb1 + kp;
  for (int e = threadIdx.x; e < k * kp; e += blockDim.x) {
    const int c = e / kp, r = e - c * kp;
    A[e] = (r < k) ? M[(size_t)c * k + r] : T(0);  // column c of M^T = row c of M
  }
  __syncthreads();
  precond_qr_r(A, k, kp, vb0, vb1, tau, qv);
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int c = e / k, r = e - c * k;
    Xg[e] = A[(size_t)c * kp + r];
  }
}

// Q (column-major, Q(t, c) at Qg[c * k + t]) from the reflectors in qv.
// One block.
template <typename T>
__global__ void __launch_bounds__(1024) precond_qr_q_kernel(int k, const T *__restrict__ qv, T *__restrict__ Qg) {
  constexpr int VN = Vec16<T>::N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int kp = (k + VN - 1) / VN * VN;
  T *A = reinterpret_cast<T *>(smem_raw);
  T *vb0 = A + (size_t)k * kp, *vb1 = vb0 + kp, *hb0 = vb1 + kp, *hb1 = hb0 + kp, *tau = hb1 + kp;
  precond_qr_q(A, k, kp, vb0, vb1, hb0, hb1, tau, qv);
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int c = e / k, t = e - c * k;
    Qg[e] = A[(size_t)c * kp + t];
  }
}

// Shared-memory bytes of the two QR kernels.
inline size_t precond_qr_smem(int k, size_t elem) {
  const size_t kp = (size_t)round_up(k, 16 / (int64_t)elem);
  return ((size_t)k * kp + 5 * kp) * elem;
}

// Rotation (cs, sn) that makes columns p, q orthogonal (Rutishauser's
// formulas): zeta = (be - al) / (2 ga), t = sign(zeta) / (|zeta| +
// sqrt(1 + zeta^2)), cs = 1 / sqrt(1 + t^2), sn = cs t.  No rotation (sn = 0)
// when |ga| <= tol sqrt(al be).  In single precision t only steers the
// convergence, so it is formed with the approximate reciprocal and
// reciprocal square root; cs is refined by one Newton step for 1/sqrt(x),
// y <- y (3 - x y^2) / 2, so that cs^2 + sn^2 = 1 to rounding and the
// rotation stays orthogonal.
template <typename T>
__device__ __forceinline__ void jac_rotation(T al, T be, T ga, T tol, T &cs, T &sn) {
  cs = T(1);
  sn = T(0);
  if (!(ga != T(0) && fabs(ga) > tol * sqrt(al * be))) return;
  if constexpr (sizeof(T) == 4) {
    const float zeta = __fdividef(be - al, 2.f * ga);
    const float a = fabsf(zeta);
    float root = a;  // sqrt(1 + a^2), = a to rounding for a >= 2^30
    if (a < 1073741824.f) {
      const float x = fmaf(a, a, 1.f);
      root = x * rsqrtf(x);
    }
    const float t = copysignf(__fdividef(1.f, a + root), zeta);
    const float x = fmaf(t, t, 1.f);
    float y = rsqrtf(x);
    y = y * fmaf(-0.5f * x, y * y, 1.5f);
    cs = y;
    sn = y * t;
  } else {
    const T zeta = (be - al) / (T(2) * ga);
    const T tt = copysign(T(1), zeta) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
    cs = T(1) / sqrt(T(1) + tt * tt);
    sn = cs * tt;
  }
}

// ---------------------------------------------------------------------------
// Cluster Jacobi.
// ---------------------------------------------------------------------------
template <typename T>
struct JacPart {
  T al, be, ga, pad;
};

// Geometry of the slabs (host and device).
struct JacGeom {
  int kk, kp, npair, hb, nvx_ctas;
};
__host__ __device__ inline JacGeom jac_geom(int k, int C, int VN) {
  JacGeom g;
  g.kk = k + (k & 1);
  g.npair = g.kk / 2;
  g.kp = (k + VN - 1) / VN * VN;
  const int nr = 2 * g.kp;                                  // rows of [X; J]
  g.hb = ((nr + C - 1) / C + VN - 1) / VN * VN;             // slab height, whole vectors
  g.nvx_ctas = (g.kp + g.hb - 1) / g.hb;                    // blocks holding rows of X
  return g;
}
// Column stride of a slab in shared memory (elements): the slab height padded
// to a number of 16-byte vectors congruent to LPP mod 8, so that the LPP
// consecutive vectors of the 32 / (4 LPP) columns a quarter-warp reads or
// writes at once fall in distinct bank groups.
__host__ __device__ inline int jac_ldcol(int hb, int VN, int lpp) {
  int nv = hb / VN;
  const int want = lpp & 7;
  while ((nv & 7) != want) ++nv;
  return nv * VN;
}
inline size_t jac_cluster_smem(int k, int C, size_t elem, int lpp) {
  const JacGeom g = jac_geom(k, C, 16 / (int)elem);
  const size_t slab = ((size_t)g.kk * jac_ldcol(g.hb, 16 / (int)elem, lpp) * elem + 15) & ~(size_t)15;
  return slab + 2 * (size_t)C * g.npair * 4 * elem + (size_t)g.kk * elem + (size_t)g.kk * sizeof(int) + 64;
}

// Shared-memory address helpers for the asynchronous exchange.
__device__ __forceinline__ unsigned jac_saddr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned jac_mapa(unsigned a, int r) {
  unsigned d;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(r));
  return d;
}
// 16 bytes to another block's shared memory, completing on its mbarrier.
__device__ __forceinline__ void jac_st_async(unsigned raddr, unsigned rmbar, float a, float b, float c, float d) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                   raddr),
               "f"(a), "f"(b), "f"(c), "f"(d), "r"(rmbar)
               : "memory");
}
__device__ __forceinline__ void jac_st_async(unsigned raddr, unsigned rmbar, double a, double b) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];" ::"r"(raddr),
               "d"(a), "d"(b), "r"(rmbar)
               : "memory");
}
__device__ __forceinline__ bool jac_try_wait(unsigned mbar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}
constexpr long long JAC_WAIT_SPINS = 1ll << 22;  // bounded mbarrier wait (about a second)

// Xin: X (column-major, X(r, c) at Xin[c * k + r]); Jin: J_0 (same layout) or
// NULL for the identity.  Uout, Vout: k x k row-major, columns in descending
// order of Sout.  LPP lanes share a pair (blockDim = kk/2 * LPP rounded up to
// whole warps, at most 512), each holding up to JAC_NVL 16-byte vectors of
// each of the two columns of the slab.
template <typename T, int LPP>
__global__ void __launch_bounds__(512) jacobi_cluster_kernel(const T *__restrict__ Xin, const T *__restrict__ Jin,
                                                              int k, T *__restrict__ Uout, T *__restrict__ Sout,
                                                              T *__restrict__ Vout, int *ctl, int max_sweeps, T tol) {
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  constexpr int VN = Vec16<T>::N;
  const JacGeom g = jac_geom(k, C, VN);
  const int kk = g.kk, kp = g.kp, npair = g.npair, hb = g.hb, nxc = g.nvx_ctas;
  const int ldc = jac_ldcol(hb, VN, LPP);                  // column stride of the slab (elements)
  const int r0 = rank * hb;                               // first stacked row of this slab
  const int nvec = max(0, min(hb, 2 * kp - r0)) / VN;     // vectors per column in the slab
  const int nvx = max(0, min(nvec, (kp - r0) / VN));      // of which rows of X
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *S = reinterpret_cast<T *>(smem_raw);                           // column c at S[c * ldc]
  JacPart<T> *inbox = reinterpret_cast<JacPart<T> *>(
      smem_raw + (((size_t)kk * ldc * sizeof(T) + 15) & ~(size_t)15));  // [2][C][npair]: partials received
  T *sig = reinterpret_cast<T *>(inbox + 2 * (size_t)C * npair);    // [kk]
  int *rnk = reinterpret_cast<int *>(sig + kk);                     // [kk]
  __shared__ __align__(8) unsigned long long s_mbar[2];             // one per round parity
  __shared__ int s_rot, s_done, s_fail;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int gl = lane % LPP;  // lane within the pair's group
  if (max_sweeps > JAC_MAX_SWEEPS) max_sweeps = JAC_MAX_SWEEPS;

  // the slab: stacked rows r0 .. r0 + hb - 1 of [X; J] (X padded to kp rows)
  for (int e = threadIdx.x; e < kk * hb; e += blockDim.x) {
    const int c = e / hb, lr = e - c * hb, gr = r0 + lr;
    T v = T(0);
    if (c < k) {
      if (gr < kp) {
        if (gr < k) v = Xin[(size_t)c * k + gr];
      } else if (gr - kp < k) {
        const int jr = gr - kp;
        v = Jin ? Jin[(size_t)c * k + jr] : ((jr == c) ? T(1) : T(0));
      }
    }
    S[(size_t)c * ldc + lr] = v;
  }
  if (threadIdx.x == 0) {
    s_rot = 0;
    s_fail = 0;
    for (int b = 0; b < 2; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(jac_saddr(&s_mbar[b])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (rank == 0 && threadIdx.x < 16) ctl[CTL_SWEEP_ROT0 + threadIdx.x] = 0;
  __syncthreads();
  cluster.sync();  // every block's barriers exist before any block sends to them
  // bytes a block receives per round: the partials of every X block, and at
  // the X blocks one 16-byte token from every other block ("your slot of the
  // round before last is free again")
  const unsigned expect = (unsigned)(nxc * npair * sizeof(JacPart<T>) + (rank < nxc ? (C - nxc) * 16 : 0));

  const int i = threadIdx.x / LPP;
  int round = 0, sweeps = 0;
  bool done = false;
  for (; sweeps < max_sweeps && !done; ++sweeps) {
    int nrot = 0;  // rotations of this sweep counted by this thread (one lane per pair)
    for (int t = 0; t < kk - 1; ++t, ++round) {
      int p = -1, q = -1;
      if (i < npair) rr_pair(t, i, kk, p, q);
      Vec16<T> xr[JAC_NVL], yr[JAC_NVL];
      T al = T(0), be = T(0), ga = T(0);
      float2 a2 = make_float2(0.f, 0.f), b2 = a2, g2 = a2;  // packed partial sums (single precision)
      if (p >= 0) {
        const T *sp = S + (size_t)p * ldc, *sq = S + (size_t)q * ldc;
#pragma unroll
        for (int l = 0; l < JAC_NVL; ++l) {
          if (LPP * l >= nvec) break;  // uniform: no issue slots for the unused tail
          const int v = gl + LPP * l;
          if (v < nvec) {
            xr[l] = ld16(sp + v * VN);
            yr[l] = ld16(sq + v * VN);
            if (v < nvx) {
              if constexpr (sizeof(T) == 4) {  // packed pairs (f32x2)
                const float2 xl = make_float2(xr[l].v[0], xr[l].v[1]), xh = make_float2(xr[l].v[2], xr[l].v[3]);
                const float2 yl = make_float2(yr[l].v[0], yr[l].v[1]), yh = make_float2(yr[l].v[2], yr[l].v[3]);
                a2 = __ffma2_rn(xh, xh, __ffma2_rn(xl, xl, a2));
                b2 = __ffma2_rn(yh, yh, __ffma2_rn(yl, yl, b2));
                g2 = __ffma2_rn(xh, yh, __ffma2_rn(xl, yl, g2));
              } else {
#pragma unroll
                for (int u = 0; u < VN; ++u) {
                  al = fma(xr[l].v[u], xr[l].v[u], al);
                  be = fma(yr[l].v[u], yr[l].v[u], be);
                  ga = fma(xr[l].v[u], yr[l].v[u], ga);
                }
              }
            }
          }
        }
      }
      if constexpr (sizeof(T) == 4) {
        al = a2.x + a2.y;
        be = b2.x + b2.y;
        ga = g2.x + g2.y;
      }
#pragma unroll
      for (int o = LPP / 2; o > 0; o >>= 1) {
        al += __shfl_xor_sync(0xffffffffu, al, o);
        be += __shfl_xor_sync(0xffffffffu, be, o);
        ga += __shfl_xor_sync(0xffffffffu, ga, o);
      }
      const int par = round & 1;
      JacPart<T> *in = inbox + (size_t)par * C * npair;  // [C][npair]
      const unsigned mbar = jac_saddr(&s_mbar[par]);
      if (rank < nxc) {
        // this block's partials to every block (the group's lanes share the destinations)
        if (p >= 0)
          for (int d = gl; d < C; d += LPP) {
            const unsigned ra = jac_mapa(jac_saddr(in + (size_t)rank * npair + i), d), rm = jac_mapa(mbar, d);
            if constexpr (sizeof(T) == 4) {
              jac_st_async(ra, rm, (float)al, (float)be, (float)ga, 0.f);
            } else {
              jac_st_async(ra, rm, (double)al, (double)be);
              jac_st_async(ra + 16, rm, (double)ga, 0.0);
            }
          }
      } else if (threadIdx.x < nxc) {
        const int d = threadIdx.x;
        jac_st_async(jac_mapa(jac_saddr(in + (size_t)rank * npair), d), jac_mapa(mbar, d), 0.f, 0.f, 0.f, 0.f);
      }
      if (threadIdx.x == 0)
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(expect) : "memory");
      if (!s_fail) {
        const unsigned phase = (unsigned)((round >> 1) & 1);
        long long spins = 0;
        while (!jac_try_wait(mbar, phase))
          if (++spins > JAC_WAIT_SPINS) {
            s_fail = 1;  // sticky: later rounds skip the wait; the sweeps end at block 0's next decision
            break;
          }
      }
      if (p >= 0) {
        // the partials of the blocks holding X rows, added in block order:
        // the same sums, hence the same rotations, in every block
        al = be = ga = T(0);
        for (int r = 0; r < nxc; ++r) {
          const JacPart<T> pr = in[(size_t)r * npair + i];
          al += pr.al;
          be += pr.be;
          ga += pr.ga;
        }
        T cs, sn;
        jac_rotation(al, be, ga, tol, cs, sn);
        if (sn != T(0)) {
          T *sp = S + (size_t)p * ldc, *sq = S + (size_t)q * ldc;
#pragma unroll
          for (int l = 0; l < JAC_NVL; ++l) {
            if (LPP * l >= nvec) break;
            const int v = gl + LPP * l;
            if (v < nvec) {
              Vec16<T> xo, yo;
              if constexpr (sizeof(T) == 4) {  // packed pairs (f32x2)
                const float2 c2 = make_float2(cs, cs), s2 = make_float2(sn, sn), n2 = make_float2(-sn, -sn);
                const float2 xl = make_float2(xr[l].v[0], xr[l].v[1]), xh = make_float2(xr[l].v[2], xr[l].v[3]);
                const float2 yl = make_float2(yr[l].v[0], yr[l].v[1]), yh = make_float2(yr[l].v[2], yr[l].v[3]);
                const float2 ol = __ffma2_rn(c2, xl, __fmul2_rn(n2, yl)), oh = __ffma2_rn(c2, xh, __fmul2_rn(n2, yh));
                const float2 pl = __ffma2_rn(s2, xl, __fmul2_rn(c2, yl)), ph = __ffma2_rn(s2, xh, __fmul2_rn(c2, yh));
                xo.v[0] = ol.x;
                xo.v[1] = ol.y;
                xo.v[2] = oh.x;
                xo.v[3] = oh.y;
                yo.v[0] = pl.x;
                yo.v[1] = pl.y;
                yo.v[2] = ph.x;
                yo.v[3] = ph.y;
              } else {
#pragma unroll
                for (int u = 0; u < VN; ++u) {
                  xo.v[u] = cs * xr[l].v[u] - sn * yr[l].v[u];
                  yo.v[u] = sn * xr[l].v[u] + cs * yr[l].v[u];
                }
              }
              st16(sp + v * VN, xo);
              st16(sq + v * VN, yo);
            }
          }
          nrot += (gl == 0);
        }
      }
      __syncthreads();
    }
    // block 0's decision, broadcast: every block leaves after the same sweep
    nrot = warp_sum(nrot);
    if (lane == 0 && nrot) atomicAdd(&s_rot, nrot);
    __syncthreads();
    if (rank == 0 && threadIdx.x < C)
      *cluster.map_shared_rank(&s_done, (unsigned)threadIdx.x) = (s_rot == 0 || s_fail) ? 1 : 0;
    if (rank == 0 && threadIdx.x == 0 && sweeps < 16) ctl[CTL_SWEEP_ROT0 + sweeps] = s_rot;
    cluster.sync();
    done = (s_done != 0);
    if (threadIdx.x == 0) s_rot = 0;
  }
  if (rank == 0 && threadIdx.x == 0) ctl[CTL_JACOBI_SWEEPS] = sweeps;
  if (threadIdx.x == 0 && s_fail) set_status(ctl, STATUS_TIMEOUT);
  // sigma: partial column norms over the X rows, pulled through DSMEM after a
  // cluster barrier (the inbox of the parity the last round did not use is free)
  {
    const int par = round & 1;
    T *pn = reinterpret_cast<T *>(inbox + (size_t)par * C * npair);  // [kk]: this block's partial norms
    if (rank < nxc) {
      for (int c = wid; c < kk; c += nwarp) {
        T acc = T(0);
        for (int v = lane; v < nvx; v += 32) {
          const Vec16<T> x = ld16(S + (size_t)c * ldc + v * VN);
#pragma unroll
          for (int u = 0; u < VN; ++u) acc = fma(x.v[u], x.v[u], acc);
        }
        acc = warp_sum(acc);
        if (lane == 0) pn[c] = acc;
      }
    }
    cluster.sync();
    for (int c = threadIdx.x; c < kk; c += blockDim.x) {
      T s2 = T(0);
      for (int r = 0; r < nxc; ++r) s2 += cluster.map_shared_rank(pn, (unsigned)r)[c];
      sig[c] = sqrt(s2);
    }
    cluster.sync();  // no block leaves while another may still read its partial norms
  }
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    const T sc = sig[c];
    int rk = 0;
    for (int d = 0; d < k; ++d) {
      const T sd = sig[d];
      rk += (sd > sc) || (sd == sc && d < c);
    }
    rnk[c] = rk;
    if (rank == 0) Sout[rk] = sc;
  }
  __syncthreads();
  // outputs: U from the rows of X (normalised columns of W), V from the rows of J
  for (int e = threadIdx.x; e < k * hb; e += blockDim.x) {
    const int c = e / hb, lr = e - c * hb, gr = r0 + lr;
    const int rk = rnk[c];
    if (gr < k) {
      const T sc = sig[c];
      Uout[(size_t)gr * k + rk] = (sc > T(0)) ? S[(size_t)c * ldc + lr] / sc : ((gr == rk) ? T(1) : T(0));
    } else if (gr >= kp && gr - kp < k) {
      Vout[(size_t)(gr - kp) * k + rk] = S[(size_t)c * ldc + lr];
    }
  }
}

}  // namespace ffq
