// jacobi.cuh -- SVD of the small k x k factor M of tmp (Alg. 9, lines 4-5) by
// one-sided (Hestenes) Jacobi, preconditioned by a QR factorisation, on a
// 2-CTA thread-block cluster.
//
//   M^T = Q R (Householder, no pivoting), X = R^T, X J = W diag(sigma):
//   pairs of columns of X (rows of R) are rotated until every pair is
//   orthogonal to within tol * ||x_p|| ||x_q||; J accumulates the rotations.
//   Then R = J diag(sigma) W^T and M = W diag(sigma) (Q J)^T, i.e. U = W
//   normalised and V = Q J.  The rows of R are graded like the singular
//   values, which makes the sweeps converge in about a third fewer sweeps
//   than on M^T itself (the QR preconditioning of one-sided Jacobi of Drmac
//   and Veselic, without the column pivoting, which gains nothing here).
//
// Rank 0 holds M^T (column-major, padded stride) in shared memory, factors it
// in place, writes the Householder vectors to global memory and publishes
// them, transposes R into X and runs the parallel round-robin ordering: kk/2
// disjoint pairs per round, every pair meets once per sweep of kk-1 rounds.
// Each pair is handled by 8 lanes (four pairs per warp) with 16-byte
// shared-memory accesses.  The (cos, sin) of every round go to a rotation log
// in global memory; every JAC_GROUP rounds one gpu-scope release publishes the
// progress counter.  Rank 1 forms Q from the published reflectors while rank
// 0 sweeps, then applies the logged rounds to it as they are published
// (acquire loads of the counter), so the two CTAs never wait on each other per
// round.  After convergence (a sweep without rotations) sigma_j = ||x_j||, the
// ranks of the sorted order go to rank 1 through DSMEM, and both write their
// outputs.  All waits are bounded.
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"

namespace ffq {

namespace cg = cooperative_groups;

constexpr int JAC_PPW = 4;      // pairs per warp, 8 lanes each (kk/2 <= 32 * JAC_PPW)
constexpr int JAC_GROUP = 16;   // rounds per published progress step
constexpr int JAC_MAX_SWEEPS = 40;

// Round-robin pairing (circle method): kk players, player kk-1 fixed.
__device__ __forceinline__ void rr_pair(int t, int i, int kk, int &p, int &q) {
  const int n1 = kk - 1;
  if (i == 0) {
    p = t % n1;
    q = n1;
  } else {
    p = (t + i) % n1;
    q = (t - i + n1) % n1;
  }
  if (p > q) {
    const int x = p;
    p = q;
    q = x;
  }
}

__device__ __forceinline__ unsigned long long jac_now() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int jac_ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void jac_st_release(int *p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
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

// Rotate columns p, q of a column-major shared matrix (stride kp) by (cs, sn);
// the 8 lanes g8 = 0..7 of a group cover the nv 16-byte vectors of a column.
template <typename T>
__device__ __forceinline__ void rotate_cols(T *Mat, int kp, int nv, int p, int q, T cs, T sn, int g8) {
  constexpr int VN = Vec16<T>::N;
  T *mp = Mat + (size_t)p * kp, *mq = Mat + (size_t)q * kp;
  for (int v = g8; v < nv; v += 8) {
    const Vec16<T> x = ld16(mp + v * VN), y = ld16(mq + v * VN);
    Vec16<T> xo, yo;
#pragma unroll
    for (int u = 0; u < VN; ++u) {
      xo.v[u] = cs * x.v[u] - sn * y.v[u];
      yo.v[u] = sn * x.v[u] + cs * y.v[u];
    }
    st16(mp + v * VN, xo);
    st16(mq + v * VN, yo);
  }
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
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int u = 0; u < NC; ++u) w[u] += __shfl_xor_sync(0xffffffffu, w[u], o);
  }
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

// M: k x k row-major.  Uout, Vout: k x k row-major (columns in descending
// order of Sout).  qv: k * kp + k scratch (reflectors and tau of the QR).
// log: [JAC_MAX_SWEEPS * (kk-1)][kk/2] pairs of (cos, sin).  ctl[CTL_JAC_PROGRESS]
// (rounds published) and ctl[CTL_JAC_TOTAL] (total rounds, -1 while running)
// must be 0 and -1 on entry.
template <typename T>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(1024)
    jacobi_svd_kernel(const T *__restrict__ Min, int k, T *__restrict__ Uout, T *__restrict__ Sout,
                      T *__restrict__ Vout, T *__restrict__ rlog, T *__restrict__ qv, int *ctl, int max_sweeps,
                      T tol) {
  cg::cluster_group cluster = cg::this_cluster();
  const unsigned rank = cluster.block_rank();
  const int kk = k + (k & 1);
  const int npair = kk / 2;
  constexpr int VN = Vec16<T>::N;
  const int kp = (k + VN - 1) / VN * VN;  // padded column stride (16-byte aligned columns)
  const int nv = kp / VN;                 // vectors per column
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *Mat = reinterpret_cast<T *>(smem_raw);      // column c at Mat[c*kp], rows >= k zero
  T *vb0 = Mat + (size_t)kk * kp;                 // QR buffers: 4 vectors of kp, tau [kp]
  T *vb1 = vb0 + kp, *hb0 = vb1 + kp, *hb1 = hb0 + kp, *tau = hb1 + kp;
  T *sig = tau + kp;                              // [kk]
  int *rnk = reinterpret_cast<int *>(sig + kk);   // [kk]
  __shared__ int s_rot, s_fail, s_avail, s_tot;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int g8 = lane & 7;
  int *progress = ctl + CTL_JAC_PROGRESS;
  int *total = ctl + CTL_JAC_TOTAL;
  if (max_sweeps > JAC_MAX_SWEEPS) max_sweeps = JAC_MAX_SWEEPS;

  for (int e = threadIdx.x; e < kk * kp; e += blockDim.x) {
    const int c = e / kp, r = e - c * kp;
    // rank 0: M^T (column c = row c of M); rank 1: zeros (Q is formed below)
    Mat[e] = (rank == 0 && c < k && r < k) ? Min[(size_t)c * k + r] : T(0);
  }
  if (threadIdx.x == 0) {
    s_rot = 0;
    s_fail = 0;
  }
  if (rank == 0 && threadIdx.x < 16) ctl[CTL_SWEEP_ROT0 + threadIdx.x] = 0;
  __syncthreads();

  if (rank == 0) {
    precond_qr_r(Mat, k, kp, vb0, vb1, tau, qv);
    if (threadIdx.x == 0) jac_st_release(ctl + CTL_JAC_QR, 1);  // the barrier ordered every write of qv
    int round = 0;
    int sweeps = 0;
    bool done = false;
    for (; sweeps < max_sweeps && !done; ++sweeps) {
      for (int t = 0; t < kk - 1; ++t, ++round) {
        const int i = wid * JAC_PPW + (lane >> 3);
        int p = -1, q = -1;
        if (i < npair) rr_pair(t, i, kk, p, q);
        T al = T(0), be = T(0), ga = T(0);
        if (p >= 0) {
          const T *mp = Mat + (size_t)p * kp, *mq = Mat + (size_t)q * kp;
          for (int v = g8; v < nv; v += 8) {
            const Vec16<T> x = ld16(mp + v * VN), y = ld16(mq + v * VN);
#pragma unroll
            for (int u = 0; u < VN; ++u) {
              al = fma(x.v[u], x.v[u], al);
              be = fma(y.v[u], y.v[u], be);
              ga = fma(x.v[u], y.v[u], ga);
            }
          }
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        T cs = T(1), sn = T(0);
        if (p >= 0 && ga != T(0) && fabs(ga) > tol * sqrt(al * be)) {
          const T zeta = (be - al) / (T(2) * ga);
          const T tt = copysign(T(1), zeta) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
          cs = T(1) / sqrt(T(1) + tt * tt);
          sn = cs * tt;
        }
        if (sn != T(0)) rotate_cols(Mat, kp, nv, p, q, cs, sn, g8);
        if (g8 == 0 && i < npair) {
          T *e = rlog + ((size_t)round * npair + i) * 2;
          e[0] = cs;
          e[1] = sn;
          if (sn != T(0)) atomicAdd(&s_rot, 1);
        }
        __syncthreads();
        if ((round + 1) % JAC_GROUP == 0 && threadIdx.x == 0) {
          // publish the rounds so far (the barrier above ordered every warp's log writes)
          asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(progress), "r"(JAC_GROUP) : "memory");
        }
      }
      done = (s_rot == 0);
      __syncthreads();
      if (threadIdx.x == 0) {
        if (sweeps < 16) ctl[CTL_SWEEP_ROT0 + sweeps] = s_rot;
        s_rot = 0;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      ctl[CTL_JACOBI_SWEEPS] = sweeps;
      jac_st_release(total, round);  // ordered after every log write by the barriers above
    }
    // sigma and the ranks of the descending order
    for (int c = wid; c < kk; c += nwarp) {
      T acc = T(0);
      if (c < k)
        for (int r = lane; r < k; r += 32) acc = fma(Mat[(size_t)c * kp + r], Mat[(size_t)c * kp + r], acc);
      acc = warp_sum(acc);
      if (lane == 0) sig[c] = sqrt(acc);
    }
    __syncthreads();
    int *rnk1 = cluster.map_shared_rank(rnk, 1);
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
      const T sc = sig[c];
      int rk = 0;
      for (int d = 0; d < k; ++d) {
        const T sd = sig[d];
        rk += (sd > sc) || (sd == sc && d < c);
      }
      rnk[c] = rk;
      rnk1[c] = rk;
    }
  } else {
    // rank 1: Q from the published reflectors, then the published rounds of the log applied to it
    if (threadIdx.x == 0) {
      const unsigned long long t0 = jac_now();
      unsigned spins = 0;
      while (jac_ld_acquire(ctl + CTL_JAC_QR) == 0) {
        if ((++spins & 255) == 0 && jac_now() - t0 > 1000000000ull) {
          s_fail = 1;
          break;
        }
      }
    }
    __syncthreads();
    if (!s_fail) precond_qr_q(Mat, k, kp, vb0, vb1, hb0, hb1, tau, qv);
    int done_rounds = 0;
    unsigned long long t_last = jac_now();
    while (!s_fail) {
      if (threadIdx.x == 0) {
        int tt = jac_ld_acquire(total);
        int avail = (tt >= 0) ? tt : jac_ld_acquire(progress);
        unsigned spins = 0;
        while (avail <= done_rounds && tt < 0) {
          if ((++spins & 255) == 0 && jac_now() - t_last > 1000000000ull) {
            s_fail = 1;
            break;
          }
          tt = jac_ld_acquire(total);
          avail = (tt >= 0) ? tt : jac_ld_acquire(progress);
        }
        t_last = jac_now();
        s_avail = avail;
        s_tot = tt;
      }
      __syncthreads();
      if (s_fail) break;
      const int avail = s_avail, tot = s_tot;
      for (int rd = done_rounds; rd < avail; ++rd) {
        const int t = rd % (kk - 1);
        for (int i = wid * JAC_PPW + (lane >> 3); i < npair; i += nwarp * JAC_PPW) {
          const T *e = rlog + ((size_t)rd * npair + i) * 2;
          const T cs = __ldcg(e), sn = __ldcg(e + 1);  // L2 only: the line may hold later rounds
          if (sn == T(0)) continue;
          int p, q;
          rr_pair(t, i, kk, p, q);
          rotate_cols(Mat, kp, nv, p, q, cs, sn, g8);
        }
        __syncthreads();
      }
      done_rounds = avail;
      if (tot >= 0 && done_rounds >= tot) break;
      __syncthreads();
    }
    if (threadIdx.x == 0 && s_fail) set_status(ctl, STATUS_TIMEOUT);
  }
  cluster.sync();  // the ranks are now in rank 1's shared memory
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int c = e / k, r = e - c * k;
    const int rk = rnk[c];
    if (rank == 0) {
      // the normalised columns of W are the left singular vectors of M
      const T sc = sig[c];
      Uout[(size_t)r * k + rk] = (sc > T(0)) ? Mat[(size_t)c * kp + r] / sc : ((r == rk) ? T(1) : T(0));
      if (r == 0) Sout[rk] = sc;
    } else {
      Vout[(size_t)r * k + rk] = Mat[(size_t)c * kp + r];  // Q J: right singular vectors of M
    }
  }
  cluster.sync();  // neither CTA leaves while the other may still read its shared memory
}


}  // namespace ffq
