// jacobi.cuh -- SVD of the small k x k factor of tmp (Alg. 9, lines 4-5) by
// one-sided (Hestenes) Jacobi, on a 2-CTA thread-block cluster.
//
//   X J = W diag(sigma) with X = M^T:  pairs of columns of X (rows of M) are
//   rotated until every pair is orthogonal to within tol * ||x_p|| ||x_q||;
//   J accumulates the rotations.  Then M = J diag(sigma) W^T, i.e. U = J and
//   V = W normalised.  (Working on the rows of M is the usual preconditioning
//   of one-sided Jacobi for a matrix built from a column-pivoted R factor.)
//
// Rank 0 holds X (column-major, padded stride) in shared memory and runs the
// parallel round-robin ordering: kk/2 disjoint pairs per round, every pair
// meets once per sweep of kk-1 rounds.  Each pair is handled by 8 lanes (four
// pairs per warp) with 16-byte shared-memory accesses.  The (cos, sin) of every
// round go to a rotation log in global memory; every JAC_GROUP rounds one
// gpu-scope release publishes the progress counter.  Rank 1 holds J and applies
// the logged rounds as they are published (acquire loads of the counter), so
// the two CTAs never wait on each other per round.  After convergence (a sweep
// without rotations) sigma_j = ||x_j||, the ranks of the sorted order go to
// rank 1 through DSMEM, and both write their outputs.  All waits are bounded.
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

// log: [JAC_MAX_SWEEPS * (kk-1)][kk/2] pairs of (cos, sin).  ctl[CTL_JAC_PROGRESS]
// (rounds published) and ctl[CTL_JAC_TOTAL] (total rounds, -1 while running)
// must be 0 and -1 on entry.
template <typename T>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(1024)
    jacobi_svd_kernel(const T *__restrict__ Min, int k, T *__restrict__ Uout, T *__restrict__ Sout,
                      T *__restrict__ Vout, T *__restrict__ rlog, int *ctl, int max_sweeps, T tol) {
  cg::cluster_group cluster = cg::this_cluster();
  const unsigned rank = cluster.block_rank();
  const int kk = k + (k & 1);
  const int npair = kk / 2;
  constexpr int VN = Vec16<T>::N;
  const int kp = (k + VN - 1) / VN * VN;  // padded column stride (16-byte aligned columns)
  const int nv = kp / VN;                 // vectors per column
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *Mat = reinterpret_cast<T *>(smem_raw);      // column c at Mat[c*kp], rows >= k zero
  T *sig = Mat + (size_t)kk * kp;                 // [kk]
  int *rnk = reinterpret_cast<int *>(sig + kk);   // [kk]
  __shared__ int s_rot, s_fail, s_avail, s_tot;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int g8 = lane & 7;
  int *progress = ctl + CTL_JAC_PROGRESS;
  int *total = ctl + CTL_JAC_TOTAL;
  if (max_sweeps > JAC_MAX_SWEEPS) max_sweeps = JAC_MAX_SWEEPS;

  for (int e = threadIdx.x; e < kk * kp; e += blockDim.x) {
    const int c = e / kp, r = e - c * kp;
    T v;
    if (rank == 0) v = (c < k && r < k) ? Min[(size_t)c * k + r] : T(0);  // X = M^T
    else v = (r == c && r < k) ? T(1) : T(0);                              // J = I
    Mat[e] = v;
  }
  if (threadIdx.x == 0) {
    s_rot = 0;
    s_fail = 0;
  }
  if (rank == 0 && threadIdx.x < 16) ctl[CTL_SWEEP_ROT0 + threadIdx.x] = 0;
  __syncthreads();

  if (rank == 0) {
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
    // rank 1: apply the published rounds of the log to J
    int done_rounds = 0;
    unsigned long long t_last = jac_now();
    while (true) {
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
      // the normalised columns of W are the right singular vectors of M
      const T sc = sig[c];
      Vout[(size_t)r * k + rk] = (sc > T(0)) ? Mat[(size_t)c * kp + r] / sc : ((r == rk) ? T(1) : T(0));
      if (r == 0) Sout[rk] = sc;
    } else {
      Uout[(size_t)r * k + rk] = Mat[(size_t)c * kp + r];  // J: left singular vectors of M
    }
  }
  cluster.sync();  // neither CTA leaves while the other may still read its shared memory
}

}  // namespace ffq
