// jacobi.cuh -- SVD of the small k x k factor of tmp (Alg. 9, lines 4-5) by
// one-sided (Hestenes) Jacobi, on a 2-CTA thread-block cluster.
//
//   M V = U diag(sigma):  pairs of columns of M are rotated until every pair is
//   orthogonal to within tol * ||m_p|| ||m_q||; V accumulates the rotations.
//
// CTA rank 0 holds M (column-major, k x kk) in its shared memory, computes the
// rotations of one round of the parallel round-robin ordering (kk/2 disjoint
// pairs, every pair meets once per sweep of kk-1 rounds) and applies them to M;
// it writes each round's (cos, sin) into rank 1's shared memory (DSMEM), and
// rank 1, which holds V, applies them one round behind.  One cluster barrier
// per round.  After convergence sigma_j = ||m_j||, U(:, j) = m_j / sigma_j,
// sorted descending (ties keep column order).
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"

namespace ffq {

namespace cg = cooperative_groups;

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

template <typename T>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(1024)
    jacobi_svd_kernel(const T *__restrict__ Min, int k, T *__restrict__ Uout, T *__restrict__ Sout,
                      T *__restrict__ Vout, int *ctl, int max_sweeps, T tol) {
  cg::cluster_group cluster = cg::this_cluster();
  const unsigned rank = cluster.block_rank();
  const int kk = k + (k & 1);
  const int npair = kk / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *Mat = reinterpret_cast<T *>(smem_raw);  // column c at Mat[c*k]
  T *rc = Mat + (size_t)kk * k;               // [2][npair] cos
  T *rs = rc + 2 * npair;                     // [2][npair] sin
  T *sig = rs + 2 * npair;                    // [kk]
  int *rnk = reinterpret_cast<int *>(sig + kk);  // [kk]
  int *flags = rnk + kk;                         // [4]: 0 rotated-this-sweep, 1 done
  T *rc1 = cluster.map_shared_rank(rc, 1);
  T *rs1 = cluster.map_shared_rank(rs, 1);
  int *rnk1 = cluster.map_shared_rank(rnk, 1);
  int *flags1 = cluster.map_shared_rank(flags, 1);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;

  for (int e = threadIdx.x; e < kk * k; e += blockDim.x) {
    const int c = e / k, r = e - c * k;
    T v;
    if (rank == 0) v = (c < k) ? Min[(size_t)r * k + c] : T(0);
    else v = (r == c) ? T(1) : T(0);
    Mat[e] = v;
  }
  if (threadIdx.x < 4) flags[threadIdx.x] = 0;
  cluster.sync();

  int sweeps = 0;
  for (; sweeps < max_sweeps; ++sweeps) {
    if (rank == 0 && threadIdx.x == 0) flags[0] = 0;
    __syncthreads();
    for (int t = 0; t < kk - 1; ++t) {
      const int buf = t & 1;
      if (rank == 0) {
        for (int i = wid; i < npair; i += nwarp) {
          int p, q;
          rr_pair(t, i, kk, p, q);
          T *mp = Mat + (size_t)p * k, *mq = Mat + (size_t)q * k;
          T al = T(0), be = T(0), ga = T(0);
          for (int r = lane; r < k; r += 32) {
            const T x = mp[r], y = mq[r];
            al = fma(x, x, al);
            be = fma(y, y, be);
            ga = fma(x, y, ga);
          }
          al = warp_sum(al);
          be = warp_sum(be);
          ga = warp_sum(ga);
          T cs = T(1), sn = T(0);
          if (ga != T(0) && fabs(ga) > tol * sqrt(al * be)) {
            const T zeta = (be - al) / (T(2) * ga);
            const T tt = copysign(T(1), zeta) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
            cs = T(1) / sqrt(T(1) + tt * tt);
            sn = cs * tt;
            for (int r = lane; r < k; r += 32) {
              const T x = mp[r], y = mq[r];
              mp[r] = cs * x - sn * y;
              mq[r] = sn * x + cs * y;
            }
            if (lane == 0) flags[0] = 1;
          }
          if (lane == 0) {
            rc1[buf * npair + i] = cs;
            rs1[buf * npair + i] = sn;
          }
        }
      }
      cluster.sync();
      if (rank == 1) {
        for (int i = wid; i < npair; i += nwarp) {
          const T cs = rc[buf * npair + i], sn = rs[buf * npair + i];
          if (sn == T(0)) continue;
          int p, q;
          rr_pair(t, i, kk, p, q);
          T *mp = Mat + (size_t)p * k, *mq = Mat + (size_t)q * k;
          for (int r = lane; r < k; r += 32) {
            const T x = mp[r], y = mq[r];
            mp[r] = cs * x - sn * y;
            mq[r] = sn * x + cs * y;
          }
        }
      }
    }
    if (rank == 0 && threadIdx.x == 0) flags1[1] = (flags[0] == 0) ? 1 : 0;
    if (rank == 0 && threadIdx.x == 0) flags[1] = (flags[0] == 0) ? 1 : 0;
    cluster.sync();
    if (flags[1]) {
      ++sweeps;
      break;
    }
  }
  // sigma, ranks (rank 0), outputs
  if (rank == 0) {
    for (int c = wid; c < kk; c += nwarp) {
      T acc = T(0);
      if (c < k)
        for (int r = lane; r < k; r += 32) acc = fma(Mat[(size_t)c * k + r], Mat[(size_t)c * k + r], acc);
      acc = warp_sum(acc);
      if (lane == 0) sig[c] = sqrt(acc);
    }
    __syncthreads();
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
    if (threadIdx.x == 0) ctl[CTL_JACOBI_SWEEPS] = sweeps;
  }
  cluster.sync();
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int c = e / k, r = e - c * k;
    const int rk = rnk[c];
    if (rank == 0) {
      const T sc = sig[c];
      Uout[(size_t)r * k + rk] = (sc > T(0)) ? Mat[(size_t)c * k + r] / sc : ((r == rk) ? T(1) : T(0));
      if (r == 0) Sout[rk] = sc;
    } else {
      Vout[(size_t)r * k + rk] = Mat[(size_t)c * k + r];
    }
  }
  cluster.sync();
}

}  // namespace ffq
