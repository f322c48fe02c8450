// srqr_swap.cuh -- the swap loop of strong rank-revealing QR (Alg. 4) as one
// cooperative persistent kernel, so the data-dependent loop "while g2 > g"
// runs on the device without a host round trip.
//
// State (original column order; position j < k of the factorisation holds
// column piv[j], position k the current candidate c = ctl[CTL_CAND]):
//   gt   (n x ldg)  R(t, col) = gt[col * ldg + t], rows t < k
//   rowk (n)        R(k, col)
//   q1   (m x ldq)  Q(:, 0:k);  qk (m) = Q(:, k)
//   z    (m)        residual of the candidate (unnormalised), alpha = ||z||
//   r    (n)        trailing-norm estimates of the unselected columns
//   sel  (n)        1 for the k selected columns
// One iteration (each phase ends with a bounded grid barrier):
//   a. q = z / alpha, row k of R = q^T A (one pass over A), zero at selected
//      columns and alpha at c; downdate r_i -= R(k, i)^2 for the trailing
//      columns (the one-step QR of the candidate, Alg. 4);
//   b. block 0: cyclic shift of positions imax..k (the leaving column
//      piv[imax] goes to position k, c enters at k - 1) and the Givens
//      rotations G(j, j+1), j = imax..k-1, that restore upper-triangular
//      form, computed by carrying the partially rotated row down;
//   c. all blocks apply the rotations to the rows of R (every column) and to
//      the columns of Q (every row);
//   d. r(leave) = R(k, leave)^2, r_i += R(k, i)^2 for the other unselected
//      columns; the new candidate is the argmax (ties: lowest column index);
//   e. one-step QR of the new candidate: z = A(:, c) - Q1 a with a =
//      R(0:k, c), re-orthogonalised once, alpha = ||z||;
//   f. R11^{-1} (warp-parallel back substitution), and the closed form
//      g2 = max(1, max_i sqrt(alpha^2 ||e_i^T R11^{-1}||^2 + ((R11^{-1} a)_i)^2))
//      with its maximising row imax (the next leaving position); or, with
//      g2_rows = d >= 1, block 0 forms Alg. 4's d-row random estimate of the
//      same column norms (g2est_block) and takes its maximum and argmax.
// Reductions are done in fixed block order, so results do not depend on
// timing.  A barrier that times out sets STATUS_TIMEOUT and every block
// returns.
#pragma once

#include "common.cuh"
#include "dense_small.cuh"

namespace ffq {

constexpr int CTL_LEAVE = 7;   // leaving column of the current swap (ctl slot)
constexpr int SWAP_GV = 16;    // columns per thread per chunk of the row-k pass

template <typename T>
struct SwapArgs {
  const T *A;
  int64_t lda, m, n;
  int k;
  T *gt;
  int64_t ldg;
  T *rowk;
  T *q1;
  int64_t ldq;
  T *qk, *z, *r;
  int *sel;
  int32_t *piv;
  T *rot;      // 2k: (cs, sn) of G(j, j+1)
  T *Rd;       // k x k: R11 in position order
  T *X;        // k x k: R11^{-1}
  T *part;     // G x max(n, k + 1) partial sums
  T *bv;       // G block argmax values
  int *bi;     // G block argmax columns
  int *ctl;
  double *dctl;
  double g;
  int max_swaps;
  long long spin_limit;
  int g2_rows;    // 0: exact g2; d >= 1: Alg. 4's d-row estimate
  uint64_t seed;  // the run's seed (the estimate's Omega_t)
};

// R(t, col) for t <= k.
template <typename T>
__device__ __forceinline__ T swap_rv(const SwapArgs<T> &a, int t, int64_t col) {
  return (t < a.k) ? a.gt[col * a.ldg + t] : a.rowk[col];
}

template <typename T>
__global__ void __launch_bounds__(512) srqr_swap_kernel(SwapArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int k = a.k;
  T *carry = reinterpret_cast<T *>(smem_raw);  // k + 1 (block 0, phase b)
  T *as = carry + (k + 1);                     // k: a = R(0:k, c)
  T *hs = as + k;                              // k: h = Q1^T z
  T *wacc = hs + k;                            // nwarp x k: per-warp rows / accumulators
  __shared__ T red_v[32];
  __shared__ int red_i[32];
  __shared__ int s_go, s_c, s_sing;
  __shared__ T s_alpha;
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nwarp = nt >> 5;
  const int64_t m = a.m, n = a.n;
  const int64_t mr0 = m * b / G, mr1 = m * (b + 1) / G;  // this block's rows
  const int64_t nc0 = n * b / G, nc1 = n * (b + 1) / G;  // this block's columns
  unsigned *bar = reinterpret_cast<unsigned *>(a.ctl + CTL_BARRIER1);
  unsigned nbar = 0;
  auto sync_grid = [&]() -> bool {
    ++nbar;
    return grid_barrier(bar, nbar * (unsigned)G, a.ctl, a.spin_limit);
  };

  for (;;) {
    if (tid == 0) s_go = a.ctl[CTL_NEED_SWAP];
    __syncthreads();
    if (!s_go) break;  // identical in every block: written before the last barrier
    const int c = a.ctl[CTL_CAND];
    const T alpha = (T)a.dctl[D_ALPHA];

    // a. q = z / alpha; row k of R = q^T A (block partials over its rows)
    for (int64_t t = mr0 + tid; t < mr1; t += nt) a.qk[t] = (alpha > T(0)) ? a.z[t] / alpha : T(0);
    __syncthreads();
    for (int64_t cb = 0; cb < n; cb += (int64_t)nt * SWAP_GV) {
      T acc[SWAP_GV];
#pragma unroll
      for (int u = 0; u < SWAP_GV; ++u) acc[u] = T(0);
      for (int64_t t = mr0; t < mr1; ++t) {
        const T qt = a.qk[t];
        const T *Ar = a.A + t * a.lda;
#pragma unroll
        for (int u = 0; u < SWAP_GV; ++u) {
          const int64_t col = cb + tid + (int64_t)u * nt;
          if (col < n) acc[u] = fma(qt, Ar[col], acc[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < SWAP_GV; ++u) {
        const int64_t col = cb + tid + (int64_t)u * nt;
        if (col < n) a.part[(int64_t)b * n + col] = acc[u];
      }
    }
    if (!sync_grid()) return;
    for (int64_t col = nc0 + tid; col < nc1; col += nt) {
      T s = T(0);
      for (int bb = 0; bb < G; ++bb) s += a.part[(int64_t)bb * n + col];
      const bool in = a.sel[col] != 0;
      const T rk = in ? T(0) : ((col == c) ? alpha : s);
      a.rowk[col] = rk;
      if (!in && col != c) a.r[col] -= rk * rk;
    }
    if (!sync_grid()) return;

    // b. cyclic shift and the Givens parameters (block 0)
    if (b == 0) {
      const int imax = a.ctl[CTL_IMAX];
      // column at position p >= imax after the shift
      auto colp = [&](int p) -> int64_t {
        return (p < k - 1) ? (int64_t)a.piv[p + 1] : ((p == k - 1) ? (int64_t)c : (int64_t)a.piv[imax]);
      };
      for (int p = imax + tid; p <= k; p += nt) carry[p] = swap_rv(a, imax, colp(p));
      __syncthreads();
      for (int j = imax; j < k; ++j) {
        const T x0 = carry[j], x1 = swap_rv(a, j + 1, colp(j));
        const T h = hypot(x0, x1);
        const T cs = (h != T(0)) ? x0 / h : T(1), sn = (h != T(0)) ? x1 / h : T(0);
        if (tid == 0) {
          a.rot[2 * j] = cs;
          a.rot[2 * j + 1] = sn;
        }
        __syncthreads();  // every thread has read carry[j]
        for (int p = j + 1 + tid; p <= k; p += nt) carry[p] = -sn * carry[p] + cs * swap_rv(a, j + 1, colp(p));
        __syncthreads();
      }
      if (tid == 0) {
        const int leave = a.piv[imax];
        for (int p = imax; p < k - 1; ++p) a.piv[p] = a.piv[p + 1];
        a.piv[k - 1] = c;
        a.sel[c] = 1;
        a.sel[leave] = 0;
        a.ctl[CTL_LEAVE] = leave;
      }
    }
    if (!sync_grid()) return;

    // c. apply G(j, j+1), j = imax..k-1, to the rows of R and the columns of Q
    {
      const int imax = a.ctl[CTL_IMAX];
      for (int64_t col = nc0 + tid; col < nc1; col += nt) {
        T cur = swap_rv(a, imax, col);
        for (int j = imax; j < k; ++j) {
          const T nxt = swap_rv(a, j + 1, col);
          const T cs = a.rot[2 * j], sn = a.rot[2 * j + 1];
          a.gt[col * a.ldg + j] = cs * cur + sn * nxt;
          cur = -sn * cur + cs * nxt;
        }
        a.rowk[col] = cur;
      }
      for (int64_t t = mr0 + tid; t < mr1; t += nt) {
        T *qr = a.q1 + t * a.ldq;
        T cur = qr[imax];
        for (int j = imax; j < k; ++j) {
          const T nxt = (j + 1 < k) ? qr[j + 1] : a.qk[t];
          const T cs = a.rot[2 * j], sn = a.rot[2 * j + 1];
          qr[j] = cs * cur + sn * nxt;
          cur = -sn * cur + cs * nxt;
        }
        a.qk[t] = cur;
      }
    }
    if (!sync_grid()) return;

    // d. trailing estimates and the new candidate
    {
      const int leave = a.ctl[CTL_LEAVE];
      T bv = neg_inf<T>();
      int bi = 0x7fffffff;
      for (int64_t col = nc0 + tid; col < nc1; col += nt) {
        if (a.sel[col]) continue;
        const T rk = a.rowk[col];
        const T rv = (col == leave) ? rk * rk : a.r[col] + rk * rk;
        a.r[col] = rv;
        if (better(rv, (int)col, bv, bi)) {
          bv = rv;
          bi = (int)col;
        }
      }
      block_argmax(bv, bi, red_v, red_i);
      if (tid == 0) {
        a.bv[b] = bv;
        a.bi[b] = bi;
      }
    }
    if (!sync_grid()) return;

    // e. one-step QR of the new candidate
    {
      T bv = neg_inf<T>();
      int bi = 0x7fffffff;
      for (int bb = tid; bb < G; bb += nt)
        if (a.bi[bb] != 0x7fffffff && better(a.bv[bb], a.bi[bb], bv, bi)) {
          bv = a.bv[bb];
          bi = a.bi[bb];
        }
      block_argmax(bv, bi, red_v, red_i);
      if (tid == 0) s_c = bi;
      __syncthreads();
    }
    const int c2 = s_c;  // a trailing column always exists while swaps run (k < n)
    for (int j = tid; j < k; j += nt) as[j] = a.gt[(int64_t)c2 * a.ldg + j];
    for (int j = tid; j < nwarp * k; j += nt) wacc[j] = T(0);
    __syncthreads();
    for (int64_t t = mr0 + wid; t < mr1; t += nwarp) {
      const T *qr = a.q1 + t * a.ldq;
      T acc = T(0);
      for (int j = lane; j < k; j += 32) acc = fma(qr[j], as[j], acc);
      acc = warp_sum(acc);
      const T zt = a.A[t * a.lda + c2] - acc;
      if (lane == 0) a.z[t] = zt;
      for (int j = lane; j < k; j += 32) wacc[wid * k + j] = fma(qr[j], zt, wacc[wid * k + j]);
    }
    __syncthreads();
    for (int j = tid; j < k; j += nt) {
      T s = T(0);
      for (int w = 0; w < nwarp; ++w) s += wacc[w * k + j];
      a.part[(int64_t)b * (k + 1) + j] = s;
    }
    if (!sync_grid()) return;
    for (int j = tid; j < k; j += nt) {
      T s = T(0);
      for (int bb = 0; bb < G; ++bb) s += a.part[(int64_t)bb * (k + 1) + j];
      hs[j] = s;
    }
    __syncthreads();
    {
      T nacc = T(0);
      for (int64_t t = mr0 + wid; t < mr1; t += nwarp) {
        const T *qr = a.q1 + t * a.ldq;
        T acc = T(0);
        for (int j = lane; j < k; j += 32) acc = fma(qr[j], hs[j], acc);
        acc = warp_sum(acc);
        const T zt = a.z[t] - acc;
        if (lane == 0) {
          a.z[t] = zt;
          nacc = fma(zt, zt, nacc);
        }
      }
      nacc = block_sum(nacc, red_v);
      // own slot k of this block's partial row: not read by the h reduction
      if (tid == 0) a.part[(int64_t)b * (k + 1) + k] = nacc;
    }
    // R11 in position order
    for (int e = b * nt + tid; e < k * k; e += G * nt) {
      const int t = e / k, j = e - t * k;
      a.Rd[e] = (t <= j) ? a.gt[(int64_t)a.piv[j] * a.ldg + t] : T(0);
    }
    if (!sync_grid()) return;
    if (tid == 0) {
      T s = T(0);
      for (int bb = 0; bb < G; ++bb) s += a.part[(int64_t)bb * (k + 1) + k];
      s_alpha = sqrt(s);
      s_sing = 0;
    }
    __syncthreads();
    if (a.g2_rows > 0) {
      // f (estimate). Block 0 draws Omega_t for test t = the new swap count
      // and takes the estimated column norms; the others wait at the barrier.
      if (b == 0) {
        const int t = a.ctl[CTL_SWAPS] + 1;
        const int zero = g2est_block<T>(a.Rd, k, as, s_alpha, k, a.g2_rows, a.seed, t, wacc);
        const T *colsq = wacc + g2est_smem_elems(k) - k;
        T bv = T(1);
        int bi = 0x7fffffff;
        for (int i = tid; i < k; i += nt) {
          const T val = sqrt(colsq[i] / T(a.g2_rows));
          if (better(val, i, bv, bi)) {
            bv = val;
            bi = i;
          }
        }
        block_argmax(bv, bi, red_v, red_i);
        if (tid == 0) {
          const double g2 = zero ? 1.0 : (double)bv;
          a.ctl[CTL_SWAPS] = t;
          a.ctl[CTL_CAND] = c2;
          a.ctl[CTL_IMAX] = (zero || bi == 0x7fffffff) ? -1 : bi;
          a.dctl[D_G2] = g2;
          a.dctl[D_ALPHA] = (double)s_alpha;
          const bool need = g2 > a.g && a.ctl[CTL_IMAX] >= 0;
          a.ctl[CTL_NEED_SWAP] = (need && t < a.max_swaps) ? 1 : 0;
          if (need && t >= a.max_swaps) set_status(a.ctl, STATUS_SWAP_CAP);
        }
      }
      if (!sync_grid()) return;
      continue;
    }
    // f. X = R11^{-1}: global warp gw solves R11 x = e_j for j = gw, gw + G*nwarp, ...
    for (int j = b * nwarp + wid; j < k; j += G * nwarp) {
      T *acc = wacc + wid * k;
      for (int i = lane; i < k; i += 32) acc[i] = (i == j) ? T(1) : T(0);
      __syncwarp();
      for (int i = j; i >= 0; --i) {
        const T d = a.Rd[i * k + i];
        const T xi = (d != T(0)) ? acc[i] / d : T(0);
        __syncwarp();
        for (int t = lane; t < i; t += 32) acc[t] = fma(-a.Rd[t * k + i], xi, acc[t]);
        if (lane == 0) acc[i] = xi;
        __syncwarp();
      }
      for (int i = lane; i < k; i += 32) a.X[(int64_t)i * k + j] = (i <= j) ? acc[i] : T(0);
      __syncwarp();
    }
    if (!sync_grid()) return;
    if (b == 0) {
      const T al = s_alpha;
      T bv = T(1);
      int bi = 0x7fffffff;
      for (int i = tid; i < k; i += nt) {
        if (a.Rd[i * k + i] == T(0)) s_sing = 1;
        T rn = T(0), u = T(0);
        for (int j = i; j < k; ++j) {
          const T x = a.X[(int64_t)i * k + j];
          rn = fma(x, x, rn);
          u = fma(x, as[j], u);
        }
        const T val = sqrt(al * al * rn + u * u);
        if (better(val, i, bv, bi)) {
          bv = val;
          bi = i;
        }
      }
      block_argmax(bv, bi, red_v, red_i);
      if (tid == 0) {
        const double g2 = s_sing ? 1.0 : (double)bv;
        const int swaps = a.ctl[CTL_SWAPS] + 1;
        a.ctl[CTL_SWAPS] = swaps;
        a.ctl[CTL_CAND] = c2;
        a.ctl[CTL_IMAX] = (s_sing || bi == 0x7fffffff) ? -1 : bi;
        a.dctl[D_G2] = g2;
        a.dctl[D_ALPHA] = (double)al;
        const bool need = g2 > a.g && a.ctl[CTL_IMAX] >= 0;
        a.ctl[CTL_NEED_SWAP] = (need && swaps < a.max_swaps) ? 1 : 0;
        if (need && swaps >= a.max_swaps) set_status(a.ctl, STATUS_SWAP_CAP);
      }
    }
    if (!sync_grid()) return;
  }
}

}  // namespace ffq
