// qrcp.cuh -- partial QR with column pivoting of the sketch B (Alg. 1 applied to
// the (b+p) x n sample of Alg. 2, b = k), as one persistent cooperative kernel.
//
// Layout: Bt = B^T (n x lds, column i of B is the contiguous row i of Bt).  The
// n columns are split into contiguous slabs, one per block; each block keeps
// its slab of B resident in shared memory for all k steps, together with the
// exact trailing squared norms ||B(j:s, i)||^2 of its columns.
//
// Step j (one bounded grid barrier per step):
//   1. every block publishes its best unselected column (largest trailing norm,
//      ties to the lowest original index) and a copy of that column; in single
//      precision the choice among blocks is one atomicMax on a 64-bit key
//      (value bits, then the complemented index) in one of three rotating
//      words, so after the barrier a block reads a single word;
//   2. barrier;
//   3. every block takes the same winner p (the key, or in double precision
//      the reduction of the published candidates), loads the winner's column
//      from its owner's copy and forms the Householder reflector
//      H = I - tau v v^T from B(j:s, p) (beta = -sign(x_j) ||x||);
//   4. each block applies H to its own unselected columns and recomputes their
//      trailing norms ||B(j+1:s, i)||^2 exactly (no downdating).
// Outputs: piv[0:k] (original indices, in pivot order), S11 (k x k, row-major,
// the R factor of the pivoted sketch columns: S11(0:j, j) = transformed pivot
// column above the diagonal, S11(j, j) = beta), status RANK_DEFICIENT if a
// winner has zero trailing norm.
#pragma once

#include "common.cuh"

namespace ffq {

template <typename T>
struct QrcpArgs {
  const T *Bt;
  int64_t n;
  int s, lds, k;
  int32_t *piv;
  T *S11;            // k x k
  T *cand_val;       // [2][G]
  int *cand_idx;     // [2][G]
  T *cand_col;       // [2][G][lds]
  int *sel;          // [n] 1 if selected (written for downstream kernels)
  int *ctl;
  long long spin_limit;
  int stall_step;      // failure injection: this step's barrier waits for one block too many (-1: none)
  int cols_per_block;  // slab width (columns)
  int s_pad;           // slab column stride in shared memory
};

// 16-byte vector of T in shared memory.
template <typename T>
struct QVec {
  static constexpr int N = 16 / sizeof(T);
  T v[N];
};
template <typename T>
__device__ __forceinline__ QVec<T> qld(const T *p) {
  QVec<T> r;
  if constexpr (sizeof(T) == 4) {
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
__device__ __forceinline__ void qst(T *p, const QVec<T> &r) {
  if constexpr (sizeof(T) == 4) *reinterpret_cast<float4 *>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
  else *reinterpret_cast<double2 *>(p) = make_double2(r.v[0], r.v[1]);
}

// Step 4: H applied to the block's columns and their trailing squared norms
// over rows > j recomputed.  v is held full length (zeros above row j), so
// rows above j are left as they are.  LPC lanes per column: a warp takes
// 32 / LPC columns at once and each lane a strided share of their 16-byte
// vectors, so the dot products and norms need only log2(LPC) shuffle levels
// (a warp per column would need five, on a chain per column).  Selected
// columns are transformed too (their values are not used again).
template <typename T, int LPC>
__device__ __forceinline__ void apply_reflector_lanes(T *slab, int ld, int ncol, const T *v, T tau, int j, T *nrm) {
  constexpr int VN = QVec<T>::N;
  constexpr int CPW = 32 / LPC;  // columns per warp and pass
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int gl = lane % LPC;
  const int q0 = j / VN, nq = ld / VN;
  for (int base = wid * CPW; base < ncol; base += nwarp * CPW) {  // warp-uniform
    const int c = base + lane / LPC;
    const bool on = c < ncol;
    T *col = slab + (size_t)(on ? c : 0) * ld;
    T w = T(0);
    if (on)
      for (int q = q0 + gl; q < nq; q += LPC) {
        const QVec<T> vv = qld(v + q * VN), xx = qld(col + q * VN);
#pragma unroll
        for (int e = 0; e < VN; ++e) w = fma(vv.v[e], xx.v[e], w);
      }
#pragma unroll
    for (int o = LPC / 2; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    w *= tau;
    T acc = T(0);
    if (on)
      for (int q = q0 + gl; q < nq; q += LPC) {
        const QVec<T> vv = qld(v + q * VN);
        QVec<T> xx = qld(col + q * VN);
#pragma unroll
        for (int e = 0; e < VN; ++e) {
          const T y = fma(-w, vv.v[e], xx.v[e]);
          xx.v[e] = y;
          if (q * VN + e > j) acc = fma(y, y, acc);
        }
        qst(col + q * VN, xx);
      }
#pragma unroll
    for (int o = LPC / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (on && gl == 0 && nrm[c] >= T(0)) nrm[c] = acc;  // selected columns keep their mark
  }
}

template <typename T>
__global__ void __launch_bounds__(512) qrcp_kernel(QrcpArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *slab = reinterpret_cast<T *>(smem_raw);                        // [cols][s_pad], rows >= s zero
  T *v = slab + (size_t)a.cols_per_block * a.s_pad;                 // [s_pad] (16-byte aligned)
  T *nrm = v + a.s_pad;                                             // [cols]
  __shared__ T red_v[32];
  __shared__ int red_i[32];
  __shared__ T s_tau, s_beta, s_scal;
  __shared__ int s_win_blk, s_win_col;

  const int G = gridDim.x, b = blockIdx.x;
  const int64_t c0 = (a.n * b) / G, c1 = (a.n * (b + 1)) / G;
  const int ncol = (int)(c1 - c0);
  const int s = a.s;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  unsigned *bar = reinterpret_cast<unsigned *>(a.ctl + CTL_BARRIER0);
  unsigned long long *wkey = reinterpret_cast<unsigned long long *>(a.ctl + CTL_WIN_KEY);  // zero on entry

  // load slab (zero padding rows), initial norms
  for (int c = wid; c < ncol; c += nwarp) {
    T acc = T(0);
    for (int t = lane; t < a.s_pad; t += 32) {
      const T x = (t < s) ? a.Bt[(c0 + c) * a.lds + t] : T(0);
      slab[(size_t)c * a.s_pad + t] = x;
      acc += x * x;
    }
    acc = warp_sum(acc);
    if (lane == 0) nrm[c] = acc;
  }
  __syncthreads();

  for (int j = 0; j < a.k; ++j) {
    const int buf = j & 1;
    // 1. local candidate
    T bv = neg_inf<T>();
    int bi = 0x7fffffff;
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
      const T x = nrm[c];
      if (x >= T(0) && better(x, (int)(c0 + c), bv, bi)) {
        bv = x;
        bi = (int)(c0 + c);
      }
    }
    block_argmax(bv, bi, red_v, red_i);
    if (threadIdx.x == 0) {
      if constexpr (sizeof(T) == 4) {
        // single precision: the winner is one atomicMax over order-preserving
        // keys (value bits high, ~index low: larger value, then lower index)
        if (bi != 0x7fffffff)
          atomicMax(wkey + j % 3, ((unsigned long long)__float_as_uint((float)bv) << 32) |
                                      (unsigned long long)(0xffffffffu - (unsigned)bi));
      } else {
        a.cand_val[buf * G + b] = bv;
        a.cand_idx[buf * G + b] = bi;
      }
    }
    if (bi != 0x7fffffff) {
      const int lc = (int)(bi - c0);
      for (int t = threadIdx.x; t < s; t += blockDim.x)
        a.cand_col[((size_t)buf * G + b) * a.lds + t] = slab[(size_t)lc * a.s_pad + t];
    }
    // 2. barrier
    if (!grid_barrier(bar, (unsigned)((j + 1) * G + (j == a.stall_step ? 1 : 0)), a.ctl, a.spin_limit)) return;
    // 3. winner, reflector
    {
      T wv = neg_inf<T>();
      int wi = 0x7fffffff, wb = -1;
      if constexpr (sizeof(T) == 4) {
        if (threadIdx.x == 0) {
          const unsigned long long key = *reinterpret_cast<volatile unsigned long long *>(wkey + j % 3);
          if (key != 0ull) {
            wv = (T)__uint_as_float((unsigned)(key >> 32));
            wi = (int)(0xffffffffu - (unsigned)(key & 0xffffffffull));
          }
          // the key of step j + 2: last read at step j - 1, next written after the barrier of step j + 1
          if (b == 0) wkey[(j + 2) % 3] = 0ull;
        }
      } else {
        for (int g = threadIdx.x; g < G; g += blockDim.x) {
          const T x = a.cand_val[buf * G + g];
          const int ix = a.cand_idx[buf * G + g];
          if (ix != 0x7fffffff && better(x, ix, wv, wi)) {
            wv = x;
            wi = ix;
          }
        }
        block_argmax(wv, wi, red_v, red_i);
      }
      if (threadIdx.x == 0 && wi == 0x7fffffff) {
        // no finite candidate left (NaN input): record and skip this step
        s_win_blk = -1;
        s_win_col = -1;
        set_status(a.ctl, STATUS_NONFINITE);
      } else if (threadIdx.x == 0) {
        // the block owning column wi: the largest b with floor(n b / G) <= wi
        wb = (int)((((int64_t)wi + 1) * G - 1) / a.n);
        s_win_blk = wb;
        s_win_col = wi;
        if (!(wv > T(0))) set_status(a.ctl, STATUS_RANK_DEFICIENT);
      }
      __syncthreads();
      wb = s_win_blk;
      wi = s_win_col;
      if (wb < 0) continue;  // uniform across blocks: every block saw the same candidates
      // one element of the winner column per thread (s_pad <= blockDim.x)
      const T *x = a.cand_col + ((size_t)buf * G + wb) * a.lds;
      const int t = threadIdx.x;
      const T xt = (t < s) ? x[t] : T(0);
      if (t == 0) {
        // the winner's trailing norm wv = ||x(j:s)||^2 is known, so the
        // reflector needs only alpha = x(j): beta = -sign(alpha) sqrt(wv);
        // ||x(j+1:s)||^2 = wv - alpha^2 only decides whether H = I
        const T alpha = x[j];
        T tau = T(0), beta = alpha;
        if (wv - alpha * alpha > T(0)) {
          const T normx = sqrt(wv);
          beta = (alpha >= T(0)) ? -normx : normx;
          tau = (beta - alpha) / beta;
        }
        s_tau = tau;
        s_beta = beta;
        s_scal = (tau != T(0)) ? T(1) / (alpha - beta) : T(0);
        if (b == 0) a.piv[j] = wi;
        a.sel[wi] = 1;
      }
      __syncthreads();
      const T tau = s_tau, beta = s_beta;
      // column j of S11: transformed pivot column above the diagonal, beta, zeros
      if (b == 0 && t < a.k) a.S11[(size_t)t * a.k + j] = (t < j) ? xt : ((t == j) ? beta : T(0));
      // v as the full-length reflector: zeros above row j and in the padding,
      // 1 at row j; rows above j then see v = 0 and stay as they are
      if (t < a.s_pad) v[t] = (t < j || t >= s) ? T(0) : ((t == j) ? T(1) : xt * s_scal);
      if (b == wb && threadIdx.x == 0) nrm[wi - c0] = T(-1);  // selected
      __syncthreads();
      // 4. apply H to the block's columns and recompute the unselected ones'
      //    trailing norms ||B(j+1:s, i)||^2 (tau = 0: norms only)
      apply_reflector_lanes<T, 2>(slab, a.s_pad, ncol, v, tau, j, nrm);
      __syncthreads();
    }
  }
}

}  // namespace ffq
