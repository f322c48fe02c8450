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
// Single precision takes up to QRCP_MAXP pivots per grid barrier: besides
// its best column every block publishes a bound, the largest trailing norm
// among its other columns.  After the barrier every block applies the
// winner's reflector H_j to the published candidates whose norm exceeds the
// largest bound (at most QRCP_MAXC of them, read from the candidate copies)
// and takes the best updated norm: trailing norms only shrink under the
// reflectors, so if that norm exceeds every bound no other column can reach
// it, and it is step j + 1's greedy winner.  The same test is repeated with
// H_{j+1} applied to the remaining candidates, and so on, until a best norm
// fails the test or QRCP_MAXP pivots are taken; all of the barrier's
// reflectors are then applied to the slabs in one pass.  Every block computes
// the same certificates from the same published data, so all take the same
// decisions.  On the benchmark sketch (k = 200) the barriers fall from 108
// (at most two pivots each) to 68.
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
  T *cand_val;       // [2][2][G]: per buffer the blocks' best trailing norms, then their bounds
  int *cand_idx;     // [2][G]
  T *cand_col;       // [2][G][lds]
  int *sel;          // [n] 1 if selected (written for downstream kernels)
  int *ctl;
  long long spin_limit;
  int stall_step;      // failure injection: this step's barrier waits for one block too many (-1: none)
  int cols_per_block;  // slab width (columns)
  int s_pad;           // slab column stride in shared memory
  // columns already selected by an earlier TRQRCP block (nonzero entries are
  // never pivots; may be sel itself: it is read before the first barrier,
  // and written only after it); nullptr: none
  const int *presel = nullptr;
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
#pragma unroll 4
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
#pragma unroll 4
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

constexpr int QRCP_MAXC = 48;  // candidate columns evaluated for further pivots per barrier
constexpr int QRCP_CPW = 3;    // of which one warp of 16 evaluates up to three
constexpr int QRCP_MAXP = 4;   // pivots taken per barrier at most (single precision)

// Shared-memory floats past the slab and its norms in single precision: the
// reflectors 2 .. QRCP_MAXP of a barrier and the QRCP_MAXC candidate columns.
__host__ __device__ inline int qrcp_pair_extra(int s_pad) { return (QRCP_MAXP - 1 + QRCP_MAXC) * s_pad; }

// H_P ... H_1 applied to the block's columns (H_i = I - tau_i v_i v_i^T from
// row j + i - 1) in one read pass and one update pass:
//   H_P ... H_1 x = x - sum_i w_i v_i,  w_i = tau_i (v_i.x - sum_{l<i} (v_i.v_l) w_l),
// trailing norms over rows > j + P - 1 recomputed; LPC lanes per column as in
// apply_reflector_lanes.  cc[i][l] = v_i.v_l for l < i.
template <int P, int LPC>
__device__ __forceinline__ void apply_reflectors_lanes(float *slab, int ld, int ncol, float *const *vp,
                                                       const float *tau, const float (*cc)[QRCP_MAXP], int j,
                                                       float *nrm) {
  constexpr int VN = 4;
  constexpr int CPW = 32 / LPC;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int gl = lane % LPC;
  const int q0 = j / VN, nq = ld / VN;
  const int jn = j + P - 1;  // norms over rows > jn
  const float *vv[P];
#pragma unroll
  for (int i = 0; i < P; ++i) vv[i] = vp[i];
  for (int base = wid * CPW; base < ncol; base += nwarp * CPW) {  // warp-uniform
    const int c = base + lane / LPC;
    const bool on = c < ncol;
    float *col = slab + (size_t)(on ? c : 0) * ld;
    float d[P];
#pragma unroll
    for (int i = 0; i < P; ++i) d[i] = 0.f;
    if (on)
#pragma unroll 2
      for (int q = q0 + gl; q < nq; q += LPC) {
        const float4 xx = *reinterpret_cast<const float4 *>(col + q * VN);
#pragma unroll
        for (int i = 0; i < P; ++i) {
          const float4 u = *reinterpret_cast<const float4 *>(vv[i] + q * VN);
          d[i] = fmaf(u.x, xx.x, fmaf(u.y, xx.y, fmaf(u.z, xx.z, fmaf(u.w, xx.w, d[i]))));
        }
      }
#pragma unroll
    for (int o = LPC / 2; o > 0; o >>= 1)
#pragma unroll
      for (int i = 0; i < P; ++i) d[i] += __shfl_xor_sync(0xffffffffu, d[i], o);
    float w[P];
#pragma unroll
    for (int i = 0; i < P; ++i) {
      float t = d[i];
#pragma unroll
      for (int l = 0; l < i; ++l) t = fmaf(-cc[i][l], w[l], t);
      w[i] = tau[i] * t;
    }
    float acc = 0.f;
    if (on)
#pragma unroll 2
      for (int q = q0 + gl; q < nq; q += LPC) {
        const float4 xx = *reinterpret_cast<const float4 *>(col + q * VN);
        float y[4] = {xx.x, xx.y, xx.z, xx.w};
#pragma unroll
        for (int i = 0; i < P; ++i) {
          const float4 u = *reinterpret_cast<const float4 *>(vv[i] + q * VN);
          y[0] = fmaf(-w[i], u.x, y[0]);
          y[1] = fmaf(-w[i], u.y, y[1]);
          y[2] = fmaf(-w[i], u.z, y[2]);
          y[3] = fmaf(-w[i], u.w, y[3]);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (q * VN + e > jn) acc = fmaf(y[e], y[e], acc);
        *reinterpret_cast<float4 *>(col + q * VN) = make_float4(y[0], y[1], y[2], y[3]);
      }
#pragma unroll
    for (int o = LPC / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (on && gl == 0 && nrm[c] >= 0.f) nrm[c] = acc;  // selected columns keep their mark
  }
}

// Block-wide top two of (value, index) pairs merged with each thread's
// second value: every thread gets the block's best (v1, i1) and the best
// value among the rest (v2).  redv / redi / red2 hold >= 32 entries.
__device__ __forceinline__ void block_top2(float &v1, int &i1, float &v2, float *redv, int *redi, float *red2) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  auto merge = [](float &a1, int &ai, float &a2, float b1, int bi, float b2) {
    if (better(b1, bi, a1, ai)) {
      a2 = fmaxf(b2, a1);
      a1 = b1;
      ai = bi;
    } else {
      a2 = fmaxf(a2, b1);
    }
  };
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float b1 = __shfl_xor_sync(0xffffffffu, v1, o), b2 = __shfl_xor_sync(0xffffffffu, v2, o);
    const int bi = __shfl_xor_sync(0xffffffffu, i1, o);
    merge(v1, i1, v2, b1, bi, b2);
  }
  __syncthreads();
  if (lane == 0) {
    redv[wid] = v1;
    redi[wid] = i1;
    red2[wid] = v2;
  }
  __syncthreads();
  if (wid == 0) {
    float a1 = (lane < nw) ? redv[lane] : -INFINITY, a2 = (lane < nw) ? red2[lane] : -INFINITY;
    int ai = (lane < nw) ? redi[lane] : 0x7fffffff;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float b1 = __shfl_xor_sync(0xffffffffu, a1, o), b2 = __shfl_xor_sync(0xffffffffu, a2, o);
      const int bi = __shfl_xor_sync(0xffffffffu, ai, o);
      merge(a1, ai, a2, b1, bi, b2);
    }
    if (lane == 0) {
      redv[0] = a1;
      redi[0] = ai;
      red2[0] = a2;
    }
  }
  __syncthreads();
  v1 = redv[0];
  i1 = redi[0];
  v2 = red2[0];
  __syncthreads();
}

// Single precision: up to QRCP_MAXP pivots per grid barrier (see the file comment).
// After the barrier only two dependent L2 round trips sit on the critical
// path: (winner key | candidate table), then (winner column | candidate
// columns, prefetched by the candidate warps into registers).
constexpr int QRCP_TAB = 8;   // candidate-table entries per lane (grid <= 256)
constexpr int QRCP_COL = 8;   // column entries per lane (s_pad <= 256)
__device__ __forceinline__ void qrcp_multi_f32(const QrcpArgs<float> &a, float *slab, float *v, float *nrm,
                                               float *vx, int64_t c0, int ncol) {
  // reflector i of a barrier: v (the winner's), then the QRCP_MAXP - 1 vectors
  // at vx; the candidate columns after them
  auto vpt = [&](int i) { return (i == 0) ? v : vx + (size_t)(i - 1) * a.s_pad; };
  float *ybuf = vx + (size_t)(QRCP_MAXP - 1) * a.s_pad;
  __shared__ float red_v[32], red_2[32];
  __shared__ int red_i[32];
  __shared__ float s_tau, s_beta, s_scal, s_wv, s_bound;
  __shared__ float s_tl[QRCP_MAXP];             // tau of the barrier's reflectors
  __shared__ float s_cc[QRCP_MAXP][QRCP_MAXP];  // v_i . v_l, l < i
  __shared__ int s_win_blk, s_win_col, s_ncand, s_pair;
  __shared__ int s_cblk[QRCP_MAXC], s_cidx[QRCP_MAXC];
  __shared__ float s_cnn[QRCP_MAXC];
  const int G = gridDim.x, b = blockIdx.x;
  const int s = a.s, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  unsigned *bar = reinterpret_cast<unsigned *>(a.ctl + CTL_BARRIER0);
  unsigned long long *wkey = reinterpret_cast<unsigned long long *>(a.ctl + CTL_WIN_KEY);  // zero on entry
  float *cv1 = a.cand_val, *cv2 = a.cand_val + 2 * G;  // [buf][G] bests, [buf][G] bounds
  int nbar = 0;
  int j = 0;
  while (j < a.k) {
    const int buf = nbar & 1;
    // 1. the block's best unselected column and its bound (best of the rest)
    float v1 = -INFINITY, v2b = -INFINITY;
    int i1 = 0x7fffffff;
    for (int c = tid; c < ncol; c += blockDim.x) {
      const float x = nrm[c];
      if (x >= 0.f) {
        if (better(x, (int)(c0 + c), v1, i1)) {
          v2b = fmaxf(v2b, v1);
          v1 = x;
          i1 = (int)(c0 + c);
        } else {
          v2b = fmaxf(v2b, x);
        }
      }
    }
    float bv = v1, bnd = v2b;  // the block's best and the best of the rest
    int bi = i1;
    block_top2(bv, bi, bnd, red_v, red_i, red_2);
    if (tid == 0) {
      if (bi != 0x7fffffff)
        atomicMax(wkey + nbar % 3, ((unsigned long long)__float_as_uint(bv) << 32) |
                                       (unsigned long long)(0xffffffffu - (unsigned)bi));
      cv1[buf * G + b] = (bi != 0x7fffffff) ? bv : -INFINITY;
      cv2[buf * G + b] = bnd;
      a.cand_idx[buf * G + b] = bi;
    }
    if (bi != 0x7fffffff) {
      const int lc = (int)(bi - c0);
      for (int t = tid; t < s; t += blockDim.x)
        a.cand_col[((size_t)buf * G + b) * a.lds + t] = slab[(size_t)lc * a.s_pad + t];
    }
    // 2. barrier (failure injection: one arrival too many at the barrier that
    //    covers the step a.stall_step)
    const bool stall = a.stall_step >= 0 && j + QRCP_MAXP - 1 >= a.stall_step;
    if (!grid_barrier(bar, (unsigned)((nbar + 1) * G + (stall ? 1 : 0)), a.ctl, a.spin_limit)) return;
    // 3. the winner (one key word) | the largest bound and the candidates above it
    if (tid == 0) {
      const unsigned long long key = *reinterpret_cast<volatile unsigned long long *>(wkey + nbar % 3);
      float wv = -INFINITY;
      int wi = 0x7fffffff;
      if (key != 0ull) {
        wv = __uint_as_float((unsigned)(key >> 32));
        wi = (int)(0xffffffffu - (unsigned)(key & 0xffffffffull));
      }
      // the key of barrier nbar + 2: last read at barrier nbar - 1, next written after barrier nbar + 1
      if (b == 0) wkey[(nbar + 2) % 3] = 0ull;
      if (wi == 0x7fffffff) {
        s_win_blk = -1;  // no finite candidate left (NaN input): record and skip this step
        s_win_col = -1;
        set_status(a.ctl, STATUS_NONFINITE);
      } else {
        s_win_blk = (int)((((int64_t)wi + 1) * G - 1) / a.n);
        s_win_col = wi;
        if (!(wv > 0.f)) set_status(a.ctl, STATUS_RANK_DEFICIENT);
      }
      s_wv = wv;
    } else if (wid == 1) {
      // the whole table in one batch of loads
      float tb1[QRCP_TAB], tb2[QRCP_TAB];
      int tbi[QRCP_TAB];
#pragma unroll
      for (int u = 0; u < QRCP_TAB; ++u) {
        const int g = lane + 32 * u;
        tb1[u] = (g < G) ? __ldcg(cv1 + buf * G + g) : -INFINITY;
        tb2[u] = (g < G) ? __ldcg(cv2 + buf * G + g) : -INFINITY;
        tbi[u] = (g < G) ? __ldcg(a.cand_idx + buf * G + g) : 0x7fffffff;
      }
      float bmax = -INFINITY;
#pragma unroll
      for (int u = 0; u < QRCP_TAB; ++u) bmax = fmaxf(bmax, tb2[u]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) bmax = fmaxf(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
      int cnt = 0;
#pragma unroll
      for (int u = 0; u < QRCP_TAB; ++u) {
        const bool on = tbi[u] != 0x7fffffff && tb1[u] > bmax;
        const unsigned m = __ballot_sync(0xffffffffu, on);
        const int pos = cnt + __popc(m & ((1u << lane) - 1u));
        if (on && pos < QRCP_MAXC) {
          s_cblk[pos] = lane + 32 * u;
          s_cidx[pos] = tbi[u];
        }
        cnt += __popc(m);
      }
      if (lane == 0) {
        s_ncand = cnt;
        s_bound = bmax;
      }
    }
    ++nbar;
    __syncthreads();
    const int wb = s_win_blk, wi = s_win_col, ncand = s_ncand;
    if (wb < 0) {  // uniform across blocks: every block saw the same candidates
      ++j;
      continue;
    }
    const bool try_more = j + 1 < a.k && ncand <= QRCP_MAXC && s_wv > 0.f;
    // 4. winner column | candidate columns (warp w holds candidates w, w + 16,
    //    w + 32 in registers)
    const float *x = a.cand_col + ((size_t)buf * G + wb) * a.lds;
    const float xt = (tid < s) ? __ldcg(x + tid) : 0.f;
    float xc[QRCP_CPW][QRCP_COL];
#pragma unroll
    for (int r = 0; r < QRCP_CPW; ++r) {
      const int q = wid + 16 * r;
      if (try_more && q < ncand && s_cidx[q] != wi) {
        const float *src = a.cand_col + ((size_t)buf * G + s_cblk[q]) * a.lds;
#pragma unroll
        for (int u = 0; u < QRCP_COL; ++u) {
          const int t = lane + 32 * u;
          xc[r][u] = (t < s) ? __ldcg(src + t) : 0.f;
        }
      }
    }
    if (tid == j) {
      // the winner's trailing norm wv = ||x(j:s)||^2 is known, so the
      // reflector needs only alpha = x(j): beta = -sign(alpha) sqrt(wv)
      const float wv = s_wv, alpha = xt;
      float tau = 0.f, beta = alpha;
      if (wv - alpha * alpha > 0.f) {
        const float normx = sqrtf(wv);
        beta = (alpha >= 0.f) ? -normx : normx;
        tau = (beta - alpha) / beta;
      }
      s_tau = tau;
      s_beta = beta;
      s_scal = (tau != 0.f) ? 1.f / (alpha - beta) : 0.f;
      s_tl[0] = tau;
      if (b == 0) a.piv[j] = wi;
      a.sel[wi] = 1;
      s_pair = -1;
    }
    __syncthreads();
    const float tau = s_tau, beta = s_beta;
    if (b == 0 && tid < a.k) a.S11[(size_t)tid * a.k + j] = (tid < j) ? xt : ((tid == j) ? beta : 0.f);
    if (tid < a.s_pad) v[tid] = (tid < j || tid >= s) ? 0.f : ((tid == j) ? 1.f : xt * s_scal);
    if (b == wb && tid == 0) nrm[wi - c0] = -1.f;  // selected
    __syncthreads();
    // 5. further pivots: the candidates above every bound, updated by the
    //    barrier's reflectors so far; the best is certified if it still
    //    exceeds every bound (see the file comment)
    int np = 1;  // pivots of this barrier
    if (try_more) {
      bool live[QRCP_CPW];
#pragma unroll
      for (int r = 0; r < QRCP_CPW; ++r) {
        const int q = wid + 16 * r;
        live[r] = q < ncand && s_cidx[q] != wi;
      }
      for (int p = 1; p < QRCP_MAXP && j + p < a.k; ++p) {
        // candidates <- H_{j+p-1} candidates (kept in registers and in ybuf),
        // their trailing norms over rows > j + p - 1; the warp's (up to)
        // three candidates side by side, so their reductions interleave
        const float *vl = vpt(p - 1);
        const float tl = s_tl[p - 1];
        const int jl = j + p - 1;
        float d[QRCP_CPW], acc[QRCP_CPW];
#pragma unroll
        for (int r = 0; r < QRCP_CPW; ++r) {
          d[r] = 0.f;
          if (live[r])
#pragma unroll
            for (int u = 0; u < QRCP_COL; ++u) {
              const int t = lane + 32 * u;
              d[r] = fmaf((t < a.s_pad) ? vl[t] : 0.f, xc[r][u], d[r]);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
          for (int r = 0; r < QRCP_CPW; ++r) d[r] += __shfl_xor_sync(0xffffffffu, d[r], o);
#pragma unroll
        for (int r = 0; r < QRCP_CPW; ++r) {
          acc[r] = 0.f;
          if (live[r]) {
            float *y = ybuf + (size_t)(wid + 16 * r) * a.s_pad;
            const float dr = d[r] * tl;
#pragma unroll
            for (int u = 0; u < QRCP_COL; ++u) {
              const int t = lane + 32 * u;
              if (t < a.s_pad) {
                const float yt = fmaf(-dr, vl[t], xc[r][u]);
                xc[r][u] = yt;
                y[t] = yt;
                if (t > jl) acc[r] = fmaf(yt, yt, acc[r]);
              }
            }
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
          for (int r = 0; r < QRCP_CPW; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
        if (lane == 0)
#pragma unroll
          for (int r = 0; r < QRCP_CPW; ++r) {
            const int q = wid + 16 * r;
            if (q < ncand) s_cnn[q] = live[r] ? acc[r] : -1.f;
          }
        __syncthreads();
        if (wid == 0) {
          // the best updated norm (ties to the lowest column index), one warp
          float bn = -1.f;
          int bq = -1, bidx = 0x7fffffff;
          for (int q = lane; q < ncand; q += 32) {
            const float nn = s_cnn[q];
            const int ci = s_cidx[q];
            if (nn >= 0.f && (nn > bn || (nn == bn && ci < bidx))) {
              bn = nn;
              bq = q;
              bidx = ci;
            }
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const float on = __shfl_xor_sync(0xffffffffu, bn, o);
            const int oq = __shfl_xor_sync(0xffffffffu, bq, o), oi = __shfl_xor_sync(0xffffffffu, bidx, o);
            if (on > bn || (on == bn && oi < bidx)) {
              bn = on;
              bq = oq;
              bidx = oi;
            }
          }
          if (lane == 0) {
            s_pair = -1;
            // certified: strictly above every bound (so above every column not
            // evaluated, whose norms only shrink under the reflectors), and
            // not zero
            if (bq >= 0 && bn > s_bound && bn > 0.f) {
              const float *y = ybuf + (size_t)bq * a.s_pad;
              const float alpha2 = y[j + p];
              float tau2 = 0.f, beta2 = alpha2;
              if (bn - alpha2 * alpha2 > 0.f) {
                const float nx = sqrtf(bn);
                beta2 = (alpha2 >= 0.f) ? -nx : nx;
                tau2 = (beta2 - alpha2) / beta2;
              }
              s_tl[p] = tau2;
              s_beta = beta2;
              s_scal = (tau2 != 0.f) ? 1.f / (alpha2 - beta2) : 0.f;
              s_pair = bq;
              s_win_col = bidx;
              if (b == 0) a.piv[j + p] = bidx;
              a.sel[bidx] = 1;
            }
          }
        }
        __syncthreads();
        const int pq = s_pair;
        if (pq < 0) break;  // uniform: every block takes the same decision
        {
          const float *y = ybuf + (size_t)pq * a.s_pad;
          const int ci = s_win_col;
          const float yt = (tid < a.s_pad) ? y[tid] : 0.f;
          if (b == 0 && tid < a.k)
            a.S11[(size_t)tid * a.k + j + p] = (tid < j + p) ? yt : ((tid == j + p) ? s_beta : 0.f);
          if (tid < a.s_pad) vpt(p)[tid] = (tid < j + p || tid >= s) ? 0.f : ((tid == j + p) ? 1.f : yt * s_scal);
          if (ci >= c0 && ci < c0 + ncol && tid == 0) nrm[ci - c0] = -1.f;
#pragma unroll
          for (int r = 0; r < QRCP_CPW; ++r)
            if (wid + 16 * r == pq) live[r] = false;
        }
        ++np;
        __syncthreads();
      }
    }
    if (np > 1) {
      // the Gram entries v_i.v_l (l < i) of the barrier's reflectors, one warp each
      constexpr int NPAIR = QRCP_MAXP * (QRCP_MAXP - 1) / 2;
      if (wid < NPAIR) {
        int ii = 1, ll = wid;
        while (ll >= ii) {
          ll -= ii;
          ++ii;
        }
        if (ii < np) {
          float c = 0.f;
          const float *vi = vpt(ii), *vl = vpt(ll);
          for (int t = lane; t < a.s_pad; t += 32) c = fmaf(vi[t], vl[t], c);
          c = warp_sum(c);
          if (lane == 0) s_cc[ii][ll] = c;
        }
      }
      __syncthreads();
      float *vps[QRCP_MAXP];
#pragma unroll
      for (int i = 0; i < QRCP_MAXP; ++i) vps[i] = vpt(i);
      switch (np) {
        case 2:
          apply_reflectors_lanes<2, 2>(slab, a.s_pad, ncol, vps, s_tl, s_cc, j, nrm);
          break;
        case 3:
          apply_reflectors_lanes<3, 2>(slab, a.s_pad, ncol, vps, s_tl, s_cc, j, nrm);
          break;
        default:
          apply_reflectors_lanes<QRCP_MAXP, 2>(slab, a.s_pad, ncol, vps, s_tl, s_cc, j, nrm);
          break;
      }
    } else {
      apply_reflector_lanes<float, 2>(slab, a.s_pad, ncol, v, tau, j, nrm);
    }
    j += np;
    __syncthreads();
  }
  if (b == 0 && tid == 0) a.ctl[CTL_QRCP_BARRIERS] = nbar;
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
    if (lane == 0) nrm[c] = (a.presel && a.presel[c0 + c]) ? T(-1) : acc;  // -1: selected
  }
  __syncthreads();
  if constexpr (sizeof(T) == 4) {
    float *vx = reinterpret_cast<float *>(nrm + a.cols_per_block);
    vx = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(vx) + 15) & ~(uintptr_t)15);
    qrcp_multi_f32(a, slab, v, nrm, vx, c0, ncol);
  } else {

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
}

}  // namespace ffq
