// chol_inv.cuh -- the Cholesky factor of a Gram matrix and its inverse in one
// launch, for the Cholesky-QR sweeps whose product X R^{-1} runs on the
// tensor cores.
//
// W = R^T R = L L^T (k x k, symmetric positive definite; its upper triangle
// is read).  The kernel factors W block column by block column (blocks of
// CI_NB, right-looking) and applies every row operation of the elimination to
// an identity matrix beside it, so that when R is complete the identity has
// become L^{-1} = R^{-T} (elimination on [W | I]).  Per block:
//   A. one warp factors the diagonal block D = L_d L_d^T in registers, lane c
//      holding column c of D and of I beside it (so L_d^{-1} comes with R_d);
//      it runs ahead: as soon as the next diagonal block has been eliminated
//      (the first piece of step C) its warp factors it while the other warps
//      finish step C;
//   B. the block's rows are multiplied by L_d^{-1}: they become rows of R
//      (right of the block) and rows of the partial inverse (left of it);
//   C. the rows below are eliminated with the multipliers R(block, i):
//      S22 -= R12^T R12, and in the inverse, Linv(below, left of and inside
//      the block) -= R12^T (the block's new rows).
// All dot products are at most CI_NB long, so the work of a block spreads
// evenly over the CTA.  Shared memory holds one k x k array: R in the upper
// triangle, the partial L^{-1} in the strict lower triangle, its diagonal in a
// vector beside it.
//
// Outputs: R (k x k, ld k, zeros below the diagonal) and the TF32 head / tail
// of L^{-1} = (R^{-1})^T (k x k, ld ldl, zeros above the diagonal): the
// K-major operand of the product X R^{-1}.  A pivot that is not positive (or
// not finite) is replaced by 1 and sets STATUS_RANK_DEFICIENT, as the
// Cholesky kernel of the FP64 path does.
#pragma once

#include "common.cuh"

namespace ffq {

constexpr int CI_NB = 16;        // block columns (the diagonal block is one warp's)
constexpr int CI_THREADS = 512;  // 16 warps
constexpr int CI_TB = 8;         // block rows per thread in step B
constexpr int CI_RT = 16;        // rows per warp in step C (lanes take 32 consecutive columns)

// Row stride of the shared k x k array (step C reads 16 rows past a tile's
// start, so rows are padded to a multiple of 16).
__host__ __device__ inline int chol_inv_lds(int k) { return (k + 15) & ~15; }

// Shared memory of chol_inv_kernel for k: the k x lds array and the inverse's
// diagonal (the blocks of L_d^{-1} are static).
inline size_t chol_inv_smem(int k) {
  const size_t lds = (size_t)chol_inv_lds(k);
  return ((size_t)k * lds + lds) * sizeof(float);
}

__device__ __forceinline__ float ci_tf32_head(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// Step A for the block at jb (nb <= CI_NB columns), one warp.  Lanes
// 0 .. CI_NB - 1 hold the columns of D (rows r <= c become R_d; the rows below
// are never read), lanes CI_NB .. 2 CI_NB - 1 the columns of I beside it
// (becoming L_d^{-1}): every row operation is the same update of v on all
// lanes.  Each step's scaled row of R_d goes through the warp's row buffer
// (one broadcast read per lane), and a D lane keeps its own diagonal entry in
// dg, so that the next pivot is ready without waiting for that buffer.
// Padding columns c >= nb are unit columns, which the elimination leaves as
// they are.  Writes R_d and L_d^{-1} into S, L_d^{-1} to Ls / LsT (zero
// outside it) and its diagonal to dinv.
__device__ __noinline__ void ci_diag_block(float *S, int lds, int jb, int nb, float (*Ls)[CI_NB],
                                           float (*LsT)[CI_NB], float *dinv, float *rowbuf, int *ctl, int lane) {
  const bool dl = lane < CI_NB;               // a column of D, else of I
  const int c = dl ? lane : lane - CI_NB;     // the column within the block
  float v[CI_NB];
  float dg = 1.f;
  bool bad = false;
#pragma unroll
  for (int r = 0; r < CI_NB; ++r) {
    float x = (r == c) ? 1.f : 0.f;
    if (dl && c < nb && r <= c) x = S[(jb + r) * lds + jb + c];
    v[r] = x;
    if (r == c) dg = x;
  }
#pragma unroll
  for (int r = 0; r < CI_NB; ++r) {
    float piv = __shfl_sync(0xffffffffu, dg, r);
    if (!(piv > 0.f)) {
      bad = true;
      piv = 1.f;
    }
    const float sd = sqrtf(piv), inv = 1.f / sd;
    // row r of [D | I] scaled by 1/sqrt(pivot)
    v[r] = (dl && c == r) ? sd : v[r] * inv;
    if (dl && c > r) dg = fmaf(-v[r], v[r], dg);
    if (r + 1 < CI_NB) {
      // rows i > r minus R(r, i) times row r (in D this also changes the
      // unread entries below the diagonal)
      if (dl) rowbuf[c] = v[r];
      __syncwarp();
      float rr[CI_NB];
#pragma unroll
      for (int q = 0; q < CI_NB / 4; ++q) {
        const float4 x4 = reinterpret_cast<const float4 *>(rowbuf)[q];
        rr[4 * q] = x4.x;
        rr[4 * q + 1] = x4.y;
        rr[4 * q + 2] = x4.z;
        rr[4 * q + 3] = x4.w;
      }
      __syncwarp();
#pragma unroll
      for (int i = 0; i < CI_NB; ++i)  // fixed trip count: unrolled, i > r folds away
        if (i > r) v[i] = fmaf(-rr[i], v[r], v[i]);
    }
  }
  if (bad && lane < nb) set_status(ctl, STATUS_RANK_DEFICIENT);
#pragma unroll
  for (int r = 0; r < CI_NB; ++r) {
    const bool in = (c < nb && r < nb);
    if (dl) {
      if (in && r <= c) S[(jb + r) * lds + jb + c] = v[r];  // R_d on and above the diagonal
    } else {
      if (in && r > c) S[(jb + r) * lds + jb + c] = v[r];   // L_d^{-1} below it
      if (in && r == c) dinv[jb + c] = v[r];
      const float l = (in && r >= c) ? v[r] : 0.f;
      Ls[r][c] = l;
      LsT[c][r] = l;
    }
  }
}

__global__ void __launch_bounds__(CI_THREADS, 1)
    chol_inv_kernel(const float *__restrict__ W, int k, float *__restrict__ R, float *__restrict__ Lh,
                    float *__restrict__ Ll, int64_t ldl, int *ctl, const int *skip) {
  if (skip && *skip) return;  // the factor was already formed by cholqr_series_kernel
  extern __shared__ __align__(16) float ci_smem[];
  // L_d^{-1} of the current and the next block (step A runs one block ahead)
  __shared__ __align__(16) float Ls[2][CI_NB][CI_NB];   // Ls[.][t][u] = L_d^{-1}(t, u), zero above the diagonal
  __shared__ __align__(16) float LsT[2][CI_NB][CI_NB];  // LsT[.][u][t] = Ls[.][t][u]
  __shared__ __align__(16) float rowbuf[CI_NB];          // step A's row broadcast
  const int lds = chol_inv_lds(k);
  float *S = ci_smem;                       // k x lds
  float *dinv = ci_smem + (size_t)k * lds;  // diagonal of L^{-1}
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = CI_THREADS / 32;

  // W's upper triangle; the strict lower triangle (the identity's part) and
  // the padding columns start at zero
  for (int e = tid; e < k * lds; e += CI_THREADS) {
    const int i = e / lds, c = e - i * lds;
    S[e] = (c >= i && c < k) ? W[(size_t)i * k + c] : 0.f;
  }
  __syncthreads();
  if (warp == 0) ci_diag_block(S, lds, 0, min(CI_NB, k), Ls[0], LsT[0], dinv, rowbuf, ctl, lane);
  __syncthreads();

  for (int jb = 0, blk = 0; jb < k; jb += CI_NB, ++blk) {
    const int nb = min(CI_NB, k - jb), t0 = jb + nb, nt = k - t0;
    const int buf = blk & 1;

    // B. the block's rows times L_d^{-1}, every column outside the block:
    //    new(t, col) = sum_{u <= t} L_d^{-1}(t, u) S(jb + u, col); a thread
    //    takes CI_TB rows of one column
    const int ncols = k - nb, ng = (nb + CI_TB - 1) / CI_TB;
    float2 out[CI_TB / 2];
    int my_col = -1, my_g = 0;
    for (int e = tid; e < ng * ncols; e += CI_THREADS) {  // at most one item a thread (k <= 256)
      my_g = e / ncols;
      const int q = e - my_g * ncols;
      my_col = (q < jb) ? q : q + nb;
#pragma unroll
      for (int h = 0; h < CI_TB / 2; ++h) out[h] = make_float2(0.f, 0.f);
      const int umax = min(CI_TB * (my_g + 1), nb);
#pragma unroll
      for (int u = 0; u < CI_NB; ++u) {
        if (u >= umax) break;
        const float sv = S[(jb + u) * lds + my_col];
        const float2 ss = make_float2(sv, sv);
        const float4 *lt = reinterpret_cast<const float4 *>(&LsT[buf][u][CI_TB * my_g]);
#pragma unroll
        for (int q4 = 0; q4 < CI_TB / 4; ++q4) {
          const float4 l4 = lt[q4];
          out[2 * q4] = __ffma2_rn(make_float2(l4.x, l4.y), ss, out[2 * q4]);
          out[2 * q4 + 1] = __ffma2_rn(make_float2(l4.z, l4.w), ss, out[2 * q4 + 1]);
        }
      }
    }
    __syncthreads();
    if (my_col >= 0) {
#pragma unroll
      for (int h = 0; h < CI_TB / 2; ++h) {
        const int t = CI_TB * my_g + 2 * h;
        if (t < nb) S[(jb + t) * lds + my_col] = out[h].x;
        if (t + 1 < nb) S[(jb + t + 1) * lds + my_col] = out[h].y;
      }
    }
    __syncthreads();

    // C. elimination of the rows below the block (nb = CI_NB here).  A warp
    //    takes CI_RT rows (i0 .. i0 + CI_RT - 1 >= t0) and 32 columns, lane l
    //    the column c0 + l: the rows' multipliers R(jb + t, i0 ..) are one
    //    broadcast read for the warp and the columns are consecutive across
    //    lanes, so no access has a bank conflict.  Columns left of t0 are the
    //    inverse's (the block's new rows of L^{-1}; inside the block
    //    L_d^{-1}), columns from the row on are the trailing upper triangle;
    //    pieces with neither are skipped.  Warp 0 takes only the piece that
    //    holds the next diagonal block, then factors that block (step A one
    //    block ahead); warps 1 .. NW - 1 take the other pieces.
    if (nt > 0) {
      const int nrt = (nt + CI_RT - 1) / CI_RT, nch = (k + 31) >> 5;
      const int units = nrt * nch, first = t0 >> 5;  // piece (row tile 0, chunk of t0) first
      for (int e = (warp == 0) ? 0 : warp; e < units; e += (warp == 0) ? units : NW - 1) {
        const int u = (first + e) % units;
        const int ti = u / nch, ch = u - ti * nch;
        const int i0 = t0 + CI_RT * ti, c0 = 32 * ch;
        if (!(c0 < t0 || c0 + 32 > i0) || c0 >= k) continue;  // warp-uniform
        const int j = c0 + lane;
        // the column's operand: the block's new row entries (stride lds),
        // L_d^{-1} inside the block (stride CI_NB), zero past column k
        const bool in_blk = j >= jb && j < t0;
        const float *bp = in_blk ? &Ls[buf][0][j - jb] : S + (size_t)jb * lds + min(j, k - 1);
        const int bs = in_blk ? CI_NB : lds;
        const float bm = (j < k) ? 1.f : 0.f;
        float2 acc[CI_RT / 2];
#pragma unroll
        for (int a2 = 0; a2 < CI_RT / 2; ++a2) acc[a2] = make_float2(0.f, 0.f);
        const float *arow = S + (size_t)jb * lds + i0;
#pragma unroll
        for (int t = 0; t < CI_NB; ++t) {
          const float bv = bp[t * bs] * bm;
          const float2 bb = make_float2(bv, bv);
#pragma unroll
          for (int a4 = 0; a4 < CI_RT / 4; ++a4) {
            const float4 a = *reinterpret_cast<const float4 *>(arow + (size_t)t * lds + 4 * a4);
            acc[2 * a4] = __ffma2_rn(make_float2(a.x, a.y), bb, acc[2 * a4]);
            acc[2 * a4 + 1] = __ffma2_rn(make_float2(a.z, a.w), bb, acc[2 * a4 + 1]);
          }
        }
#pragma unroll
        for (int a2 = 0; a2 < CI_RT / 2; ++a2)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int i = i0 + 2 * a2 + h;
            // the inverse left of t0 (all below row i), the upper triangle
            // from the diagonal on (the lower one is the inverse's)
            if (i < k && (j < t0 || (j >= i && j < k))) S[(size_t)i * lds + j] -= h ? acc[a2].y : acc[a2].x;
          }
      }
      if (warp == 0) {
        __syncwarp();
        ci_diag_block(S, lds, t0, min(CI_NB, nt), Ls[buf ^ 1], LsT[buf ^ 1], dinv, rowbuf, ctl, lane);
      }
    }
    __syncthreads();
  }

  // R (upper triangle) and the split of L^{-1} (lower triangle and diagonal)
  for (int e = tid; e < k * k; e += CI_THREADS) {
    const int i = e / k, c = e - i * k;
    const float sv = S[i * lds + c];
    R[e] = (c >= i) ? sv : 0.f;
    const float l = (c < i) ? sv : ((c == i) ? dinv[i] : 0.f);
    const float h = ci_tf32_head(l);
    Lh[(size_t)i * ldl + c] = h;
    Ll[(size_t)i * ldl + c] = l - h;
  }
}

// The second Cholesky-QR sweep sees W = X1^T X1 = I + E with E small (X1
// is the first sweep's output).  Its factor is then I + U with U = Phi(E)
// (the strict upper triangle of E plus half its diagonal) up to terms of
// order ||E||^2, and M = I - U inverts it to the same order: with Q = X1 M,
// Q^T Q = (I - U)^T (I + E) (I - U) = I + E - U - U^T + O(||E||^2)
// = I + O(||E||^2), since U + U^T = E.  So when ||E||_F <= tol the kernel
// writes R = I + U and the split of M^T (the operand of X1 M) and sets *skip,
// and the exact chol_inv_kernel launched after it returns at once; otherwise
// it leaves both to chol_inv_kernel.  Every CTA computes ||E||_F over all of
// W in the same order (so all take the same decision) and writes its own
// CS_THREADS entries; block 0 records the decision.
// Counters: ctl[CTL_SERIES] / ctl[CTL_SERIES_EXACT] count the sweeps that took
// the expansion / the exact factorization.
constexpr int CS_THREADS = 1024;

inline int cholqr_series_grid(int k) { return (k * k + CS_THREADS - 1) / CS_THREADS; }

__global__ void __launch_bounds__(CS_THREADS, 1)
    cholqr_series_kernel(const float *__restrict__ W, int k, float tol, float *__restrict__ R,
                         float *__restrict__ Lh, float *__restrict__ Ll, int64_t ldl, int *ctl, int *skip) {
  __shared__ float red[CS_THREADS / 32];
  __shared__ int s_use;
  const int tid = threadIdx.x;
  float ss = 0.f;
  for (int e = tid; e < k * k; e += CS_THREADS) {
    const int i = e / k, j = e - i * k;
    const float d = W[e] - ((i == j) ? 1.f : 0.f);
    ss = fmaf(d, d, ss);
  }
  ss = warp_sum(ss);
  if ((tid & 31) == 0) red[tid >> 5] = ss;
  __syncthreads();
  if (tid < 32) {
    float t = red[tid];
    t = warp_sum(t);
    if (tid == 0) {
      const int use = (t <= tol * tol) ? 1 : 0;  // false for a NaN
      s_use = use;
      if (blockIdx.x == 0) {
        *skip = use;
        atomicAdd(ctl + (use ? CTL_SERIES : CTL_SERIES_EXACT), 1);
      }
    }
  }
  __syncthreads();
  if (!s_use) return;
  const int e = blockIdx.x * CS_THREADS + tid;
  if (e < k * k) {
    const int i = e / k, j = e - i * k;
    // U(i, j) for i <= j (upper triangle); W's upper triangle is read
    const float u = (i < j) ? W[e] : ((i == j) ? 0.5f * (W[e] - 1.f) : 0.f);
    R[e] = ((i == j) ? 1.f : 0.f) + u;
    // M^T(i, j) = M(j, i) = delta - U(j, i), nonzero for j <= i
    const float ut = (j < i) ? W[(size_t)j * k + i] : ((i == j) ? 0.5f * (W[e] - 1.f) : 0.f);
    const float mt = ((i == j) ? 1.f : 0.f) - ut;
    const float h = ci_tf32_head(mt);
    Lh[(size_t)i * ldl + j] = h;
    Ll[(size_t)i * ldl + j] = mt - h;
  }
}

}  // namespace ffq
