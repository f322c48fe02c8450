// dense_small.cuh -- the thin and k x k dense steps around the three passes:
// gathers, row-wise triangular solves, Cholesky, the SRQR trailing-norm
// estimate and g2 test (Alg. 4), the singular-vector sign rule and the pivot
// output.  All kernels are templated on the working precision T.
#pragma once

#include "common.cuh"
#include "philox.cuh"

namespace ffq {

// ---------------------------------------------------------------------------
// Gathers
// ---------------------------------------------------------------------------
// P (m x ldp) = A(:, piv[0:k]); the pivoted panel of Alg. 2.
template <typename T>
__global__ void gather_cols_kernel(const T *__restrict__ A, int64_t lda, int64_t m, int k,
                                   const int32_t *__restrict__ piv, T *__restrict__ P, int64_t ldp) {
  // a warp per row; lane l copies columns l, l + 32, ... of the row, with the
  // pivot indices held in registers, so each lane has up to 8 independent
  // (scattered) loads in flight
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int j0 = 0; j0 < k; j0 += 256) {
    int pj[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int j = j0 + lane + 32 * u;
      pj[u] = (j < k) ? piv[j] : 0;
    }
    for (int64_t i = w0; i < m; i += nw) {
      const T *a = A + i * lda;
      T v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = j0 + lane + 32 * u;
        if (j < k) v[u] = a[pj[u]];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = j0 + lane + 32 * u;
        if (j < k) P[i * ldp + j] = v[u];
      }
    }
  }
}

// Dst (k x ldd) row l = Src row piv[l] (first `cols` entries).
template <typename T>
__global__ void gather_rows_kernel(const T *__restrict__ Src, int64_t lds, int k, int cols,
                                   const int32_t *__restrict__ piv, T *__restrict__ Dst, int64_t ldd) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * cols; e += gridDim.x * blockDim.x) {
    const int l = e / cols, t = e - l * cols;
    Dst[(int64_t)l * ldd + t] = Src[(int64_t)piv[l] * lds + t];
  }
}

// R11 (k x k) = upper triangle of G(:, J) where G^T = Gt (n x ldg):
// R11(i, j) = Gt[piv[j], i] for i <= j.  Skipped when gate is given and
// *gate == 0 (the device-side swap count: nothing to redo without swaps).
template <typename T>
__global__ void extract_r11_kernel(const T *__restrict__ Gt, int64_t ldg, int k,
                                   const int32_t *__restrict__ piv, T *__restrict__ R11,
                                   const int *gate) {
  if (gate && *gate == 0) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * k; e += gridDim.x * blockDim.x) {
    const int i = e / k, j = e - i * k;
    R11[e] = (i <= j) ? Gt[(int64_t)piv[j] * ldg + i] : T(0);
  }
}

// Make the diagonal of an upper-triangular k x k matrix non-negative by
// flipping rows (left multiplication by a sign matrix).  One warp per row:
// every lane reads the diagonal before any lane writes the row.
template <typename T>
__global__ void posdiag_rows_kernel(T *__restrict__ R, int k) {
  const int lane = threadIdx.x & 31;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < k; i += (gridDim.x * blockDim.x) >> 5) {
    const bool neg = R[(int64_t)i * k + i] < T(0);
    __syncwarp();
    if (neg)
      for (int j = lane; j < k; j += 32) R[(int64_t)i * k + j] = -R[(int64_t)i * k + j];
  }
}

// Dst (rows x cols) = Src^T, Src (cols x rows) with leading dims.
template <typename T>
__global__ void transpose_kernel(const T *__restrict__ Src, int64_t lds, int64_t rows, int64_t cols,
                                 T *__restrict__ Dst, int64_t ldd) {
  __shared__ T tile[32][33];
  const int64_t r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int64_t sr = c0 + yy, sc = r0 + threadIdx.x;  // Src row = dst col
    tile[yy][threadIdx.x] = (sr < cols && sc < rows) ? Src[sr * lds + sc] : T(0);
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int64_t dr = r0 + yy, dc = c0 + threadIdx.x;
    if (dr < rows && dc < cols) Dst[dr * ldd + dc] = tile[threadIdx.x][yy];
  }
}

// ---------------------------------------------------------------------------
// Row-wise triangular solve  Y P = X  (in place on X, M x k, leading dim ldx).
// FWD: P upper triangular (forward substitution over columns 0..k-1).
// !FWD: P lower triangular (backward substitution over columns k-1..0).
// P(i, j) = Pm[i*psi + j*psj] (so P may be the transpose of a stored matrix).
// Each row is solved independently by substitution (multiplying by the
// rounded reciprocal of each pivot), so each row's result is backward stable:
// y (P + dP) = x with |dP| <= gamma_{k+1} |P|.
// A warp solves R rows at a time; lane l owns columns l, l+32, ... (NS slots).
// ---------------------------------------------------------------------------
// The k x k factor of a row solve into shared memory, Ps[j k + c] =
// Pm[j psi + c psj], with its reciprocal diagonal.  Contiguous rows (psj = 1)
// or columns (psi = 1) are read along memory, eight loads in flight a thread,
// so that the copy costs a few memory latencies rather than one per element.
template <typename T>
__device__ __forceinline__ void trsm_load_factor(T *Ps, T *dinv, const T *__restrict__ Pm, int64_t psi,
                                                 int64_t psj, int k) {
  const int n = k * k;
  const bool rows = (psj == 1), cols = (psi == 1);
  for (int e0 = threadIdx.x; e0 < n; e0 += 8 * blockDim.x) {
    T v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e < n) {
        const int a = e / k, b = e - a * k;  // memory order: element b of line a
        if (rows) v[u] = Pm[(int64_t)a * psi + b];
        else if (cols) v[u] = Pm[(int64_t)a * psj + b];
        else v[u] = Pm[(int64_t)a * psi + (int64_t)b * psj];
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e < n) {
        const int a = e / k, b = e - a * k;
        if (cols) Ps[b * k + a] = v[u];  // line a is column a of P
        else Ps[e] = v[u];
      }
    }
  }
  for (int j = threadIdx.x; j < k; j += blockDim.x) dinv[j] = T(1) / Pm[(int64_t)j * psi + (int64_t)j * psj];
}

template <typename T, int NS, int R, bool FWD>
__global__ void __launch_bounds__(512) trsm_rows_kernel(T *__restrict__ X, int64_t ldx, int64_t M,
                                                        int k, const T *__restrict__ Pm,
                                                        int64_t psi, int64_t psj, const int *gate) {
  if (gate && *gate == 0) return;  // gated recomputation (see extract_r11_kernel)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *Ps = reinterpret_cast<T *>(smem_raw);  // k x k, row-major, P(j, c) at Ps[j*k + c]
  T *dinv = Ps + (size_t)k * k;             // 1 / P(j, j)
  trsm_load_factor(Ps, dinv, Pm, psi, psj, k);
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int64_t ngroups = (M + R - 1) / R;
  for (int64_t grp = (int64_t)blockIdx.x * nwarp + wid; grp < ngroups;
       grp += (int64_t)gridDim.x * nwarp) {
    const int64_t r0 = grp * R;
    T x[R][NS];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int sl = 0; sl < NS; ++sl) {
        const int c = lane + 32 * sl;
        x[r][sl] = (r0 + r < M && c < k) ? X[(r0 + r) * ldx + c] : T(0);
      }
    if (FWD) {
#pragma unroll
      for (int jb = 0; jb < NS; ++jb) {
#pragma unroll 1
        for (int ln = 0; ln < 32; ++ln) {
          const int j = jb * 32 + ln;
          if (j >= k) break;
          const T di = dinv[j];
          T yv[R];
#pragma unroll
          for (int r = 0; r < R; ++r) yv[r] = __shfl_sync(0xffffffffu, x[r][jb] * di, ln);
          if (lane == ln) {
#pragma unroll
            for (int r = 0; r < R; ++r) x[r][jb] = yv[r];
          }
#pragma unroll
          for (int sl = jb; sl < NS; ++sl) {
            const int c = lane + 32 * sl;
            const T pc = (c > j && c < k) ? Ps[j * k + c] : T(0);
#pragma unroll
            for (int r = 0; r < R; ++r) x[r][sl] = fma(-yv[r], pc, x[r][sl]);
          }
        }
      }
    } else {
#pragma unroll
      for (int jb = NS - 1; jb >= 0; --jb) {
#pragma unroll 1
        for (int ln = 31; ln >= 0; --ln) {
          const int j = jb * 32 + ln;
          if (j >= k) continue;
          const T di = dinv[j];
          T yv[R];
#pragma unroll
          for (int r = 0; r < R; ++r) yv[r] = __shfl_sync(0xffffffffu, x[r][jb] * di, ln);
          if (lane == ln) {
#pragma unroll
            for (int r = 0; r < R; ++r) x[r][jb] = yv[r];
          }
#pragma unroll
          for (int sl = 0; sl <= jb; ++sl) {
            const int c = lane + 32 * sl;
            const T pc = (c < j) ? Ps[j * k + c] : T(0);
#pragma unroll
            for (int r = 0; r < R; ++r) x[r][sl] = fma(-yv[r], pc, x[r][sl]);
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int sl = 0; sl < NS; ++sl) {
        const int c = lane + 32 * sl;
        if (r0 + r < M && c < k) X[(r0 + r) * ldx + c] = x[r][sl];
      }
  }
}

// Single precision, 2*RP rows per warp held as row pairs, so each update is
// one packed f32x2 FMA for two rows (same arithmetic as trsm_rows_kernel).
template <int NS, int RP, bool FWD>
__global__ void __launch_bounds__(512) trsm_rows2_kernel(float *__restrict__ X, int64_t ldx, int64_t M, int k,
                                                         const float *__restrict__ Pm, int64_t psi, int64_t psj,
                                                         const int *gate) {
  if (gate && *gate == 0) return;  // gated recomputation (see extract_r11_kernel)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *Ps = reinterpret_cast<float *>(smem_raw);  // k x k, row-major, P(j, c) at Ps[j*k + c]
  float *dinv = Ps + (size_t)k * k;                 // 1 / P(j, j)
  trsm_load_factor(Ps, dinv, Pm, psi, psj, k);
  __syncthreads();
  constexpr int R = 2 * RP;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int64_t ngroups = (M + R - 1) / R;
  for (int64_t grp = (int64_t)blockIdx.x * nwarp + wid; grp < ngroups; grp += (int64_t)gridDim.x * nwarp) {
    const int64_t r0 = grp * R;
    float2 x[RP][NS];  // x[rp][sl] = rows (r0 + 2 rp, r0 + 2 rp + 1), column lane + 32 sl
#pragma unroll
    for (int rp = 0; rp < RP; ++rp)
#pragma unroll
      for (int sl = 0; sl < NS; ++sl) {
        const int c = lane + 32 * sl;
        const int64_t ra = r0 + 2 * rp, rb = ra + 1;
        x[rp][sl].x = (ra < M && c < k) ? X[ra * ldx + c] : 0.f;
        x[rp][sl].y = (rb < M && c < k) ? X[rb * ldx + c] : 0.f;
      }
    auto step = [&](int j, int jb, int ln, int slo, int shi) {
      const float di = dinv[j];
      float2 y[RP];
#pragma unroll
      for (int rp = 0; rp < RP; ++rp) {
        y[rp].x = __shfl_sync(0xffffffffu, x[rp][jb].x * di, ln);
        y[rp].y = __shfl_sync(0xffffffffu, x[rp][jb].y * di, ln);
      }
      if (lane == ln) {
#pragma unroll
        for (int rp = 0; rp < RP; ++rp) x[rp][jb] = y[rp];
      }
#pragma unroll
      for (int sl = 0; sl < NS; ++sl) {
        if (sl < slo || sl > shi) continue;
        const int c = lane + 32 * sl;
        const bool on = FWD ? (c > j && c < k) : (c < j);
        const float pc = on ? Ps[j * k + c] : 0.f;
        const float2 p2 = make_float2(pc, pc);
#pragma unroll
        for (int rp = 0; rp < RP; ++rp) x[rp][sl] = __ffma2_rn(make_float2(-y[rp].x, -y[rp].y), p2, x[rp][sl]);
      }
    };
    if (FWD) {
#pragma unroll
      for (int jb = 0; jb < NS; ++jb) {
#pragma unroll 1
        for (int ln = 0; ln < 32; ++ln) {
          const int j = jb * 32 + ln;
          if (j >= k) break;
          step(j, jb, ln, jb, NS - 1);
        }
      }
    } else {
#pragma unroll
      for (int jb = NS - 1; jb >= 0; --jb) {
#pragma unroll 1
        for (int ln = 31; ln >= 0; --ln) {
          const int j = jb * 32 + ln;
          if (j >= k) continue;
          step(j, jb, ln, 0, jb);
        }
      }
    }
#pragma unroll
    for (int rp = 0; rp < RP; ++rp)
#pragma unroll
      for (int sl = 0; sl < NS; ++sl) {
        const int c = lane + 32 * sl;
        const int64_t ra = r0 + 2 * rp, rb = ra + 1;
        if (ra < M && c < k) X[ra * ldx + c] = x[rp][sl].x;
        if (rb < M && c < k) X[rb * ldx + c] = x[rp][sl].y;
      }
  }
}

// ---------------------------------------------------------------------------
// Cholesky  W = R^T R  (one block; W symmetric k x k, only its upper triangle
// is read).  R is written upper triangular (k x k, zero below).  A non-positive
// pivot marks the status RANK_DEFICIENT and continues with a unit pivot.
//
// Blocked right-looking factorisation in shared memory with 8-column steps:
//   1. one thread factors the 8 x 8 diagonal block and inverts its factor,
//      X = R_dd^{-1}, entirely in registers (no shuffles or barriers on the
//      sequential chain of pivots);
//   2. the panel R12 = R_dd^{-T} S12 = X^T S12, one thread per column;
//   3. the symmetric rank-8 update S22 -= R12^T R12 of the upper triangle in
//      4 x 4 register tiles (upper-triangle tiles only).
// The diagonal blocks are at least as well conditioned as R, so multiplying
// by their explicit inverses keeps FP32 accuracy for the Gram matrices this
// library factors.
// ---------------------------------------------------------------------------
constexpr int CHOL_NB = 8;

template <typename T>
__global__ void __launch_bounds__(512, 1) cholesky_kernel(const T *__restrict__ W, int k,
                                                          T *__restrict__ R, int *ctl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *S = reinterpret_cast<T *>(smem_raw);  // k x k, row-major; becomes R in place
  __shared__ T Xs[CHOL_NB][CHOL_NB];         // X = R_dd^{-1}, Xs[j][t] = X(j, t)
  const int tid = threadIdx.x, nthr = blockDim.x;
  const bool vec = (sizeof(T) == 4) && ((k & 3) == 0) && (((uintptr_t)W & 15) == 0) && (((uintptr_t)R & 15) == 0);
  if (vec) {
    const float4 *W4 = reinterpret_cast<const float4 *>(W);
    float4 *S4 = reinterpret_cast<float4 *>(S);
#pragma unroll 4
    for (int e = tid; e < (k * k) >> 2; e += nthr) S4[e] = W4[e];
  } else {
#pragma unroll 4
    for (int e = tid; e < k * k; e += nthr) S[e] = W[e];
  }
  __syncthreads();
  for (int jb = 0; jb < k; jb += CHOL_NB) {
    const int nb = min(CHOL_NB, k - jb);
    // 1. diagonal block (padded with the identity beyond nb)
    if (tid == 0) {
      T a[CHOL_NB][CHOL_NB];
#pragma unroll
      for (int r = 0; r < CHOL_NB; ++r)
#pragma unroll
        for (int c = 0; c < CHOL_NB; ++c)
          a[r][c] = (r <= c && c < nb) ? S[(jb + r) * k + jb + c] : ((r == c) ? T(1) : T(0));
      bool bad = false;
#pragma unroll
      for (int r = 0; r < CHOL_NB; ++r) {
        T d = a[r][r];
        if (!(d > T(0))) {
          bad = true;
          d = T(1);
        }
        const T sd = sqrt(d);
        const T inv = T(1) / sd;
        a[r][r] = sd;
#pragma unroll
        for (int c = r + 1; c < CHOL_NB; ++c) a[r][c] *= inv;
#pragma unroll
        for (int i = r + 1; i < CHOL_NB; ++i)
#pragma unroll
          for (int c = i; c < CHOL_NB; ++c) a[i][c] = fma(-a[r][i], a[r][c], a[i][c]);
      }
      if (bad) set_status(ctl, STATUS_RANK_DEFICIENT);
#pragma unroll
      for (int r = 0; r < CHOL_NB; ++r)
#pragma unroll
        for (int c = r; c < CHOL_NB; ++c)
          if (c < nb) S[(jb + r) * k + jb + c] = a[r][c];
      // X = R_dd^{-1} by back substitution, column by column
      T rinv[CHOL_NB];
#pragma unroll
      for (int r = 0; r < CHOL_NB; ++r) rinv[r] = T(1) / a[r][r];
#pragma unroll
      for (int c = 0; c < CHOL_NB; ++c) {
        T x[CHOL_NB];
#pragma unroll
        for (int r = CHOL_NB - 1; r >= 0; --r) {
          if (r > c) {
            x[r] = T(0);
          } else {
            T acc = (r == c) ? T(1) : T(0);
#pragma unroll
            for (int j = r + 1; j <= c; ++j) acc = fma(-a[r][j], x[j], acc);
            x[r] = acc * rinv[r];
          }
        }
#pragma unroll
        for (int r = 0; r < CHOL_NB; ++r) Xs[r][c] = x[r];
      }
    }
    __syncthreads();
    const int t0 = jb + nb;  // first trailing column
    const int nt = k - t0;
    if (nt <= 0) break;
    // 2. panel R12(t, c) = sum_{j <= t} X(j, t) S12(j, c), one thread per column
    for (int c = t0 + tid; c < k; c += nthr) {
      T sv[CHOL_NB];
#pragma unroll
      for (int j = 0; j < CHOL_NB; ++j) sv[j] = (j < nb) ? S[(jb + j) * k + c] : T(0);
#pragma unroll
      for (int t = 0; t < CHOL_NB; ++t) {
        T acc = T(0);
#pragma unroll
        for (int j = 0; j <= t; ++j) acc = fma(Xs[j][t], sv[j], acc);
        if (t < nb) S[(jb + t) * k + c] = acc;
      }
    }
    __syncthreads();
    // 3. trailing update S(i, c) -= sum_t R(t, i) R(t, c), t0 <= i <= c < k,
    //    over the upper-triangle 4 x 4 tiles (ti <= tc).  e -> (a, b), b <= a,
    //    by the triangular-number inverse, then ti = nt4 - 1 - a, tc = ti + b:
    //    consecutive threads take consecutive column tiles of one tile row,
    //    so their shared-memory rows are contiguous (no bank conflicts).
    //    Entries below the diagonal inside diagonal tiles are updated too;
    //    the lower triangle is never read.
    const int nt4 = (nt + 3) >> 2;
    const int ntiles = nt4 * (nt4 + 1) / 2;
    const bool v4 = (sizeof(T) == 4) && ((k & 3) == 0) && ((t0 & 3) == 0);
    for (int e = tid; e < ntiles; e += nthr) {
      int a = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
      while (a * (a + 1) / 2 > e) --a;
      while ((a + 1) * (a + 2) / 2 <= e) ++a;
      const int ti = nt4 - 1 - a, tc = ti + (e - a * (a + 1) / 2);
      const int i0 = t0 + 4 * ti, c0 = t0 + 4 * tc;
      T acc[4][4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[q][u] = T(0);
#pragma unroll
      for (int t = 0; t < CHOL_NB; ++t) {
        if (t < nb) {
          const T *row = S + (jb + t) * k;
          T av[4], bv[4];
          if (v4) {
            const float4 fa = *reinterpret_cast<const float4 *>(row + i0);
            const float4 fb = *reinterpret_cast<const float4 *>(row + c0);
            av[0] = fa.x; av[1] = fa.y; av[2] = fa.z; av[3] = fa.w;
            bv[0] = fb.x; bv[1] = fb.y; bv[2] = fb.z; bv[3] = fb.w;
          } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              av[q] = (i0 + q < k) ? row[i0 + q] : T(0);
              bv[q] = (c0 + q < k) ? row[c0 + q] : T(0);
            }
          }
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[q][u] = fma(av[q], bv[u], acc[q][u]);
        }
      }
      if (v4) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (i0 + q < k) {
            float4 *p4 = reinterpret_cast<float4 *>(S + (i0 + q) * k + c0);
            float4 v = *p4;
            v.x -= (float)acc[q][0];
            v.y -= (float)acc[q][1];
            v.z -= (float)acc[q][2];
            v.w -= (float)acc[q][3];
            *p4 = v;
          }
        }
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (i0 + q < k && c0 + u < k && c0 + u >= i0 + q) S[(i0 + q) * k + c0 + u] -= acc[q][u];
      }
    }
    __syncthreads();
  }
  if (vec) {
    float4 *R4 = reinterpret_cast<float4 *>(R);
    const float4 *S4 = reinterpret_cast<const float4 *>(S);
    const int k4 = k >> 2;
    for (int e = tid; e < k * k4; e += nthr) {
      const int i = e / k4, c = (e - i * k4) * 4;
      float4 v = S4[e];
      if (c + 0 < i) v.x = 0.f;
      if (c + 1 < i) v.y = 0.f;
      if (c + 2 < i) v.z = 0.f;
      if (c + 3 < i) v.w = 0.f;
      R4[e] = v;
    }
  } else {
    for (int e = tid; e < k * k; e += nthr) {
      const int i = e / k, c = e - i * k;
      R[e] = (c >= i) ? S[e] : T(0);
    }
  }
}

// C (k x k) = A B for upper-triangular A, B (k x k) -- products of triangular
// factors (R2 R1 in CholeskyQR2).
template <typename T>
__global__ void trmm_upper_kernel(const T *__restrict__ Am, const T *__restrict__ Bm, int k,
                                  T *__restrict__ C) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * k; e += gridDim.x * blockDim.x) {
    const int i = e / k, j = e - i * k;
    T acc = T(0);
    for (int l = i; l <= j; ++l) acc = fma(Am[i * k + l], Bm[l * k + j], acc);
    C[e] = (j >= i) ? acc : T(0);
  }
}

// ---------------------------------------------------------------------------
// Alg. 4, trailing-norm estimate:  r_i = ||B(:,i) - B_J Z(:,i)||^2 / (k+p) for
// columns i not in J, where Z = R11^{-1} G (so B - B_J Z is the sample
// B2 - B1 R11^{-1} R12 of A(l+1:m, l+1:n)); CBt = (B_J Z)^T (n x lds).
// Writes r (n; 0 for J) and a per-block argmax (value, index).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) trailing_norms_kernel(const T *__restrict__ Bt,
                                                             const T *__restrict__ CBt, int64_t lds,
                                                             int64_t n, int s, const int *__restrict__ sel,
                                                             T *__restrict__ r, T *__restrict__ blk_v,
                                                             int *__restrict__ blk_i) {
  __shared__ T red_v[32];
  __shared__ int red_i[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  T bv = neg_inf<T>();
  int bi = 0x7fffffff;
  // a warp per column, CPI columns per iteration so that their loads are in
  // flight together
  constexpr int CPI = 4;
  const int64_t stride = (int64_t)gridDim.x * nwarp;
  for (int64_t i0 = (int64_t)blockIdx.x * nwarp + wid; i0 < n; i0 += CPI * stride) {
    T acc[CPI];
#pragma unroll
    for (int q = 0; q < CPI; ++q) acc[q] = T(0);
    for (int t = lane; t < s; t += 32) {
#pragma unroll
      for (int q = 0; q < CPI; ++q) {
        const int64_t i = i0 + q * stride;
        if (i < n) {
          const T d = Bt[i * lds + t] - CBt[i * lds + t];
          acc[q] = fma(d, d, acc[q]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < CPI; ++q) {
      const int64_t i = i0 + q * stride;
      const T a = warp_sum(acc[q]) / T(s);
      if (i < n) {
        const bool inJ = sel[i] != 0;
        if (lane == 0) r[i] = inJ ? T(0) : a;
        if (!inJ && better(a, (int)i, bv, bi)) {
          bv = a;
          bi = (int)i;
        }
      }
    }
  }
  block_argmax(bv, bi, red_v, red_i);
  if (threadIdx.x == 0) {
    blk_v[blockIdx.x] = bv;
    blk_i[blockIdx.x] = bi;
  }
}

// ---------------------------------------------------------------------------
// SRQR one-step QR of the candidate column c (Alg. 4): z = A(:,c) - Q1 a with
// a = G(:,c) = Q1^T A(:,c), then one re-orthogonalisation z -= Q1 (Q1^T z);
// alpha = ||z||.  Three small kernels with block partial sums reduced in a
// fixed order (deterministic).
// ---------------------------------------------------------------------------
// Final argmax over the per-block candidates -> ctl[CTL_CAND]; copies
// a = Gt[c, :] into avec.
template <typename T>
__global__ void srqr_pick_kernel(const T *__restrict__ blk_v, const int *__restrict__ blk_i,
                                 int nblk, const T *__restrict__ Gt, int64_t ldg, int k,
                                 T *__restrict__ avec, int *ctl) {
  __shared__ T red_v[32];
  __shared__ int red_i[32];
  T bv = neg_inf<T>();
  int bi = 0x7fffffff;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
    if (blk_i[b] != 0x7fffffff && better(blk_v[b], blk_i[b], bv, bi)) {
      bv = blk_v[b];
      bi = blk_i[b];
    }
  }
  block_argmax(bv, bi, red_v, red_i);
  if (threadIdx.x == 0) ctl[CTL_CAND] = bi;
  if (bi == 0x7fffffff) return;
  for (int j = threadIdx.x; j < k; j += blockDim.x) avec[j] = Gt[(int64_t)bi * ldg + j];
}

// z_i = A(i, c) - sum_j Q1(i, j) a_j; partial h = Q1^T z per block (per-warp
// partial rows summed in warp order, so the result does not depend on timing).
template <typename T>
__global__ void __launch_bounds__(256) srqr_resid_kernel(const T *__restrict__ A, int64_t lda,
                                                         int64_t m, const T *__restrict__ Q1,
                                                         int64_t ldq, int k, const T *__restrict__ avec,
                                                         const int *ctl, T *__restrict__ z,
                                                         T *__restrict__ hpart) {
  // a warp takes SR_ROWS rows at a time (their loads and warp sums
  // interleave) and keeps its part of h = Q1^T z in registers (k <= 256)
  constexpr int SR_ROWS = 4, NJ = 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nwarp = blockDim.x >> 5;
  T *hw = reinterpret_cast<T *>(smem_raw);  // nwarp x k (the first k entries hold a first)
  const int c = ctl[CTL_CAND];
  if (c == 0x7fffffff) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T as[NJ], hacc[NJ];
#pragma unroll
  for (int u = 0; u < NJ; ++u) {
    const int j = lane + 32 * u;
    as[u] = (j < k) ? avec[j] : T(0);
    hacc[u] = T(0);
  }
  const int64_t rows_per = (m + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * rows_per, i1 = min(m, i0 + rows_per);
  for (int64_t base = i0 + (int64_t)wid * SR_ROWS; base < i1; base += (int64_t)nwarp * SR_ROWS) {
    T q[SR_ROWS][NJ], acc[SR_ROWS], ac[SR_ROWS];
#pragma unroll
    for (int r = 0; r < SR_ROWS; ++r) {
      const int64_t i = base + r;
      acc[r] = T(0);
      ac[r] = (i < i1) ? A[i * lda + c] : T(0);
#pragma unroll
      for (int u = 0; u < NJ; ++u) {
        const int j = lane + 32 * u;
        q[r][u] = (i < i1 && j < k) ? Q1[i * ldq + j] : T(0);
        acc[r] = fma(q[r][u], as[u], acc[r]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int r = 0; r < SR_ROWS; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
#pragma unroll
    for (int r = 0; r < SR_ROWS; ++r) {
      const int64_t i = base + r;
      if (i < i1) {
        const T zi = ac[r] - acc[r];
        if (lane == 0) z[i] = zi;
#pragma unroll
        for (int u = 0; u < NJ; ++u) hacc[u] = fma(q[r][u], zi, hacc[u]);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < NJ; ++u) {
    const int j = lane + 32 * u;
    if (j < k) hw[wid * k + j] = hacc[u];
  }
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    T acc = T(0);
    for (int w = 0; w < nwarp; ++w) acc += hw[w * k + j];
    hpart[(int64_t)blockIdx.x * k + j] = acc;
  }
}

// h = sum over the nhp block partials of srqr_resid_kernel (k entries), in a
// fixed order: one block; G = blockDim / k groups, group g adds the partials
// g, g + G, ... (loads unrolled, so several are in flight), then the groups'
// sums are added in group order.  The reorthogonalisation's blocks then read h
// instead of each reducing all partials on a chain of dependent loads.
template <typename T>
__global__ void __launch_bounds__(1024) srqr_hsum_kernel(const T *__restrict__ hpart, int nhp, int k,
                                                         const int *ctl, T *__restrict__ h) {
  __shared__ T part[1024];
  if (ctl[CTL_CAND] == 0x7fffffff) return;
  const int G = max(1, (int)blockDim.x / k);
  const int t = threadIdx.x, g = t / k, j = t - g * k;
  if (g < G) {
    T acc = T(0);
#pragma unroll 8
    for (int b = g; b < nhp; b += G) acc += hpart[(int64_t)b * k + j];
    part[t] = acc;
  }
  __syncthreads();
  for (int jj = t; jj < k; jj += blockDim.x) {
    T acc = T(0);
    for (int gg = 0; gg < G; ++gg) acc += part[gg * k + jj];
    h[jj] = acc;
  }
}

// z -= Q1 h (h from srqr_hsum_kernel), partial ||z||^2 per block.
template <typename T>
__global__ void __launch_bounds__(256) srqr_reorth_kernel(int64_t m, const T *__restrict__ Q1,
                                                          int64_t ldq, int k, const T *__restrict__ h,
                                                          const int *ctl, T *__restrict__ z,
                                                          T *__restrict__ npart) {
  constexpr int SR_ROWS = 4, NJ = 8;
  __shared__ T red[32];
  if (ctl[CTL_CAND] == 0x7fffffff) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  T hv[NJ];
#pragma unroll
  for (int u = 0; u < NJ; ++u) {
    const int j = lane + 32 * u;
    hv[u] = (j < k) ? h[j] : T(0);
  }
  const int64_t rows_per = (m + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * rows_per, i1 = min(m, i0 + rows_per);
  T nacc = T(0);
  for (int64_t base = i0 + (int64_t)wid * SR_ROWS; base < i1; base += (int64_t)nwarp * SR_ROWS) {
    // all of the rows' loads first (in flight together), then the products
    T q[SR_ROWS][NJ], acc[SR_ROWS], zz[SR_ROWS];
#pragma unroll
    for (int r = 0; r < SR_ROWS; ++r) {
      const int64_t i = base + r;
      zz[r] = (i < i1) ? z[i] : T(0);
#pragma unroll
      for (int u = 0; u < NJ; ++u) {
        const int j = lane + 32 * u;
        q[r][u] = (i < i1 && j < k) ? Q1[i * ldq + j] : T(0);
      }
    }
#pragma unroll
    for (int r = 0; r < SR_ROWS; ++r) {
      acc[r] = T(0);
#pragma unroll
      for (int u = 0; u < NJ; ++u) acc[r] = fma(q[r][u], hv[u], acc[r]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int r = 0; r < SR_ROWS; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
#pragma unroll
    for (int r = 0; r < SR_ROWS; ++r) {
      const int64_t i = base + r;
      if (i < i1) {
        const T zi = zz[r] - acc[r];
        if (lane == 0) {
          z[i] = zi;
          nacc = fma(zi, zi, nacc);
        }
      }
    }
  }
  nacc = block_sum(nacc, red);
  if (threadIdx.x == 0) npart[blockIdx.x] = nacc;
}

// alpha = sqrt(sum npart); g2 = max(1, max_i sqrt(alpha^2 ||e_i^T R11^{-1}||^2 +
// ((R11^{-1} a)_i)^2)) -- the closed form of |alpha| ||Rtilde^{-T}||_{1,2}
// (Sec. 2.2); R11^{-1} a = Zt[c, :].  Rinv = R11^{-1} (k x k).
template <typename T>
__global__ void __launch_bounds__(512) srqr_g2_kernel(const T *__restrict__ npart, int nnp,
                                                       const T *__restrict__ Rinv,
                               int k, const T *__restrict__ Zt, int64_t ldz, double g, int max_swaps,
                               int *ctl, double *dctl, int first) {
  __shared__ T red_v[32];
  __shared__ int red_i[32];
  __shared__ T s_alpha;
  const int c = ctl[CTL_CAND];
  if (c == 0x7fffffff) {
    if (threadIdx.x == 0) {
      dctl[D_G2] = 1.0;
      if (first) dctl[D_G2_FIRST] = 1.0;
      ctl[CTL_NEED_SWAP] = 0;
    }
    return;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  if (wid == 0) {  // alpha^2 = sum of the block partials, lanes in order then a fixed tree
    T acc = T(0);
    for (int b = lane; b < nnp; b += 32) acc += npart[b];
    acc = warp_sum(acc);
    if (lane == 0) s_alpha = sqrt(acc);
  }
  __syncthreads();
  const T alpha = s_alpha;
  T bv = T(1);
  int bi = 0x7fffffff;
  // a warp per row i of R11^{-1} (coalesced loads of its entries j >= i),
  // G2_RPW rows at a time so that their loads are in flight together
  constexpr int G2_RPW = 4;
  for (int i0 = wid; i0 < k; i0 += G2_RPW * nwarp) {
    T rn[G2_RPW];
#pragma unroll
    for (int r = 0; r < G2_RPW; ++r) {
      const int i = i0 + r * nwarp;
      rn[r] = T(0);
#pragma unroll
      for (int u = 0; u < 8; ++u) {  // k <= 256
        const int j = lane + 32 * u;
        const T x = (i < k && j >= i && j < k) ? Rinv[i * k + j] : T(0);
        rn[r] = fma(x, x, rn[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < G2_RPW; ++r) {
      const int i = i0 + r * nwarp;
      const T sq = warp_sum(rn[r]);
      if (i < k) {
        const T u = Zt[(int64_t)c * ldz + i];
        const T val = sqrt(alpha * alpha * sq + u * u);
        if (lane == 0 && better(val, i, bv, bi)) {
          bv = val;
          bi = i;
        }
      }
    }
  }
  block_argmax(bv, bi, red_v, red_i);
  if (threadIdx.x == 0) {
    const double g2 = (double)bv;
    dctl[D_G2] = g2;
    dctl[D_ALPHA] = (double)alpha;
    if (first) {
      dctl[D_G2_FIRST] = g2;
      dctl[D_ALPHA_FIRST] = (double)alpha;
      ctl[CTL_CAND_FIRST] = c;
    }
    ctl[CTL_IMAX] = (bi == 0x7fffffff) ? -1 : bi;
    const int need = (g2 > g) ? 1 : 0;
    ctl[CTL_NEED_SWAP] = (need && ctl[CTL_SWAPS] < max_swaps) ? 1 : 0;
    if (need && ctl[CTL_SWAPS] >= max_swaps) set_status(ctl, STATUS_SWAP_CAP);
  }
}

// ---------------------------------------------------------------------------
// Alg. 4's d-row random estimate of g2 = |alpha| ||Rtilde^{-T}||_{1,2}:
//   g2 ~ |alpha| / sqrt(d) ||Omega_t Rtilde^{-T}||_{1,2},
// Omega_t in N(0,1)^{d x (k+1)} drawn afresh for test t (0: the first test,
// s: the test after the s-th swap); element (r, j) is element (t d + r)(k+1) + j
// of Philox stream G2EST_STREAM under the run's seed.  Column r of
// |alpha| Rtilde^{-1} Omega_t^T is, with Rtilde = [[R11, a], [0, alpha]] and
// alpha >= 0, [R11^{-1} (alpha w_top - a w_k); w_k] (w = row r of Omega_t),
// so one back substitution with R11 per row of Omega_t gives it, also at
// alpha = 0.  The candidate's own column of Rtilde^{-T} is e_{k+1} / alpha,
// whose term is exactly 1; only columns 0..k-1 are estimated, and the
// estimate is max(1, max_i sqrt(sum_r y_r(i)^2 / d)) like the exact form.
// ---------------------------------------------------------------------------
constexpr uint32_t G2EST_STREAM = 1;
constexpr int G2EST_MAX_D = 32;
constexpr int G2EST_YU = 8;  // rows per lane: k <= 256

// Shared memory (elements of T) of g2est_block for depth k.
__host__ __device__ inline int g2est_smem_elems(int k) { return ((k + 31) / 32) * 32 * 33 + k; }

// One block: colsq[i] = sum_r y_r(i)^2 for i < k (rows r in increasing order).
// R11 (k x k, upper, row-major, leading dimension ldr), a (k) and alpha as
// above.  The block's warps take the rows of Omega_t in rounds; R11 is staged
// through shared memory 32 columns at a time (padded to 33) for all warps.
// Returns nonzero (in every thread) if R11 has a zero diagonal entry.
template <typename T>
__device__ int g2est_block(const T *__restrict__ R11, int64_t ldr, const T *a, T alpha, int k, int d,
                           uint64_t seed, int64_t t, T *smem) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int nchunk = (k + 31) / 32;
  T *chunk = smem;                    // (32 nchunk) x 33
  T *colsq = smem + nchunk * 32 * 33;  // k
  __shared__ int s_zero;
  if (threadIdx.x == 0) s_zero = 0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) colsq[i] = T(0);
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x)
    if (R11[(int64_t)i * ldr + i] == T(0)) s_zero = 1;
  for (int r0 = 0; r0 < d; r0 += nwarp) {
    const int r = r0 + wid;
    const bool solver = r < d;
    const uint64_t e0 = (uint64_t)((t * d + r) * (int64_t)(k + 1));
    T y[G2EST_YU];
    const T wk = solver ? gauss_elem<T>(seed, G2EST_STREAM, e0 + (uint64_t)k) : T(0);
#pragma unroll
    for (int u = 0; u < G2EST_YU; ++u) {
      const int row = lane + 32 * u;
      y[u] = (solver && row < k) ? fma(alpha, gauss_elem<T>(seed, G2EST_STREAM, e0 + (uint64_t)row), -a[row] * wk)
                                 : T(0);
    }
#pragma unroll
    for (int ub = G2EST_YU - 1; ub >= 0; --ub) {
      if (ub >= nchunk) continue;
      const int i0 = ub * 32, rows = i0 + 32;
      __syncthreads();  // the previous chunk is consumed
      for (int e = threadIdx.x; e < rows * 32; e += blockDim.x) {
        const int row = e >> 5, col = i0 + (e & 31);
        chunk[row * 33 + (e & 31)] = (col < k && row <= col) ? R11[(int64_t)row * ldr + col] : T(0);
      }
      __syncthreads();
      if (solver) {
        const int top = min(31, k - 1 - i0);
        for (int ii = top; ii >= 0; --ii) {
          const T dg = chunk[(i0 + ii) * 33 + ii];
          const T yv = __shfl_sync(0xffffffffu, y[ub], ii);
          const T yi = (dg != T(0)) ? yv / dg : T(0);
#pragma unroll
          for (int u = 0; u < G2EST_YU; ++u) {
            if (u > ub) continue;
            const int row = lane + 32 * u;
            if (row < i0 + ii) y[u] = fma(-chunk[row * 33 + ii], yi, y[u]);
          }
          if (lane == ii) y[ub] = yi;
        }
      }
    }
    // fixed-order accumulation over the rows of Omega_t
    for (int w = 0; w < nwarp; ++w) {
      if (w == wid && solver) {
#pragma unroll
        for (int u = 0; u < G2EST_YU; ++u) {
          const int row = lane + 32 * u;
          if (row < k) colsq[row] = fma(y[u], y[u], colsq[row]);
        }
      }
      __syncthreads();
    }
  }
  __syncthreads();
  return s_zero;
}

// The first SRQR test with the d-row estimate (one block, 1024 threads,
// dynamic shared memory g2est_smem_elems(k) elements): alpha from the
// residual partial sums, R11 in position order, a = R(0:k, c) = Gt row c.
template <typename T>
__global__ void __launch_bounds__(1024) srqr_g2est_kernel(const T *__restrict__ npart, int nnp,
                                                          const T *__restrict__ R11, int k,
                                                          const T *__restrict__ Gt, int64_t ldg, int d,
                                                          uint64_t seed, double g, int max_swaps, int *ctl,
                                                          double *dctl) {
  extern __shared__ __align__(16) unsigned char g2e_raw[];
  T *sm = reinterpret_cast<T *>(g2e_raw);
  __shared__ T red_v[32];
  __shared__ int red_i[32];
  __shared__ T s_alpha;
  const int c = ctl[CTL_CAND];
  if (c == 0x7fffffff) {
    if (threadIdx.x == 0) {
      dctl[D_G2] = 1.0;
      dctl[D_G2_FIRST] = 1.0;
      ctl[CTL_NEED_SWAP] = 0;
    }
    return;
  }
  if (threadIdx.x < 32) {  // alpha^2 = sum of the block partials (as srqr_g2_kernel)
    T acc = T(0);
    for (int b = threadIdx.x; b < nnp; b += 32) acc += npart[b];
    acc = warp_sum(acc);
    if (threadIdx.x == 0) s_alpha = sqrt(acc);
  }
  __syncthreads();
  const T alpha = s_alpha;
  const int zero = g2est_block<T>(R11, k, Gt + (int64_t)c * ldg, alpha, k, d, seed, 0, sm);
  const T *colsq = sm + ((k + 31) / 32) * 32 * 33;
  T bv = T(1);
  int bi = 0x7fffffff;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const T val = sqrt(colsq[i] / T(d));
    if (better(val, i, bv, bi)) {
      bv = val;
      bi = i;
    }
  }
  block_argmax(bv, bi, red_v, red_i);
  if (threadIdx.x == 0) {
    const double g2 = zero ? 1.0 : (double)bv;
    dctl[D_G2] = g2;
    dctl[D_ALPHA] = (double)alpha;
    dctl[D_G2_FIRST] = g2;
    dctl[D_ALPHA_FIRST] = (double)alpha;
    ctl[CTL_CAND_FIRST] = c;
    ctl[CTL_IMAX] = (zero || bi == 0x7fffffff) ? -1 : bi;
    const int need = (g2 > g && !zero && bi != 0x7fffffff) ? 1 : 0;
    ctl[CTL_NEED_SWAP] = (need && ctl[CTL_SWAPS] < max_swaps) ? 1 : 0;
    if (need && ctl[CTL_SWAPS] >= max_swaps) set_status(ctl, STATUS_SWAP_CAP);
  }
}

// ---------------------------------------------------------------------------
// Output helpers
// ---------------------------------------------------------------------------
// piv[k:n] = columns not in J, ascending (one block, chunked scan).
__global__ void __launch_bounds__(1024) piv_rest_kernel(const int *__restrict__ sel, int64_t n, int k,
                                                        int32_t *__restrict__ piv) {
  // tiles of 8 blockDim.x consecutive columns, eight per thread; a block-wide
  // exclusive scan of the per-thread counts of unselected columns gives each
  // of them its position
  constexpr int E = 8;
  __shared__ int wsum[32];
  __shared__ int s_base;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) s_base = k;
  __syncthreads();
  for (int64_t t0 = 0; t0 < n; t0 += (int64_t)E * blockDim.x) {
    const int64_t i0 = t0 + (int64_t)threadIdx.x * E;
    int f[E], cnt = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      f[e] = (i0 + e < n && sel[i0 + e] == 0) ? 1 : 0;
      cnt += f[e];
    }
    int x = cnt;  // inclusive warp scan of the counts
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
      int z = (lane < nw) ? wsum[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, z, o);
        if (lane >= o) z += y;
      }
      if (lane < nw) wsum[lane] = z;  // inclusive over warps
    }
    __syncthreads();
    const int base = s_base;
    int pos = base + (w > 0 ? wsum[w - 1] : 0) + x - cnt;
#pragma unroll
    for (int e = 0; e < E; ++e)
      if (f[e]) {
        if (pos < n) piv[pos] = (int32_t)(i0 + e);
        ++pos;
      }
    __syncthreads();
    if (threadIdx.x == 0) s_base = base + wsum[nw - 1];
    __syncthreads();
  }
}

// Sign rule, stage 1: for each column j of U (m x k), the row of the
// largest |U(i,j)| in each row chunk (ties -> lowest row).
template <typename T>
__global__ void __launch_bounds__(256) sign_partial_kernel(const T *__restrict__ U, int64_t ldu,
                                                           int64_t m, int k, T *__restrict__ pv,
                                                           int *__restrict__ pi) {
  const int64_t rows_per = (m + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * rows_per, i1 = min(m, i0 + rows_per);
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    T bv = T(-1);
    int bi = 0x7fffffff;
    int64_t i = i0;
    // four rows' loads in flight, compared in row order
    for (; i + 4 <= i1; i += 4) {
      T a[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = fabs(U[(i + u) * ldu + j]);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (a[u] > bv) {
          bv = a[u];
          bi = (int)(i + u);
        }
    }
    for (; i < i1; ++i) {
      const T a = fabs(U[i * ldu + j]);
      if (a > bv) {
        bv = a;
        bi = (int)i;
      }
    }
    pv[(int64_t)blockIdx.x * k + j] = bv;
    pi[(int64_t)blockIdx.x * k + j] = bi;
  }
}

// Stage 2: pick the winning row per column, sgn[j] = sign of U(row, j).
template <typename T>
__global__ void sign_final_kernel(const T *__restrict__ U, int64_t ldu, int k, const T *__restrict__ pv,
                                  const int *__restrict__ pi, int nparts, T *__restrict__ sgn) {
  // a warp per column: lanes scan the parts, then a warp reduction; the
  // winner is the largest value, ties to the lowest row (an order-free rule)
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < k; j += nw) {
    T bv = T(-1);
    int bi = 0x7fffffff;
    for (int b = lane; b < nparts; b += 32) {
      const T v = pv[(int64_t)b * k + j];
      const int i = pi[(int64_t)b * k + j];
      if (i != 0x7fffffff && (v > bv || (v == bv && i < bi))) {
        bv = v;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (oi != 0x7fffffff && (ov > bv || (ov == bv && oi < bi))) {
        bv = ov;
        bi = oi;
      }
    }
    if (lane == 0) sgn[j] = (bi != 0x7fffffff && U[(int64_t)bi * ldu + j] < T(0)) ? T(-1) : T(1);
  }
}

// X(i, j) *= sgn[j]
template <typename T>
__global__ void scale_cols_kernel(T *__restrict__ X, int64_t ldx, int64_t rows, int k,
                                  const T *__restrict__ sgn) {
  // a warp per row, lanes along the row
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < rows; i += nw)
    for (int j = lane; j < k; j += 32) X[i * ldx + j] *= sgn[j];
}

// Copy a rows x cols block between leading dimensions.
template <typename T>
__global__ void copy2d_kernel(const T *__restrict__ Src, int64_t lds, T *__restrict__ Dst, int64_t ldd,
                              int64_t rows, int64_t cols, const int *gate) {
  if (gate && *gate == 0) return;
  // a warp per row, lanes along the row
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < rows; i += nw)
    for (int64_t j = lane; j < cols; j += 32) Dst[i * ldd + j] = Src[i * lds + j];
}

// Control-word defaults: g2 = 1 (no test possible when k = n), no candidate.
__global__ void init_ctl_kernel(int *ctl, double *dctl) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    dctl[D_G2] = 1.0;
    dctl[D_G2_FIRST] = 1.0;
    ctl[CTL_CAND_FIRST] = -1;
    ctl[CTL_CAND] = 0x7fffffff;
  }
}

// Identity (k x k).
template <typename T>
__global__ void eye_kernel(T *__restrict__ X, int k, int64_t ld) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * k; e += gridDim.x * blockDim.x) {
    const int i = e / k, j = e - i * k;
    X[i * ld + j] = (i == j) ? T(1) : T(0);
  }
}

// Non-finite scan of A (sets status NONFINITE).
template <typename T>
__global__ void nonfinite_kernel(const T *__restrict__ A, int64_t lda, int64_t m, int64_t n, int *ctl) {
  const int64_t total = m * n;
  int bad = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e - i * n;
    const T v = A[i * lda + j];
    bad |= !(v - v == T(0));
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) {
    atomicExch(ctl + CTL_NONFINITE, 1);
    set_status(ctl, STATUS_NONFINITE);
  }
}

}  // namespace ffq
