// tucker.cu -- Tucker approximations of dense tensors (Sec. 3.1) with
// Flip-Flop SRQR (Alg. 9) as the approximate rank-k_r SVD of each unfolding:
// the sequentially truncated HOSVD (Alg. 6) and the HOSVD (Alg. 5).
//
// The tensor is dense, row-major over its modes (the last index fastest).  The
// unfolding G_(r) has the mode-r index as its row and, as its column, the
// row-major linear index of the remaining indices in increasing mode order.
// (The column order of an unfolding only permutes the rows of V; Sec. 3.1
// leaves it open.)
//
// ST-HOSVD, processing step j (r = order[j]):
//   G_(r) is materialised as an m x n row-major matrix (row stride a multiple
//   of 4 elements, so the tensor-core passes can read it with TMA);
//   ffsrqr_run gives U_r, S, V (n x k_r);
//   the core update G_(r) <- diag(S) V^T (Alg. 6) is never stored as such: the
//   permute kernel reads S and V directly when it lays out the next unfolding
//   (or, after the last step, the core tensor in row-major mode order).
// HOSVD: U_r from ffsrqr_run on every unfolding X_(r) of the input, then the
//   core G = X x_1 U_1^T ... x_d U_d^T one mode at a time: G_(r)^T U_r is the
//   plan's pass-2 product (ffq_project), whose n x k_r result has the same
//   layout as V above, so the same permute lays out the next unfolding.
// Everything is enqueued on the caller's stream; nothing synchronises.
#include <cuda_runtime.h>

#include <new>

#include "../../include/ffsrqr.h"

void ffq_set_last_error(const char *what, cudaError_t e);  // ffsrqr.cu
int ffq_project(ffsrqr_plan_t P, const void *A, int64_t lda, const void *X, int64_t ldx, void *Gt, int64_t ldg,
                void *workspace, cudaStream_t st, int *launches);  // ffsrqr.cu

namespace {

constexpr int ST_MAX_D = 8;
constexpr int PERM_TILE = 32;
constexpr int PERM_ROWS = 8;  // tile kernel: block is PERM_TILE x PERM_ROWS threads

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int cuda_fail(const char *what, cudaError_t e) {
  ffq_set_last_error(what, e);
  return FFSRQR_STATUS_CUDA;
}

// A permutation of a strided tensor into a strided output, optionally scaled
// along one axis: dst[sum_t i_t dstr[t]] = src[sum_t i_t sstr[t]] * scale[i_sa].
// Axes are in output order; the last one has output stride 1.
struct PermArgs {
  int nd;
  int u;   // output axis whose input stride is 1 (a transpose through shared memory), or -1
  int sa;  // axis the scale vector runs along, or -1
  int pad;
  int64_t size[ST_MAX_D];
  int64_t sstr[ST_MAX_D];
  int64_t dstr[ST_MAX_D];
  int64_t rows;   // row kernel: product of all sizes but the last
  int64_t batch;  // tile kernel: product of the sizes of the axes other than u and the last
  int64_t tiles_u, tiles_w;
};

// Rows of the output (all indices but the last fixed), read along the last
// axis with its input stride.  Used when the input's unit-stride axis is also
// the output's last axis, so reads and writes are both coalesced.
template <typename T>
__global__ void __launch_bounds__(128) perm_rows_kernel(const T *__restrict__ src, T *__restrict__ dst,
                                                        const T *__restrict__ scale, PermArgs a) {
  const int w = a.nd - 1;
  const int64_t nw = a.size[w], sw = a.sstr[w];
  for (int64_t r = blockIdx.x; r < a.rows; r += gridDim.x) {
    int64_t rem = r, so = 0, dof = 0;
    T c = T(1);
    for (int t = w - 1; t >= 0; --t) {
      const int64_t i = rem % a.size[t];
      rem /= a.size[t];
      so += i * a.sstr[t];
      dof += i * a.dstr[t];
      if (t == a.sa) c = scale[i];
    }
    for (int64_t i = threadIdx.x; i < nw; i += blockDim.x) {
      const T v = src[so + i * sw];
      dst[dof + i] = v * (a.sa == w ? scale[i] : c);
    }
  }
}

// 32 x 32 tiles of the (u, last) plane, loaded along u (unit input stride)
// and stored along the last axis (unit output stride).
template <typename T>
__global__ void __launch_bounds__(PERM_TILE *PERM_ROWS) perm_tile_kernel(const T *__restrict__ src, T *__restrict__ dst,
                                                                        const T *__restrict__ scale, PermArgs a) {
  __shared__ T tile[PERM_TILE][PERM_TILE + 1];
  const int w = a.nd - 1, u = a.u;
  const int64_t nu = a.size[u], nw = a.size[w], su = a.sstr[u], sw = a.sstr[w], du = a.dstr[u];
  const int64_t total = a.batch * a.tiles_u * a.tiles_w;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
    int64_t rem = t;
    const int64_t w0 = (rem % a.tiles_w) * PERM_TILE;
    rem /= a.tiles_w;
    const int64_t u0 = (rem % a.tiles_u) * PERM_TILE;
    rem /= a.tiles_u;
    int64_t so = 0, dof = 0;
    T c = T(1);
    for (int x = w - 1; x >= 0; --x) {
      if (x == u) continue;
      const int64_t i = rem % a.size[x];
      rem /= a.size[x];
      so += i * a.sstr[x];
      dof += i * a.dstr[x];
      if (x == a.sa) c = scale[i];
    }
    __syncthreads();  // the previous tile has been stored
    for (int j = ty; j < PERM_TILE; j += PERM_ROWS) {
      const int64_t iu = u0 + tx, iw = w0 + j;
      if (iu < nu && iw < nw) {
        const T f = a.sa == u ? scale[iu] : (a.sa == w ? scale[iw] : c);
        tile[j][tx] = src[so + iu * su + iw * sw] * f;
      }
    }
    __syncthreads();
    for (int j = ty; j < PERM_TILE; j += PERM_ROWS) {
      const int64_t iu = u0 + j, iw = w0 + tx;
      if (iu < nu && iw < nw) dst[dof + iu * du + iw] = tile[tx][j];
    }
  }
}

// The tensor a step reads from: per mode, its size and its stride in the
// buffer, and the mode (if any) that is scaled by S.
struct View {
  const void *ptr;
  int64_t size[ST_MAX_D];
  int64_t str[ST_MAX_D];
  int scale_mode;
  const void *scale;
};

// Output axes for the unfolding of mode q (q first, then the other modes in
// increasing order; row stride ldo), or for the core (q < 0: every mode in
// order, row-major, no padding).
PermArgs perm_args(const View &v, int d, int q, int64_t ldo) {
  PermArgs a{};
  a.nd = d;
  int order[ST_MAX_D], t = 0;
  if (q >= 0) order[t++] = q;
  for (int x = 0; x < d; ++x)
    if (x != q) order[t++] = x;
  for (int x = 0; x < d; ++x) {
    a.size[x] = v.size[order[x]];
    a.sstr[x] = v.str[order[x]];
  }
  int64_t s = 1;
  for (int x = d - 1; x >= (q >= 0 ? 1 : 0); --x) {
    a.dstr[x] = s;
    s *= a.size[x];
  }
  if (q >= 0) a.dstr[0] = ldo;
  a.sa = -1;
  a.u = -1;
  for (int x = 0; x < d; ++x) {
    if (order[x] == v.scale_mode) a.sa = x;
    if (a.sstr[x] == 1 && a.size[x] > 1 && x != d - 1) a.u = x;
  }
  if (a.sstr[d - 1] == 1 && a.size[d - 1] > 1) a.u = -1;  // already coalesced both ways
  a.rows = 1;
  for (int x = 0; x < d - 1; ++x) a.rows *= a.size[x];
  a.batch = 1;
  for (int x = 0; x < d - 1; ++x)
    if (x != a.u) a.batch *= a.size[x];
  if (a.u >= 0) {
    a.tiles_u = (a.size[a.u] + PERM_TILE - 1) / PERM_TILE;
    a.tiles_w = (a.size[d - 1] + PERM_TILE - 1) / PERM_TILE;
  }
  return a;
}

// The tensor whose mode-r unfolding is diag(scale) Y^T for Y (n x k, leading
// dimension ld, row index = the other modes row-major): mode r has stride 1,
// the other modes the row-major strides of Y's row index times ld.
void set_view_from_rows(View &v, int d, const void *Y, int r, int64_t k, int64_t ld, const void *scale) {
  v.ptr = Y;
  v.scale = scale;
  v.scale_mode = scale ? r : -1;
  v.size[r] = k;
  int64_t s = ld;
  for (int x = d - 1; x >= 0; --x) {
    if (x == r) continue;
    v.str[x] = s;
    s *= v.size[x];
  }
  v.str[r] = 1;
}

void set_view_dense(View &v, int d, const void *X, const int64_t *dims) {
  v.ptr = X;
  v.scale = nullptr;
  v.scale_mode = -1;
  int64_t s = 1;
  for (int x = d - 1; x >= 0; --x) {
    v.size[x] = dims[x];
    v.str[x] = s;
    s *= dims[x];
  }
}

template <typename T>
int launch_perm(const View &v, int d, int q, int64_t ldo, void *dst, cudaStream_t st) {
  const PermArgs a = perm_args(v, d, q, ldo);
  const int64_t cap = 152 * 16;
  if (a.u >= 0) {
    const int64_t work = a.batch * a.tiles_u * a.tiles_w;
    const int grid = (int)(work < cap ? work : cap);
    if (grid == 0) return 0;
    perm_tile_kernel<T><<<grid, dim3(PERM_TILE, PERM_ROWS), 0, st>>>(
        static_cast<const T *>(v.ptr), static_cast<T *>(dst), static_cast<const T *>(v.scale), a);
  } else {
    const int grid = (int)(a.rows < cap ? a.rows : cap);
    if (grid == 0) return 0;
    perm_rows_kernel<T><<<grid, 128, 0, st>>>(static_cast<const T *>(v.ptr), static_cast<T *>(dst),
                                              static_cast<const T *>(v.scale), a);
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : cuda_fail("sthosvd permute", e);
}

}  // namespace

struct Unf {  // one unfolding the run factors or projects
  ffsrqr_plan_t plan = nullptr;
  int mode = 0;
  int64_t m = 0, n = 0, ld = 0;
  bool direct = false;  // the input tensor itself (mode 0, row length a multiple of 4)
};

struct ffsrqr_tucker_s {
  int method = 0, d = 0, p = 0, mode = 0;
  size_t elem = 4;
  int64_t dims[ST_MAX_D] = {};
  int32_t ranks[ST_MAX_D] = {};
  Unf fac[ST_MAX_D];   // factor steps, in processing order
  Unf proj[ST_MAX_D];  // HOSVD: core projections, mode by mode
  size_t off_buf = 0, off_v = 0, off_s = 0, off_piv = 0, total = 0;
  int launches = 0;
};

namespace {

// Adds the plan of one unfolding (m x n, rank k) and grows the buffer sizes.
int add_unf(ffsrqr_tucker_s *t, Unf &u, int r, int64_t m, int64_t n, int k, int p, const ffsrqr_opts_t *opts,
            bool first, size_t &ws, size_t &buf, size_t &vsz, size_t &psz) {
  u.mode = r;
  u.m = m;
  u.n = n;
  u.ld = (n + 3) / 4 * 4;
  u.direct = first && r == 0 && n % 4 == 0;
  size_t w = 0;
  const int rc = ffsrqr_plan(&u.plan, m, n, k, p, t->mode, opts, &w);
  if (rc != 0) return rc < 0 ? -11 : rc;
  if (w > ws) ws = w;
  if (!u.direct && (size_t)m * u.ld * t->elem > buf) buf = (size_t)m * u.ld * t->elem;
  if ((size_t)n * k * t->elem > vsz) vsz = (size_t)n * k * t->elem;
  if ((size_t)n * sizeof(int32_t) > psz) psz = (size_t)n * sizeof(int32_t);
  return 0;
}

}  // namespace

extern "C" {

int ffsrqr_tucker_destroy(ffsrqr_tucker_t t) {
  if (!t) return -1;
  for (int j = 0; j < ST_MAX_D; ++j) {
    if (t->fac[j].plan) ffsrqr_destroy(t->fac[j].plan);
    if (t->proj[j].plan) ffsrqr_destroy(t->proj[j].plan);
  }
  delete t;
  return 0;
}

int ffsrqr_tucker_plan(ffsrqr_tucker_t *out, int32_t method, int32_t d, const int64_t *dims, const int32_t *ranks,
                       const int32_t *order, int32_t p, int32_t mode, const ffsrqr_opts_t *opts,
                       size_t *workspace_bytes) {
  if (!out) return -1;
  *out = nullptr;
  if (method != FFSRQR_TUCKER_STHOSVD && method != FFSRQR_TUCKER_HOSVD) return -2;
  if (d < 2 || d > ST_MAX_D) return -3;
  if (!dims) return -4;
  for (int x = 0; x < d; ++x)
    if (dims[x] < 1) return -4;
  if (!ranks) return -5;
  for (int x = 0; x < d; ++x)
    if (ranks[x] < 1 || ranks[x] > dims[x]) return -5;
  int ord[ST_MAX_D];
  bool seen[ST_MAX_D] = {};
  for (int j = 0; j < d; ++j) {
    ord[j] = (order && method == FFSRQR_TUCKER_STHOSVD) ? order[j] : j;
    if (ord[j] < 0 || ord[j] >= d || seen[ord[j]]) return -6;
    seen[ord[j]] = true;
  }
  if (p < 0) return -7;
  if (mode != FFSRQR_PLAIN_FP32 && mode != FFSRQR_MIXED && mode != FFSRQR_MIXED_BF16X3 && mode != FFSRQR_FP64) return -8;
  if (!workspace_bytes) return -10;
  ffsrqr_tucker_s *t = new (std::nothrow) ffsrqr_tucker_s();
  if (!t) return FFSRQR_STATUS_WORKSPACE;
  t->method = method;
  t->d = d;
  t->p = p;
  t->mode = mode;
  t->elem = mode == FFSRQR_FP64 ? 8 : 4;
  int64_t cur[ST_MAX_D], total = 1;
  for (int x = 0; x < d; ++x) {
    t->dims[x] = dims[x];
    t->ranks[x] = ranks[x];
    cur[x] = dims[x];
    total *= dims[x];
  }
  size_t ws = 0, buf = 0, vsz = 0, psz = 0;
  int rc = 0;
  for (int j = 0; j < d && rc == 0; ++j) {
    const int r = ord[j];
    int64_t n = 1;
    for (int x = 0; x < d; ++x)
      if (x != r) n *= cur[x];
    rc = add_unf(t, t->fac[j], r, cur[r], n, ranks[r], p, opts, j == 0, ws, buf, vsz, psz);
    if (method == FFSRQR_TUCKER_STHOSVD) cur[r] = ranks[r];
  }
  if (method == FFSRQR_TUCKER_HOSVD) {
    // G <- G x_r U_r^T for r = 0 .. d-1 (the pass-2 product; no oversampling)
    for (int r = 0; r < d && rc == 0; ++r) {
      const int64_t n = total / cur[r];
      rc = add_unf(t, t->proj[r], r, cur[r], n, ranks[r], 0, opts, r == 0, ws, buf, vsz, psz);
      total = n * ranks[r];
      cur[r] = ranks[r];
    }
  }
  if (rc != 0) {
    ffsrqr_tucker_destroy(t);
    return rc;
  }
  t->off_buf = align256(ws);
  t->off_v = align256(t->off_buf + buf);
  t->off_s = align256(t->off_v + vsz);
  t->off_piv = align256(t->off_s + ST_MAX_D * 256 * t->elem);
  t->total = align256(t->off_piv + psz);
  *workspace_bytes = t->total;
  *out = t;
  return 0;
}

int ffsrqr_tucker_run(ffsrqr_tucker_t t, const void *X, uint64_t seed, void *const *U, void *const *S, void *core,
                      void *workspace, void *stream, ffsrqr_info_t *infos) {
  if (!t) return -1;
  if (!X) return -2;
  if (!U) return -4;
  for (int x = 0; x < t->d; ++x)
    if (!U[x]) return -4;
  if (!core) return -6;
  if (!workspace || ((uintptr_t)workspace & 255u)) return -7;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  unsigned char *ws = static_cast<unsigned char *>(workspace);
  const int d = t->d;
  const bool f64 = t->mode == FFSRQR_FP64;
  int launches = 0, rc = 0;
  void *buf = ws + t->off_buf;
  void *vbuf = ws + t->off_v;
  int32_t *piv = reinterpret_cast<int32_t *>(ws + t->off_piv);
  View v{}, vx{};
  set_view_dense(vx, d, X, t->dims);
  // the unfolding u of the tensor v, as a matrix (pointer, leading dimension)
  auto unfold = [&](const View &src, const Unf &u, const void **A, int64_t *lda) -> int {
    if (u.direct) {
      *A = X;
      *lda = u.n;
      return 0;
    }
    ++launches;
    *A = buf;
    *lda = u.ld;
    return f64 ? launch_perm<double>(src, d, u.mode, u.ld, buf, st) : launch_perm<float>(src, d, u.mode, u.ld, buf, st);
  };
  v = vx;
  for (int j = 0; j < d; ++j) {
    const Unf &u = t->fac[j];
    const int r = u.mode;
    const int64_t k = t->ranks[r];
    const void *A;
    int64_t lda;
    if ((rc = unfold(t->method == FFSRQR_TUCKER_STHOSVD ? v : vx, u, &A, &lda))) return rc;
    void *s_out = (S && S[r]) ? S[r] : static_cast<void *>(ws + t->off_s + (size_t)r * 256 * t->elem);
    if ((rc = ffsrqr_run(u.plan, A, lda, seed + (uint64_t)j, U[r], k, s_out, vbuf, k, piv, ws, st,
                         infos ? infos + j : nullptr)))
      return rc;
    launches += ffsrqr_launch_count(u.plan);
    // ST-HOSVD: the core becomes the tensor with G_(r) = diag(S) V^T
    if (t->method == FFSRQR_TUCKER_STHOSVD) set_view_from_rows(v, d, vbuf, r, k, k, s_out);
  }
  if (t->method == FFSRQR_TUCKER_HOSVD) {
    v = vx;
    for (int r = 0; r < d; ++r) {
      const Unf &u = t->proj[r];
      const int64_t k = t->ranks[r];
      const void *A;
      int64_t lda;
      if ((rc = unfold(v, u, &A, &lda))) return rc;
      int nl = 0;
      if ((rc = ffq_project(u.plan, A, lda, U[r], k, vbuf, k, ws, st, &nl))) return rc;
      launches += nl;
      set_view_from_rows(v, d, vbuf, r, k, k, nullptr);
    }
  }
  ++launches;
  if ((rc = f64 ? launch_perm<double>(v, d, -1, 0, core, st) : launch_perm<float>(v, d, -1, 0, core, st)))
    return rc;
  t->launches = launches;
  return 0;
}

int ffsrqr_tucker_launch_count(ffsrqr_tucker_t t) {
  if (!t) return -1;
  return t->launches;
}

}  // extern "C"
