// ffsrqr.cu -- plan, workspace layout, pipeline and C ABI of the Flip-Flop SRQR
// library (Feng, Xiao & Gu, arXiv 1803.01982, Alg. 9 with Alg. 4 and Alg. 2).
//
// Pipeline of ffsrqr_run (every step is a kernel of this library):
//   a1  Omega = Philox/Box-Muller (s x m), s = k + p             (Alg. 2)
//   a2  B^T = A^T Omega^T                                       pass 1 over A
//   a3  partial QRCP of B, k steps -> piv[0:k], S11              (Alg. 1 on B)
//   a4  panel A(:, J): Y = A_J S11^{-1}; CholeskyQR2(Y) -> Q1     (Alg. 2 QR)
//   a5  G^T = A^T Q1  (= (R11 R12)^T, original column order)    pass 2 over A
//   a6  R11 = triu(G(:, J)); Z^T = G^T R11^{-T}; trailing-norm estimate
//       r_i = ||B(:,i) - B_J Z(:,i)||^2 / s; candidate c; alpha; g2  (Alg. 4)
//   a7  swap loop while g2 > g (Alg. 4)                         [srqr_swap.cuh]
//   a8  V' = orth(Z^T) = Pi Qhat1 up to a k x k rotation         (Alg. 9)
//   a9  tmp = A V'                                               pass 3 over A
//   a10 Y_t = tmp (R11 R_z^T)^{-1}; CholeskyQR2(Y_t) -> Q_t, R_t;
//       M_t = R_t R11 R_z^T (tmp = Q_t M_t); Jacobi SVD of M_t   (Alg. 9)
//   a11 U = Q_t U_s, V = V' V_s, sign rule                       (Alg. 9)
// The thin QR factorisations are preconditioned Cholesky-QR: each tall matrix
// is first multiplied by the inverse of a triangular factor that makes it
// well conditioned (the sketch's R factor S11 for the panel, R11 for G^T, and
// R11 R_z^T for tmp), so two Cholesky-QR sweeps in FP32 give an orthonormal
// basis of the same column space as Householder QR.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/ffsrqr.h"
#include "common.cuh"
#include "chol_inv.cuh"
#include "dense_small.cuh"
#include "gemm_simt.cuh"
#include "jacobi.cuh"
#include "jacobi_blk.cuh"
#include "philox.cuh"
#include "qrcp.cuh"
#include "srqr_swap.cuh"
#include "tc_gemm.cuh"

#include <cudaTypedefs.h>

using namespace ffq;

namespace {

thread_local std::string g_last_cuda_error;

bool cuda_ok(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return true;
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  g_last_cuda_error = buf;
  return false;
}

#define CK(call)                                    \
  do {                                              \
    if (!cuda_ok((call), #call)) return FFSRQR_STATUS_CUDA; \
  } while (0)

// Kernel launches enqueued by the current ffsrqr_run on this thread.
thread_local int g_launches = 0;

#define CKL(what)                                             \
  do {                                                        \
    ++g_launches;                                             \
    if (!cuda_ok(cudaGetLastError(), what)) return FFSRQR_STATUS_CUDA; \
  } while (0)

struct Item {
  size_t off = 0;
  int64_t rows = 0, cols = 0, ld = 0;
  int elem = 0;
};

}  // namespace

// The two mixed modes run the passes on the tensor cores.
inline bool tc_mode(int mode) { return mode == FFSRQR_MIXED_TF32X3 || mode == FFSRQR_MIXED_BF16X3; }

// Shared with the batch and server translation units (not part of the C ABI).
void ffq_set_last_error(const char *what, cudaError_t e) { cuda_ok(e, what); }

struct ffsrqr_plan_s {
  int64_t m, n;
  int k, p, s, mode;
  int kout;                       // rank returned (Alg. 9's k); k above is the SRQR depth l >= kout
  int rsi_q;                      // >= 0: the plan runs randomized subspace iteration with q iterations
  size_t off_uo, off_so, off_vo;  // l > kout: the depth-l U, S, V before truncation
  double g;
  int max_swaps, flags;
  int device, num_sms;
  int elem;  // bytes per element of the working precision
  int64_t ldm, ldn, lds, ldk;
  // workspace items
  size_t ws_bytes;
  size_t off_ctl, off_dctl, off_info, off_om, off_bt, off_sel, off_s11, off_cval, off_cidx, off_ccol;
  size_t off_q1, off_w, off_rc1, off_rc2, off_gt, off_r11, off_rinv, off_zt, off_bjt, off_cbt,
      off_r, off_bv, off_bi, off_avec, off_z, off_hpart, off_npart, off_vp, off_rz, off_tmp,
      off_yt, off_rt, off_t1, off_mt, off_us, off_vs, off_qv, off_qg, off_part, off_sgnv, off_sgni, off_sgn;
  size_t off_tcpart, off_tt, off_bh, off_bl;  // tensor-core passes (the mixed modes)
  size_t off_omb;                             // BF16 copy of Omega (FFSRQR_MIXED_BF16X3)
  size_t off_sinv, off_sh, off_sl, off_scr;   // tensor-core small products (FFSRQR_MIXED)
  int jac_cluster, jac_lpp;                   // blocks of the Jacobi cluster, lanes per pair
  cudaStream_t side = nullptr;                // forms Q of the small QR while the Jacobi runs
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  size_t off_rowk, off_qk, off_rot, off_rd, off_xinv, off_swpart, off_swbv, off_swbi;  // swap loop
  int swap_grid;
  size_t swap_smem;
  int g2_rows = 0;  // 0: exact g2; d >= 1: Alg. 4's d-row random estimate
  int blk = 0;      // TRQRCP block size b (Alg. 2); b = k: one block
  size_t part_cap;  // elements of the split-K buffer
  int qrcp_grid, qrcp_threads;
  int smem_optin;  // max dynamic shared memory per block (bytes)
  size_t qrcp_smem;
  int qrcp_cols, qrcp_spad;
  int nblk_tn;  // blocks of the trailing-norm kernel
  int nblk_res; // blocks of the SRQR residual kernels
  int nblk_sign;
  Item items[10];
  // phase events (FFSRQR_FLAG_PHASE_TIMES), two sets used by alternate runs
  // so that a run's times can be read while the next run executes
  cudaEvent_t ev[2][13];
  cudaEvent_t ev_tc[2][3][2];  // around each tensor-core pass kernel
  int evset;                   // set of the current / last run
  // tensor-core launch configuration per call site (0: the default), set by
  // ffsrqr_plan_tune: sites 0-2 the passes over A (pipeline depth), site 3
  // the Grams of the Cholesky-QR sweeps (stream-K grid)
  int tc_stages[4] = {0, 0, 0, 0};
  int tc_grid[4] = {0, 0, 0, 0};
  int tc_sk[4] = {0, 0, 0, 0};  // 1: all stream-K (no data-parallel tiles first)
  mutable int tc_stages_fit[4] = {0, 0, 0, 0};  // stages the shared memory holds (recorded by launch_tc)
  long long runs;
  int launches;        // kernel launches of the last run
  bool ev_ok;
};

#define MARK(i)                                                          \
  do {                                                                   \
    if (P->ev_ok) cuda_ok(cudaEventRecord(P->ev[P->evset][(i)], st), "event"); \
  } while (0)

namespace {

// Dynamic shared memory of srqr_swap_kernel: carry (k + 1), a, h (k each)
// and the per-warp rows (16 k), which the d-row g2 estimate reuses for its
// staged R11 columns and column sums.
size_t swap_smem_bytes(int k, int g2_rows, size_t elem) {
  const size_t tail = (size_t)(g2_rows > 0 ? std::max(16 * k, g2est_smem_elems(k)) : 16 * k);
  return ((size_t)(3 * k + 1) + tail) * elem;
}

constexpr long long kSpinLimit = 2000000;  // ~1 s of polling (each poll is an L2 round trip + 20 ns sleep)
// Largest ||X1^T X1 - I||_F for which the second Cholesky-QR sweep uses the
// first-order expansion of its factor: the dropped terms leave
// ||Q^T Q - I|| <= 3 ||E||^2 <= 3e-6.
constexpr float kSeriesTol = 1e-3f;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

template <typename T>
int launch_gemm(cudaStream_t st, const ffsrqr_plan_s *P, unsigned char *ws, int M, int N, int K,
                const T *X, int64_t ldx, bool XM, const T *Y, int64_t ldy, bool YN, T *C,
                int64_t ldc, T alpha = T(1), T beta = T(0)) {
  if (M <= 0 || N <= 0) return 0;
  T *part = reinterpret_cast<T *>(ws + P->off_part);
  const bool wide = N > 64;
  // small products (k x k factors): 32 x 32 tiles so that more blocks run
  const bool small = cdiv(M, 64) * cdiv(N, 64) < P->num_sms / 2 && K < 512;
  const int BM = small ? 32 : 64, BN = small ? 32 : (wide ? 128 : 64);
  const int64_t tiles = cdiv(M, BM) * cdiv(N, BN);
  int splits = 1;
  if (small && K >= 128 && K < 512) {
    // a k x k product: four K slices, so that four times the blocks run
    // (each a quarter of the dependent loads) and one reduction adds them
    splits = (int)std::min<int64_t>(4, (int64_t)P->part_cap / ((int64_t)M * N));
    if (splits < 1) splits = 1;
  } else if (tiles < 2 * P->num_sms && K >= 512) {
    splits = (int)cdiv(2 * P->num_sms, tiles);
    splits = (int)std::min<int64_t>(splits, K / 256);
    const int64_t cap = (int64_t)P->part_cap / ((int64_t)M * N);
    splits = (int)std::min<int64_t>(splits, cap);
    if (splits < 1) splits = 1;
  }
  const int klen = (int)round_up(cdiv(K, splits), 16);
  splits = (int)cdiv(K, klen);
  dim3 grid((unsigned)cdiv(M, BM), (unsigned)cdiv(N, BN), (unsigned)splits);
#define GEMM_CASE(XMv, YNv)                                                                        \
  if (XM == XMv && YN == YNv) {                                                                    \
    if (small)                                                                                     \
      gemm_simt_kernel<T, 32, 32, 16, 2, 2, XMv, YNv>                                              \
          <<<grid, 256, 0, st>>>(M, N, K, X, ldx, Y, ldy, C, ldc, klen, part, alpha, beta);        \
    else if (wide)                                                                                 \
      gemm_simt_kernel<T, 64, 128, 8, 4, 8, XMv, YNv>                                              \
          <<<grid, 256, 0, st>>>(M, N, K, X, ldx, Y, ldy, C, ldc, klen, part, alpha, beta);        \
    else                                                                                           \
      gemm_simt_kernel<T, 64, 64, 16, 4, 4, XMv, YNv>                                              \
          <<<grid, 256, 0, st>>>(M, N, K, X, ldx, Y, ldy, C, ldc, klen, part, alpha, beta);        \
  }
  GEMM_CASE(true, true)
  GEMM_CASE(true, false)
  GEMM_CASE(false, true)
  GEMM_CASE(false, false)
#undef GEMM_CASE
  CKL("gemm_simt");
  if (splits > 1) {
    const int64_t total = (int64_t)M * N;
    splitk_reduce_kernel<T><<<(unsigned)std::min<int64_t>(cdiv(total, 256), 4 * P->num_sms), 256, 0, st>>>(
        M, N, splits, part, C, ldc, alpha, beta);
    CKL("splitk_reduce");
  }
  return 0;
}

// ---------------------------------------------------------------------------
// Tensor-core passes
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void *p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 2-D tensor map over a row-major (outer x inner) array of FP32 (or BF16,
// bf = true) with leading dimension ld (elements), box (box_inner x
// box_outer), 64B/128B swizzle by the box row's bytes.
bool make_map(CUtensorMap *map, const void *ptr, int64_t inner, int64_t outer, int64_t ld,
              int box_inner, int box_outer, bool bf = false) {
  auto fn = encode_fn();
  if (!fn) {
    g_last_cuda_error = "cuTensorMapEncodeTiled entry point unavailable";
    return false;
  }
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  const int el = bf ? 2 : 4;
  cuuint64_t strides[1] = {(cuuint64_t)ld * el};
  cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapSwizzle swz =
      (box_inner * el == 128) ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  CUresult r = fn(map, bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                  const_cast<void *>(ptr), dims, strides, box,
                  estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    char buf[128];
    snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    g_last_cuda_error = buf;
    return false;
  }
  return true;
}


// D (M x N) = sum_k Aop(m,k) Bop(k,n) on the tensor cores (see tc_gemm.cuh).
// A: the big matrix (row-major, lda), A_MN selects the contraction over its
// rows (passes 1, 2) or its columns (pass 3).  Bt / Btl: thin operand (and its
// TF32 tail for nprod = 3) stored N x K row-major with leading dim ldb.
// pass 0..2 records the pass-kernel events; -1 for the other products.
// bf: BF16 operands (Bt / Btl are BF16 arrays, A is converted on chip).
int launch_tc(cudaStream_t st, const ffsrqr_plan_s *P, unsigned char *ws, int pass, int nprod, bool a_mn, int M,
              int N, int K, const float *A, int64_t lda, const void *Bt, const void *Btl, int64_t ldb,
              float *C, int64_t ldc, bool bf = false) {
  const int BK = (nprod == 1 || bf) ? 32 : 16;
  const int ntile = (int)round_up(N, 16);
  if (ntile > TC_MAX_NT) return FFSRQR_STATUS_UNSUPPORTED;
  CUtensorMap mA, mB, mBl;
  if (a_mn) {
    // A^T tile: inner = A's column index (M), outer = A's row index (K)
    if (!make_map(&mA, A, M, K, lda, 32, BK)) return FFSRQR_STATUS_CUDA;
  } else {
    if (!make_map(&mA, A, K, M, lda, BK, TC_BM)) return FFSRQR_STATUS_CUDA;
  }
  if (!make_map(&mB, Bt, K, N, ldb, BK, ntile, bf)) return FFSRQR_STATUS_CUDA;
  if (!make_map(&mBl, Btl ? Btl : Bt, K, N, ldb, BK, ntile, bf)) return FFSRQR_STATUS_CUDA;
  TcSched sc;
  sc.M = M;
  sc.N = N;
  sc.K = K;
  sc.KB = (int)cdiv(K, BK);
  sc.tiles = (int)cdiv(M, TC_BM);
  sc.U = (long long)sc.tiles * sc.KB;
  sc.G = (int)std::min<long long>(std::min(P->num_sms, TC_MAX_GRID), sc.U);
  sc.ntile = ntile;
  sc.ldc = ldc;
  sc.C = C;
  sc.part = reinterpret_cast<float *>(ws + P->off_tcpart);
  sc.ctl = reinterpret_cast<int *>(ws + P->off_ctl);
  sc.vec4 = ((uintptr_t)C % 16 == 0) && (ldc % 4 == 0);
  // short K (a tall matrix times a k x k factor): whole tiles per block,
  // written directly, no fixup; the extra tile some blocks take costs less
  // than the partials and their fixup
  sc.whole_tiles = (sc.KB <= 64) ? 1 : 0;
  if (sc.whole_tiles) sc.G = std::min(sc.G, sc.tiles);
  const int site = (pass >= 0) ? pass : ((!sc.whole_tiles && a_mn) ? 3 : -1);
  if (site >= 0 && P->tc_grid[site] > 0) sc.G = std::min(sc.G, P->tc_grid[site]);
  // data-parallel whole tiles first (a multiple of G), stream-K on the rest,
  // when the rest gives every block at least one unit (else all stream-K)
  sc.dpt = 0;
  if (!sc.whole_tiles && sc.tiles >= sc.G && !(site >= 0 && P->tc_sk[site])) {
    const int rest = sc.tiles % sc.G;
    if (rest == 0 || (long long)rest * sc.KB >= sc.G) sc.dpt = sc.tiles - rest;
  }
  // few stream-K tiles shared by many blocks (a Gram): one row per fixup block
  sc.fix_rows = (8LL * (sc.tiles - sc.dpt) < sc.G) ? 1 : 4;
  int stage_bytes = 0;
  if (bf && nprod == 1 && a_mn) stage_bytes = TcStage<32, 1, true, true>::bytes(ntile);
  else if (bf && nprod == 3 && a_mn) stage_bytes = TcStage<32, 3, true, true>::bytes(ntile);
  else if (bf && nprod == 3) stage_bytes = TcStage<32, 3, false, true>::bytes(ntile);
  else if (nprod == 1 && a_mn) stage_bytes = TcStage<32, 1, true>::bytes(ntile);
  else if (nprod == 3 && a_mn) stage_bytes = TcStage<16, 3, true>::bytes(ntile);
  else stage_bytes = TcStage<16, 3, false>::bytes(ntile);
  const int budget = P->smem_optin - 2048;  // static shared memory and alignment slack
  sc.stages = std::min(TC_MAX_STAGES, budget / stage_bytes);
  if (site >= 0) P->tc_stages_fit[site] = sc.stages;
  if (site >= 0 && P->tc_stages[site] > 0) sc.stages = std::min(sc.stages, P->tc_stages[site]);
  if (sc.stages < 2) return FFSRQR_STATUS_UNSUPPORTED;
  const size_t smem = (size_t)sc.stages * stage_bytes + 1024;
#define TC_LAUNCH(BKv, NPv, AMNv, BFv)                                                               \
  {                                                                                                  \
    auto fn = tc_gemm_kernel<BKv, NPv, AMNv, BFv>;                                                   \
    CK(smem_cap_max((const void *)fn));                                                               \
    if (P->ev_ok && pass >= 0) cudaEventRecord(P->ev_tc[P->evset][pass][0], st);                     \
    fn<<<sc.G, TC_THREADS, smem, st>>>(mA, mB, mBl, sc);                                             \
    if (P->ev_ok && pass >= 0) cudaEventRecord(P->ev_tc[P->evset][pass][1], st);                     \
  }
  if (bf && nprod == 1 && a_mn) TC_LAUNCH(32, 1, true, true)
  else if (bf && nprod == 3 && a_mn) TC_LAUNCH(32, 3, true, true)
  else if (bf && nprod == 3 && !a_mn) TC_LAUNCH(32, 3, false, true)
  else if (!bf && nprod == 1 && a_mn) TC_LAUNCH(32, 1, true, false)
  else if (!bf && nprod == 3 && a_mn) TC_LAUNCH(16, 3, true, false)
  else if (!bf && nprod == 3 && !a_mn) TC_LAUNCH(16, 3, false, false)
  else return FFSRQR_STATUS_UNSUPPORTED;
#undef TC_LAUNCH
  CKL("tc_gemm");
  if (!sc.whole_tiles && sc.dpt < sc.tiles) {
    tc_fixup_kernel<<<dim3(sc.tiles - sc.dpt, TC_BM / sc.fix_rows), 256, 0, st>>>(sc);
    CKL("tc_fixup");
  }
  return 0;
}

// Whether the tensor-core passes can address A with TMA (16-byte aligned base
// and row stride); otherwise the CUDA-core passes are used.
bool tc_ok(const void *A, int64_t lda) {
  return ((uintptr_t)A % 16 == 0) && (lda % 4 == 0);
}

template <typename T, bool FWD>
int launch_trsm(cudaStream_t st, const ffsrqr_plan_s *P, T *X, int64_t ldx, int64_t M, const T *Pm,
                int64_t psi, int64_t psj, const int *gate = nullptr) {
  const int k = P->k;
  const size_t smem = (size_t)k * (k + 1) * sizeof(T);
  const int threads = 512;
  // rows per warp: many rows -> 8 (FP32) / 4 (FP64) for reuse of each pivot
  // row; few rows (a k x k inverse) -> 1, to spread them over more warps
  // FP32 many rows: 10 rows per warp as 5 packed row pairs, so that one wave of
  // warps (num_sms x 16) covers 20000 rows without a second round
  const bool few = M < 4096;
  const bool packed = !few && sizeof(T) == 4;
  const int rr = few ? 1 : (packed ? 10 : 4);
  const int64_t groups = cdiv(M, rr);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(groups, threads / 32), P->num_sms));
  const int ns = (int)cdiv(k, 32);
#define TRSM_CASE(NSv)                                                                                 \
  if (ns <= NSv) {                                                                                     \
    if constexpr (sizeof(T) == 4) {                                                                    \
      if (packed) {                                                                                    \
        auto fn2 = trsm_rows2_kernel<NSv, 5, FWD>;                                                     \
        CK(smem_cap_max((const void *)fn2));                                                            \
        fn2<<<grid, threads, smem, st>>>((float *)X, ldx, M, k, (const float *)Pm, psi, psj, gate);    \
        CKL("trsm_rows2");                                                                             \
        return 0;                                                                                      \
      }                                                                                                \
    }                                                                                                  \
    auto fn = few ? trsm_rows_kernel<T, NSv, 1, FWD> : trsm_rows_kernel<T, NSv, 4, FWD>;               \
    CK(smem_cap_max((const void *)fn));                                                                 \
    fn<<<grid, threads, smem, st>>>(X, ldx, M, k, Pm, psi, psj, gate);                                 \
    CKL("trsm_rows");                                                                                  \
    return 0;                                                                                          \
  }
  TRSM_CASE(1)
  TRSM_CASE(2)
  TRSM_CASE(4)
  TRSM_CASE(7)
#undef TRSM_CASE
  return FFSRQR_STATUS_UNSUPPORTED;
}

template <typename T>
int launch_chol(cudaStream_t st, const ffsrqr_plan_s *P, const T *W, T *R, int *ctl) {
  const int k = P->k;
  const size_t smem = (size_t)k * k * sizeof(T);
  CK(smem_cap_max((const void *)cholesky_kernel<T>));
  cholesky_kernel<T><<<1, 512, smem, st>>>(W, k, R, ctl);
  CKL("cholesky");
  return 0;
}

// CholeskyQR2 on X (M x k, ldx) in place: X <- orthonormal Q, Rout = R2 R1.
template <typename T>
int cholqr2(cudaStream_t st, const ffsrqr_plan_s *P, unsigned char *ws, T *X, int64_t ldx, int64_t M,
            T *Rout) {
  const int k = P->k;
  T *W = reinterpret_cast<T *>(ws + P->off_w);
  T *R1 = reinterpret_cast<T *>(ws + P->off_rc1);
  T *R2 = reinterpret_cast<T *>(ws + P->off_rc2);
  int *ctl = reinterpret_cast<int *>(ws + P->off_ctl);
  int rc;
  if ((rc = launch_gemm<T>(st, P, ws, k, k, (int)M, X, ldx, true, X, ldx, true, W, k))) return rc;
  if ((rc = launch_chol<T>(st, P, W, R1, ctl))) return rc;
  if ((rc = launch_trsm<T, true>(st, P, X, ldx, M, R1, k, 1))) return rc;
  if ((rc = launch_gemm<T>(st, P, ws, k, k, (int)M, X, ldx, true, X, ldx, true, W, k))) return rc;
  if ((rc = launch_chol<T>(st, P, W, R2, ctl))) return rc;
  if ((rc = launch_trsm<T, true>(st, P, X, ldx, M, R2, k, 1))) return rc;
  if (Rout) {
    trmm_upper_kernel<T><<<(unsigned)cdiv((int64_t)k * k, 256), 256, 0, st>>>(R2, R1, k, Rout);
    CKL("trmm_upper");
  }
  return 0;
}

template <typename T>
struct WsPtrs {
  int *ctl;
  double *dctl;
  T *om, *bt, *s11, *cval, *ccol, *q1, *gt, *r11, *rinv, *zt, *bjt, *cbt, *r, *bv, *avec, *z, *hpart,
      *npart, *vp, *rz, *tmp, *yt, *rt, *t1, *mt, *us, *vs, *qv, *qg, *sgnv, *sgn;
  int *sel, *cidx, *bi, *sgni;
};

template <typename T>
WsPtrs<T> ws_ptrs(const ffsrqr_plan_s *P, unsigned char *ws) {
  WsPtrs<T> w;
#define PT(name, off) w.name = reinterpret_cast<decltype(w.name)>(ws + P->off)
  PT(ctl, off_ctl);
  PT(dctl, off_dctl);
  PT(om, off_om);
  PT(bt, off_bt);
  PT(s11, off_s11);
  PT(cval, off_cval);
  PT(ccol, off_ccol);
  PT(q1, off_q1);
  PT(gt, off_gt);
  PT(r11, off_r11);
  PT(rinv, off_rinv);
  PT(zt, off_zt);
  PT(bjt, off_bjt);
  PT(cbt, off_cbt);
  PT(r, off_r);
  PT(bv, off_bv);
  PT(avec, off_avec);
  PT(z, off_z);
  PT(hpart, off_hpart);
  PT(npart, off_npart);
  PT(vp, off_vp);
  PT(rz, off_rz);
  PT(tmp, off_tmp);
  PT(yt, off_yt);
  PT(rt, off_rt);
  PT(t1, off_t1);
  PT(mt, off_mt);
  PT(us, off_us);
  PT(vs, off_vs);
  PT(qv, off_qv);
  PT(qg, off_qg);
  PT(sgnv, off_sgnv);
  PT(sgn, off_sgn);
  PT(sel, off_sel);
  PT(cidx, off_cidx);
  PT(bi, off_bi);
  PT(sgni, off_sgni);
#undef PT
  return w;
}

__global__ void info_kernel(const int *ctl, const double *dctl, ffsrqr_info_t *info) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  info->status = ctl[CTL_STATUS];
  info->swaps = ctl[CTL_SWAPS];
  info->g2_first = dctl[D_G2_FIRST];
  info->g2_final = dctl[D_G2];
  info->cand_first = ctl[CTL_CAND_FIRST];
  info->jacobi_sweeps = ctl[CTL_JACOBI_SWEEPS];
  info->alpha_first = dctl[D_ALPHA_FIRST];
}

// SRQR test on the current candidate (Alg. 4): pick c from the trailing
// estimates, one-step QR residual alpha, closed-form g2.
template <typename T>
int srqr_test(cudaStream_t st, const ffsrqr_plan_s *P, WsPtrs<T> &w, const T *A, int64_t lda,
              uint64_t seed, int first) {
  const int k = P->k;
  srqr_pick_kernel<T><<<1, 256, 0, st>>>(w.bv, w.bi, P->nblk_tn, w.gt, P->ldk, k, w.avec, w.ctl);
  CKL("srqr_pick");
  const int threads = 256;
  const size_t smem1 = (size_t)(k + (threads / 32) * k) * sizeof(T);
  srqr_resid_kernel<T><<<P->nblk_res, threads, smem1, st>>>(A, lda, P->m, w.q1, P->ldk, k, w.avec,
                                                            w.ctl, w.z, w.hpart);
  CKL("srqr_resid");
  // h = Q1^T z: the block partials added once, into the row after them
  T *h = w.hpart + (size_t)P->nblk_res * k;
  srqr_hsum_kernel<T><<<1, 1024, 0, st>>>(w.hpart, P->nblk_res, k, w.ctl, h);
  CKL("srqr_hsum");
  srqr_reorth_kernel<T><<<P->nblk_res, threads, 0, st>>>(P->m, w.q1, P->ldk, k, h, w.ctl, w.z, w.npart);
  CKL("srqr_reorth");
  if (P->g2_rows > 0) {
    srqr_g2est_kernel<T><<<1, 1024, (size_t)g2est_smem_elems(k) * sizeof(T), st>>>(
        w.npart, P->nblk_res, w.r11, k, w.gt, P->ldk, P->g2_rows, seed, P->g, P->max_swaps, w.ctl, w.dctl);
    CKL("srqr_g2est");
    return 0;
  }
  srqr_g2_kernel<T><<<1, 512, 0, st>>>(w.npart, P->nblk_res, w.rinv, k, w.zt, P->ldk, P->g,
                                       P->max_swaps, w.ctl, w.dctl, first);
  CKL("srqr_g2");
  return 0;
}

template <typename T>
bool use_tc(const ffsrqr_plan_s *P, const T *A, int64_t lda) {
  // the tensor-core epilogue holds N tiles of up to TC_MAX_NT columns (the
  // sketch has s columns); wider problems run the CUDA-core passes
  return sizeof(T) == 4 && tc_mode(P->mode) && tc_ok(A, lda) && round_up(P->s, 16) <= TC_MAX_NT;
}

// Pass 2 (a_mn: G^T = A^T X, X = Q1 with rows = m) or pass 3 (tmp = A X,
// X = V' with rows = n): X (rows x k, ld ldk) is transposed to K-major and split
// into its TF32 head and tail, then the 3-product tensor-core pass runs.
int tc_thin_pass(cudaStream_t st, const ffsrqr_plan_s *P, unsigned char *ws, bool a_mn, const float *A,
                 int64_t lda, const float *X, int64_t rows, float *C) {
  const int k = P->k;
  const int M = (int)(a_mn ? P->n : P->m);
  if (P->mode == FFSRQR_MIXED_BF16X3) {
    // BF16 head and tail of X^T (k x rows, K-major), one transposing pass
    const int64_t ldb = round_up(rows, 8);
    __nv_bfloat16 *bh = reinterpret_cast<__nv_bfloat16 *>(ws + P->off_bh);
    __nv_bfloat16 *bl = reinterpret_cast<__nv_bfloat16 *>(ws + P->off_bl);
    transpose_split_bf16_kernel<<<dim3((unsigned)cdiv(rows, 32), (unsigned)cdiv(k, 32)), dim3(32, 8), 0, st>>>(
        X, P->ldk, rows, k, bh, bl, ldb);
    CKL("transpose_split_bf16");
    return launch_tc(st, P, ws, a_mn ? 1 : 2, 3, a_mn, M, k, (int)rows, A, lda, bh, bl, ldb, C, P->ldk, true);
  }
  const int64_t ldt = round_up(rows, 4);
  float *tt = reinterpret_cast<float *>(ws + P->off_tt);
  float *bh = reinterpret_cast<float *>(ws + P->off_bh);
  float *bl = reinterpret_cast<float *>(ws + P->off_bl);
  transpose_kernel<float><<<dim3((unsigned)cdiv(rows, 32), (unsigned)cdiv(k, 32)), dim3(32, 8), 0, st>>>(
      X, P->ldk, k, rows, tt, ldt);
  CKL("transpose_thin");
  split_tf32_kernel<<<(unsigned)std::min<int64_t>(cdiv((int64_t)k * rows, 256), 8 * P->num_sms), 256, 0, st>>>(
      tt, ldt, k, rows, bh, bl);
  CKL("split_tf32");
  return launch_tc(st, P, ws, a_mn ? 1 : 2, 3, a_mn, M, k, (int)rows, A, lda, bh, bl, ldt, C, P->ldk);
}

// ---------------------------------------------------------------------------
// Tensor-core dense products of the mixed mode (3xTF32: FP32-level accuracy)
// ---------------------------------------------------------------------------
struct TcBufs {
  float *bh, *bl;    // K-major split of a tall operand (k x max(m, n))
  float *sinv;       // k x k (ld ldk): (R^{-1})^T
  float *sh, *sl;    // split of a small operand (<= 256 x k, ld ldk)
  float *scr;        // max(m, n) x k (ld ldk) scratch
};

TcBufs tc_bufs(const ffsrqr_plan_s *P, unsigned char *ws) {
  TcBufs b;
  b.bh = reinterpret_cast<float *>(ws + P->off_bh);
  b.bl = reinterpret_cast<float *>(ws + P->off_bl);
  b.sinv = reinterpret_cast<float *>(ws + P->off_sinv);
  b.sh = reinterpret_cast<float *>(ws + P->off_sh);
  b.sl = reinterpret_cast<float *>(ws + P->off_sl);
  b.scr = reinterpret_cast<float *>(ws + P->off_scr);
  return b;
}

// Dh / Dl (cols x rows, ld ldd) = TF32 head / tail of Src^T (Src rows x cols).
int tc_split_t(cudaStream_t st, const float *Src, int64_t lds, int64_t rows, int64_t cols, float *Dh,
               float *Dl, int64_t ldd) {
  transpose_split_kernel<<<dim3((unsigned)cdiv(rows, 32), (unsigned)cdiv(cols, 32)), dim3(32, 8), 0, st>>>(
      Src, lds, rows, cols, Dh, Dl, ldd);
  CKL("transpose_split");
  return 0;
}

// W (k x k) = X^T X for X rows x k (ld ldx, 16-byte aligned rows).
int tc_gram(cudaStream_t st, const ffsrqr_plan_s *P, unsigned char *ws, const float *X, int64_t ldx,
            int64_t rows, float *W) {
  const int k = P->k;
  const TcBufs b = tc_bufs(P, ws);
  const int64_t ldt = round_up(rows, 4);
  int rc;
  if ((rc = tc_split_t(st, X, ldx, rows, k, b.bh, b.bl, ldt))) return rc;
  return launch_tc(st, P, ws, -1, 3, true, k, k, (int)rows, X, ldx, b.bh, b.bl, ldt, W, k);
}

// R (upper triangular, k x k) = chol(W) and sh / sl = split of (R^{-1})^T,
// the K-major operand of the product X R^{-1}, in one launch.
// second: W is the Gram of a first sweep's output (I + E); if ||E||_F is
// small the factor comes from its first-order expansion (cholqr_series_kernel)
// and the exact kernel returns at once.
int tc_chol_inv(cudaStream_t st, const ffsrqr_plan_s *P, unsigned char *ws, const float *W, float *R,
                bool second = false) {
  const int k = P->k;
  if (k > 256) return FFSRQR_STATUS_UNSUPPORTED;
  const TcBufs b = tc_bufs(P, ws);
  int *ctl = reinterpret_cast<int *>(ws + P->off_ctl);
  const int *skip = nullptr;
  if (second) {
    cholqr_series_kernel<<<cholqr_series_grid(k), CS_THREADS, 0, st>>>(W, k, kSeriesTol, R, b.sh, b.sl, P->ldk, ctl,
                                                   ctl + CTL_SERIES_SKIP);
    CKL("cholqr_series");
    skip = ctl + CTL_SERIES_SKIP;
  }
  CK(smem_cap_max((const void *)chol_inv_kernel));
  chol_inv_kernel<<<1, CI_THREADS, chol_inv_smem(k), st>>>(W, k, R, b.sh, b.sl, P->ldk, ctl, skip);
  CKL("chol_inv");
  return 0;
}

// C (rows x N, ldc) = X (rows x K, ldx) Op, with Op's K-major split (N x K,
// ld ldk) already in sh / sl.
int tc_mul(cudaStream_t st, const ffsrqr_plan_s *P, unsigned char *ws, const float *X, int64_t ldx,
           int64_t rows, int N, int K, float *C, int64_t ldc) {
  const TcBufs b = tc_bufs(P, ws);
  return launch_tc(st, P, ws, -1, 3, false, (int)rows, N, K, X, ldx, b.sh, b.sl, P->ldk, C, ldc);
}

// CholeskyQR2 on the tensor cores: Q (rows x k, ld ldk) = X R^{-1}, R = R2 R1
// (Rout, optional).  Each sweep forms the Gram X^T X, its Cholesky factor, the
// explicit inverse of the factor and the product; X is first brought to a
// small condition number by the caller, so the explicit inverse is accurate.
// Q may alias X.
int cholqr2_tc(cudaStream_t st, const ffsrqr_plan_s *P, unsigned char *ws, const float *X, int64_t rows,
               float *Q, float *Rout) {
  const int k = P->k;
  const int64_t ldk = P->ldk;
  const TcBufs b = tc_bufs(P, ws);
  float *W = reinterpret_cast<float *>(ws + P->off_w);
  float *R1 = reinterpret_cast<float *>(ws + P->off_rc1);
  float *R2 = reinterpret_cast<float *>(ws + P->off_rc2);
  int rc;
  if ((rc = tc_gram(st, P, ws, X, ldk, rows, W))) return rc;
  if ((rc = tc_chol_inv(st, P, ws, W, R1))) return rc;
  if ((rc = tc_mul(st, P, ws, X, ldk, rows, k, k, b.scr, ldk))) return rc;
  if ((rc = tc_gram(st, P, ws, b.scr, ldk, rows, W))) return rc;
  if ((rc = tc_chol_inv(st, P, ws, W, R2, true))) return rc;
  if ((rc = tc_mul(st, P, ws, b.scr, ldk, rows, k, k, Q, ldk))) return rc;
  if (Rout) {
    trmm_upper_kernel<float><<<(unsigned)cdiv((int64_t)k * k, 256), 256, 0, st>>>(R2, R1, k, Rout);
    CKL("trmm_upper");
  }
  return 0;
}

// Cluster launch of the Jacobi kernel for the plan's (blocks, lanes per pair).
template <typename T, int LPP>
cudaError_t launch_jacobi_lpp(cudaStream_t st, int C, int k, const T *X, const T *J, T *U, T *S, T *V, int *ctl,
                              T tol, bool query, int *clusters) {
  const JacGeom g = jac_geom(k, C, 16 / (int)sizeof(T));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)C);
  cfg.blockDim = dim3((unsigned)round_up((int64_t)g.npair * LPP, 32));
  cfg.dynamicSmemBytes = jac_cluster_smem(k, C, sizeof(T), LPP);
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (query) return cudaOccupancyMaxActiveClusters(clusters, jacobi_cluster_kernel<T, LPP>, &cfg);
  return cudaLaunchKernelEx(&cfg, jacobi_cluster_kernel<T, LPP>, X, J, k, U, S, V, ctl, (int)JAC_MAX_SWEEPS, tol);
}

template <typename T>
cudaError_t launch_jacobi_any(cudaStream_t st, int C, int lpp, int k, const T *X, const T *J, T *U, T *S, T *V,
                              int *ctl, T tol, bool query, int *clusters) {
  switch (lpp) {
    case 2: return launch_jacobi_lpp<T, 2>(st, C, k, X, J, U, S, V, ctl, tol, query, clusters);
    case 4: return launch_jacobi_lpp<T, 4>(st, C, k, X, J, U, S, V, ctl, tol, query, clusters);
    default: return launch_jacobi_lpp<T, 8>(st, C, k, X, J, U, S, V, ctl, tol, query, clusters);
  }
}

template <typename T>
int launch_jacobi(cudaStream_t st, const ffsrqr_plan_s *P, const T *X, const T *J, T *U, T *S, T *V, int *ctl,
                  T tol) {
  CK(launch_jacobi_any<T>(st, P->jac_cluster, P->jac_lpp, P->k, X, J, U, S, V, ctl, tol, false, nullptr));
  ++g_launches;
  return 0;
}

// Single-precision SVD of the small factor M (kk x kk, row-major, leading
// dimension ldm): U_s, V_s (kk x kk, row-major) and S by the column-block
// cluster Jacobi on M^T.  query: only ask how many such clusters the device
// can hold at once.
cudaError_t launch_jacobi_blk(cudaStream_t st, const float *M, int kk, int ldm, float *Us, float *S, float *Vs,
                              int *ctl, bool query = false, int *clusters = nullptr) {
  const int C = jb_cluster_for(kk);
  const JbGeom g = jb_geom(kk, C);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)C);
  cfg.blockDim = dim3((unsigned)(32 * g.nw));
  cfg.dynamicSmemBytes = jb_smem_bytes(kk);
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (query) return cudaOccupancyMaxActiveClusters(clusters, jacobi_blk_kernel, &cfg);
  const float tol = 4.f * sqrtf((float)kk) * 5.9604645e-8f;
  return cudaLaunchKernelEx(&cfg, jacobi_blk_kernel, M, kk, ldm, tol, (int)JB_MAX_SWEEPS, Us, S, Vs, ctl);
}

// Alg. 9 up to the small SVD: a1-a10 without the SVD of M_t (M_t, workspace
// item 8, and Q_t, V' in place).  The phase-batched runs of a batch or a
// server run this part of several problems, their small SVDs in one launch,
// then run_post.
// Alg. 2 (TRQRCP) with block size b < k, replacing the one-block a3-a5.
// The sketch B (b + p rows) is copied to a working sample (the trailing-norm
// buffer, free until the SRQR test); for the block at positions jb..jb+bb-1:
//   - partial QRCP for bb steps on the working sample, the columns selected
//     by earlier blocks excluded (their marks in sel), pivots to piv[jb:];
//   - Y = A(:, J_j), projected twice against Q1(:, 0:jb) (block classical
//     Gram-Schmidt, the products on the CUDA cores), preconditioned by the
//     sample's R factor S11 of the block and orthonormalised by CholeskyQR2
//     into Q1(:, jb:jb+bb);
//   - one pass over A: G^T(:, jb:jb+bb) = A^T Q_j (the rows of R = Q1^T A Pi
//     that the one-block pipeline forms in its pass 2);
//   - unless it is the last block, the sample update
//     B <- B - B(:, J_j) R_jj^{-1} G_j   (R_jj the upper triangle of G_j(:, J_j)),
//     so that the sample stays Omega (I - Q Q^T) A, the sample of the
//     trailing matrix.
// The block's factor products run through a copy of the plan with k = bb
// (leading dimensions unchanged).  b is a multiple of 8 (plan check), so
// every block's first column keeps 32-byte row alignment.
template <typename T>
int run_blocked(ffsrqr_plan_s *P, const T *A, int64_t lda, int32_t *piv, unsigned char *ws, WsPtrs<T> &w,
                cudaStream_t st, bool tc) {
  const int64_t m = P->m, n = P->n;
  const int k = P->k, s = P->s, b = P->blk;
  const int64_t lds = P->lds, ldk = P->ldk;
  const int nsm = P->num_sms;
  T *smp = w.cbt;
  int rc;
  CK(cudaMemcpyAsync(smp, w.bt, (size_t)n * lds * sizeof(T), cudaMemcpyDeviceToDevice, st));
  for (int jb = 0; jb < k; jb += b) {
    const int bb = std::min(b, k - jb);
    const bool last = jb + bb == k;
    ffsrqr_plan_s Pb = *P;
    Pb.k = bb;
    if (jb > 0) {  // the QRCP kernel's barrier counter and winner keys start at zero
      CK(cudaMemsetAsync(w.ctl + CTL_BARRIER0, 0, sizeof(int), st));
      CK(cudaMemsetAsync(w.ctl + CTL_WIN_KEY, 0, 6 * sizeof(int), st));
    }
    QrcpArgs<T> qa;
    qa.Bt = smp;
    qa.n = n;
    qa.s = s;
    qa.lds = (int)lds;
    qa.k = bb;
    qa.piv = piv + jb;
    qa.S11 = w.s11;
    qa.cand_val = w.cval;
    qa.cand_idx = w.cidx;
    qa.cand_col = w.ccol;
    qa.sel = w.sel;
    qa.presel = w.sel;
    qa.ctl = w.ctl;
    qa.spin_limit = kSpinLimit;
    qa.stall_step = (last && (P->flags & FFSRQR_FLAG_TEST_STALL)) ? bb - 1 : -1;
    qa.cols_per_block = P->qrcp_cols;
    qa.s_pad = P->qrcp_spad;
    void *args[] = {&qa};
    CK(smem_cap_max((const void *)qrcp_kernel<T>));
    CK(cudaLaunchCooperativeKernel((void *)qrcp_kernel<T>, dim3(P->qrcp_grid), dim3(P->qrcp_threads), args,
                                   P->qrcp_smem, st));
    ++g_launches;
    posdiag_rows_kernel<T><<<(unsigned)cdiv((int64_t)bb * 32, 256), 256, 0, st>>>(w.s11, bb);
    CKL("posdiag");
    T *Y = w.q1 + jb;
    gather_cols_kernel<T><<<(unsigned)std::min<int64_t>(cdiv(m * bb, 256), 8 * nsm), 256, 0, st>>>(
        A, lda, m, bb, piv + jb, Y, ldk);
    CKL("gather_cols");
    for (int r = 0; r < 2 && jb > 0; ++r) {
      // C (jb x bb) = Q1(:, 0:jb)^T Y, then Y -= Q1(:, 0:jb) C
      if ((rc = launch_gemm<T>(st, P, ws, jb, bb, (int)m, w.q1, ldk, true, Y, ldk, true, w.rinv, bb))) return rc;
      if ((rc = launch_gemm<T>(st, P, ws, (int)m, bb, jb, w.q1, ldk, false, w.rinv, bb, true, Y, ldk, T(-1),
                               T(1))))
        return rc;
    }
    if ((rc = launch_trsm<T, true>(st, &Pb, Y, ldk, m, w.s11, bb, 1))) return rc;
    if (tc) {
      if ((rc = cholqr2_tc(st, &Pb, ws, (const float *)Y, m, (float *)Y, nullptr))) return rc;
      if ((rc = tc_thin_pass(st, &Pb, ws, true, (const float *)A, lda, (const float *)Y, m, (float *)(w.gt + jb))))
        return rc;
    } else {
      if ((rc = cholqr2<T>(st, &Pb, ws, Y, ldk, m, nullptr))) return rc;
      if ((rc = launch_gemm<T>(st, P, ws, (int)n, bb, (int)m, A, lda, true, Y, ldk, true, w.gt + jb, ldk)))
        return rc;
    }
    if (last) break;
    // sample update: B^T -= Z_j^T B(:, J_j)^T, Z_j^T = G_j^T R_jj^{-T}
    extract_r11_kernel<T><<<(unsigned)cdiv((int64_t)bb * bb, 256), 256, 0, st>>>(w.gt + jb, ldk, bb, piv + jb,
                                                                                  w.r11, nullptr);
    CKL("extract_r11");
    copy2d_kernel<T><<<(unsigned)std::min<int64_t>(cdiv(n * 32, 256), 8 * nsm), 256, 0, st>>>(w.gt + jb, ldk, w.zt,
                                                                                           ldk, n, bb, nullptr);
    CKL("copy_zt");
    if ((rc = launch_trsm<T, false>(st, &Pb, w.zt, ldk, n, w.r11, 1, bb))) return rc;
    gather_rows_kernel<T><<<(unsigned)cdiv((int64_t)bb * s, 256), 256, 0, st>>>(smp, lds, bb, s, piv + jb, w.bjt,
                                                                                lds);
    CKL("gather_rows");
    if ((rc = launch_gemm<T>(st, P, ws, (int)n, s, bb, w.zt, ldk, false, w.bjt, lds, true, smp, lds, T(-1),
                             T(1))))
      return rc;
  }
  return 0;
}

template <typename T>
int run_pre(ffsrqr_plan_s *P, const T *A, int64_t lda, uint64_t seed, int32_t *piv, unsigned char *ws,
            cudaStream_t st) {
  const int64_t m = P->m, n = P->n;
  const int k = P->k, s = P->s;
  const int64_t ldm = P->ldm, lds = P->lds, ldk = P->ldk;
  WsPtrs<T> w = ws_ptrs<T>(P, ws);
  const int nsm = P->num_sms;
  const bool tc = use_tc<T>(P, A, lda);
  int rc;

  CK(cudaMemsetAsync(ws + P->off_ctl, 0, CTL_WORDS * sizeof(int), st));
  CK(cudaMemsetAsync(ws + P->off_dctl, 0, D_WORDS * sizeof(double), st));
  CK(cudaMemsetAsync(w.sel, 0, (size_t)n * sizeof(int), st));
  CK(cudaMemsetAsync(piv, 0, (size_t)n * sizeof(int32_t), st));
  init_ctl_kernel<<<1, 32, 0, st>>>(w.ctl, w.dctl);
  CKL("init_ctl");
  if (P->flags & 1) {
    nonfinite_kernel<T><<<4 * nsm, 256, 0, st>>>(A, lda, m, n, w.ctl);
    CKL("nonfinite");
  }

  // a1: Omega
  MARK(0);
  {
    const int64_t nq = cdiv((int64_t)s * m, 4);
    omega_kernel<T><<<(unsigned)std::min<int64_t>(cdiv(nq, 256), 8 * nsm), 256, 0, st>>>(w.om, s, m, ldm,
                                                                                         seed);
    CKL("omega");
  }
  MARK(1);
  // a2: pass 1, B^T (n x s) = A^T Omega^T
  if (tc && P->mode == FFSRQR_MIXED_BF16X3) {
    // BF16 sketch: Omega rounded to BF16 once, A converted on chip
    const int64_t ldb = round_up(m, 8);
    __nv_bfloat16 *omb = reinterpret_cast<__nv_bfloat16 *>(ws + P->off_omb);
    to_bf16_kernel<<<(unsigned)std::min<int64_t>(cdiv((int64_t)s * m, 256), 8 * nsm), 256, 0, st>>>(
        (const float *)w.om, ldm, s, m, omb, ldb);
    CKL("to_bf16");
    if ((rc = launch_tc(st, P, ws, 0, 1, true, (int)n, s, (int)m, (const float *)A, lda, omb, nullptr, ldb,
                        (float *)w.bt, lds, true)))
      return rc;
  } else if (tc) {
    if ((rc = launch_tc(st, P, ws, 0, 1, true, (int)n, s, (int)m, (const float *)A, lda, (const float *)w.om,
                        nullptr, ldm, (float *)w.bt, lds)))
      return rc;
  } else if ((rc = launch_gemm<T>(st, P, ws, (int)n, s, (int)m, A, lda, true, w.om, ldm, false, w.bt, lds))) {
    return rc;
  }
  // a3: QRCP on the sketch
  MARK(2);
  if (P->blk < k) {
    // a3-a5 block by block (Alg. 2 with b < k); its phase times all fall
    // under the QRCP mark
    if ((rc = run_blocked<T>(P, A, lda, piv, ws, w, st, tc))) return rc;
    MARK(3);
    MARK(4);
  } else {
  {
    QrcpArgs<T> qa;
    qa.Bt = w.bt;
    qa.n = n;
    qa.s = s;
    qa.lds = (int)lds;
    qa.k = k;
    qa.piv = piv;
    qa.S11 = w.s11;
    qa.cand_val = w.cval;
    qa.cand_idx = w.cidx;
    qa.cand_col = w.ccol;
    qa.sel = w.sel;
    qa.ctl = w.ctl;
    qa.spin_limit = kSpinLimit;
    qa.stall_step = (P->flags & FFSRQR_FLAG_TEST_STALL) ? k - 1 : -1;
    qa.cols_per_block = P->qrcp_cols;
    qa.s_pad = P->qrcp_spad;
    void *args[] = {&qa};
    CK(smem_cap_max((const void *)qrcp_kernel<T>));
    CK(cudaLaunchCooperativeKernel((void *)qrcp_kernel<T>, dim3(P->qrcp_grid), dim3(P->qrcp_threads),
                                   args, P->qrcp_smem, st));
    ++g_launches;
  }
  posdiag_rows_kernel<T><<<(unsigned)cdiv((int64_t)k * 32, 256), 256, 0, st>>>(w.s11, k);
  CKL("posdiag");
  MARK(3);
  // a4: panel Y = A_J S11^{-1}, CholeskyQR2 -> Q1
  gather_cols_kernel<T><<<(unsigned)std::min<int64_t>(cdiv(m * k, 256), 8 * nsm), 256, 0, st>>>(
      A, lda, m, k, piv, w.q1, ldk);
  CKL("gather_cols");
  if ((rc = launch_trsm<T, true>(st, P, w.q1, ldk, m, w.s11, k, 1))) return rc;
  if (tc) {
    if ((rc = cholqr2_tc(st, P, ws, (const float *)w.q1, m, (float *)w.q1, nullptr))) return rc;
  } else if ((rc = cholqr2<T>(st, P, ws, w.q1, ldk, m, nullptr))) {
    return rc;
  }
  MARK(4);
  // a5: pass 2, G^T (n x k) = A^T Q1
  if (tc) {
    if ((rc = tc_thin_pass(st, P, ws, true, (const float *)A, lda, (const float *)w.q1, m, (float *)w.gt)))
      return rc;
  } else if ((rc = launch_gemm<T>(st, P, ws, (int)n, k, (int)m, A, lda, true, w.q1, ldk, true, w.gt, ldk))) {
    return rc;
  }
  }
  MARK(5);
  // a6: R11, R11^{-1}, Z^T = G^T R11^{-T}
  extract_r11_kernel<T><<<(unsigned)cdiv((int64_t)k * k, 256), 256, 0, st>>>(w.gt, ldk, k, piv, w.r11, nullptr);
  CKL("extract_r11");
  const bool fork_rinv = P->g2_rows == 0;  // the estimate solves with R11 itself
  if (fork_rinv) {
    // R11^{-1} for the exact g2, on the plan's side stream while Z^T and the
    // trailing-norm estimate are formed (joined before the g2 kernel)
    CK(cudaEventRecord(P->ev_fork, st));
    CK(cudaStreamWaitEvent(P->side, P->ev_fork, 0));
    eye_kernel<T><<<(unsigned)cdiv((int64_t)k * k, 256), 256, 0, P->side>>>(w.rinv, k, k);
    CKL("eye");
    if ((rc = launch_trsm<T, true>(P->side, P, w.rinv, k, k, w.r11, k, 1))) return rc;
    CK(cudaEventRecord(P->ev_join, P->side));
  }
  copy2d_kernel<T><<<(unsigned)std::min<int64_t>(cdiv(n * k, 256), 8 * nsm), 256, 0, st>>>(w.gt, ldk, w.zt,
                                                                                          ldk, n, k, nullptr);
  CKL("copy_zt");
  if ((rc = launch_trsm<T, false>(st, P, w.zt, ldk, n, w.r11, 1, k))) return rc;
  // trailing-norm estimate and the first SRQR test
  gather_rows_kernel<T><<<(unsigned)cdiv((int64_t)k * s, 256), 256, 0, st>>>(w.bt, lds, k, s, piv, w.bjt,
                                                                             lds);
  CKL("gather_rows");
  if (tc) {
    const TcBufs tb = tc_bufs(P, ws);
    if ((rc = tc_split_t(st, (const float *)w.bjt, lds, k, s, tb.sh, tb.sl, ldk))) return rc;
    if ((rc = tc_mul(st, P, ws, (const float *)w.zt, ldk, n, s, k, (float *)w.cbt, lds))) return rc;
  } else if ((rc = launch_gemm<T>(st, P, ws, (int)n, s, k, w.zt, ldk, false, w.bjt, lds, true, w.cbt, lds))) {
    return rc;
  }
  trailing_norms_kernel<T><<<P->nblk_tn, 256, 0, st>>>(w.bt, w.cbt, lds, n, s, w.sel, w.r, w.bv, w.bi);
  CKL("trailing_norms");
  if (fork_rinv) CK(cudaStreamWaitEvent(st, P->ev_join, 0));
  if (k < n) {
    if ((rc = srqr_test<T>(st, P, w, A, lda, seed, 1))) return rc;
  }
  MARK(6);
  // a7: swap loop (Alg. 4) while g2 > g, entirely on the device; afterwards
  // R11 and Z^T are rebuilt for the final column set (skipped on the device
  // when no swap happened)
  if (k < n) {
    SwapArgs<T> sa;
    sa.A = A;
    sa.lda = lda;
    sa.m = m;
    sa.n = n;
    sa.k = k;
    sa.gt = w.gt;
    sa.ldg = ldk;
    sa.rowk = reinterpret_cast<T *>(ws + P->off_rowk);
    sa.q1 = w.q1;
    sa.ldq = ldk;
    sa.qk = reinterpret_cast<T *>(ws + P->off_qk);
    sa.z = w.z;
    sa.r = w.r;
    sa.sel = w.sel;
    sa.piv = piv;
    sa.rot = reinterpret_cast<T *>(ws + P->off_rot);
    sa.Rd = reinterpret_cast<T *>(ws + P->off_rd);
    sa.X = reinterpret_cast<T *>(ws + P->off_xinv);
    sa.part = reinterpret_cast<T *>(ws + P->off_swpart);
    sa.bv = reinterpret_cast<T *>(ws + P->off_swbv);
    sa.bi = reinterpret_cast<int *>(ws + P->off_swbi);
    sa.ctl = w.ctl;
    sa.dctl = w.dctl;
    sa.g = P->g;
    sa.max_swaps = P->max_swaps;
    sa.spin_limit = kSpinLimit;
    sa.g2_rows = P->g2_rows;
    sa.seed = seed;
    void *args[] = {&sa};
    CK(smem_cap_max((const void *)srqr_swap_kernel<T>));
    CK(cudaLaunchCooperativeKernel((void *)srqr_swap_kernel<T>, dim3(P->swap_grid), dim3(512), args,
                                   P->swap_smem, st));
    ++g_launches;
    const int *gate = w.ctl + CTL_SWAPS;
    extract_r11_kernel<T><<<(unsigned)cdiv((int64_t)k * k, 256), 256, 0, st>>>(w.gt, ldk, k, piv, w.r11, gate);
    CKL("extract_r11_swapped");
    copy2d_kernel<T><<<(unsigned)std::min<int64_t>(cdiv(n * k, 256), 8 * nsm), 256, 0, st>>>(w.gt, ldk, w.zt,
                                                                                            ldk, n, k, gate);
    CKL("copy_zt_swapped");
    if ((rc = launch_trsm<T, false>(st, P, w.zt, ldk, n, w.r11, 1, k, gate))) return rc;
  }
  MARK(7);
  // a8: V' = orth(Z^T), R_z
  if (tc) {
    if ((rc = cholqr2_tc(st, P, ws, (const float *)w.zt, n, (float *)w.vp, (float *)w.rz))) return rc;
  } else {
    copy2d_kernel<T><<<(unsigned)std::min<int64_t>(cdiv(n * k, 256), 8 * nsm), 256, 0, st>>>(w.zt, ldk, w.vp,
                                                                                            ldk, n, k, nullptr);
    CKL("copy_vp");
    if ((rc = cholqr2<T>(st, P, ws, w.vp, ldk, n, w.rz))) return rc;
  }
  MARK(8);
  // a9: pass 3, tmp (m x k) = A V'
  if (tc) {
    if ((rc = tc_thin_pass(st, P, ws, false, (const float *)A, lda, (const float *)w.vp, n, (float *)w.tmp)))
      return rc;
  } else if ((rc = launch_gemm<T>(st, P, ws, (int)m, k, (int)n, A, lda, false, w.vp, ldk, true, w.tmp, ldk))) {
    return rc;
  }
  MARK(9);
  // a10: Y_t = tmp R_z^{-T} R11^{-1}; CholeskyQR2 -> Q_t, R_t; M_t = R_t R11 R_z^T
  copy2d_kernel<T><<<(unsigned)std::min<int64_t>(cdiv(m * k, 256), 8 * nsm), 256, 0, st>>>(w.tmp, ldk, w.yt,
                                                                                          ldk, m, k, nullptr);
  CKL("copy_yt");
  if ((rc = launch_trsm<T, false>(st, P, w.yt, ldk, m, w.rz, 1, k))) return rc;
  if ((rc = launch_trsm<T, true>(st, P, w.yt, ldk, m, w.r11, k, 1))) return rc;
  if (tc) {
    if ((rc = cholqr2_tc(st, P, ws, (const float *)w.yt, m, (float *)w.yt, (float *)w.rt))) return rc;
  } else if ((rc = cholqr2<T>(st, P, ws, w.yt, ldk, m, w.rt))) {
    return rc;
  }
  if ((rc = launch_gemm<T>(st, P, ws, k, k, k, w.rt, k, false, w.r11, k, true, w.t1, k))) return rc;
  if ((rc = launch_gemm<T>(st, P, ws, k, k, k, w.t1, k, false, w.rz, k, false, w.mt, k))) return rc;
  MARK(10);
  return 0;
}

// The SVD of M_t (k x k): S (k) and U_s, V_s into the workspace.
template <typename T>
int run_small_svd(ffsrqr_plan_s *P, T *S, unsigned char *ws, cudaStream_t st) {
  const int k = P->k;
  WsPtrs<T> w = ws_ptrs<T>(P, ws);
  int rc;
  if constexpr (sizeof(T) == 4) {
    // single precision: column-block cluster Jacobi on M_t^T
    CK(launch_jacobi_blk(st, (const float *)w.mt, k, k, (float *)w.us, (float *)S, (float *)w.vs, w.ctl));
    ++g_launches;
  } else {
    // M_t^T = Q R: X = R^T to t1 and the reflectors to qv; Q (to qg) is formed
    // on the plan's side stream while the cluster Jacobi runs on [X; I]; then
    // V_s = Q J (J to t1, which the Jacobi no longer needs once loaded)
    const size_t qsmem = precond_qr_smem(k, sizeof(T));
    precond_qr_r_kernel<T><<<1, 1024, qsmem, st>>>(w.mt, k, w.t1, w.qv);
    CKL("precond_qr_r");
    CK(cudaEventRecord(P->ev_fork, st));
    CK(cudaStreamWaitEvent(P->side, P->ev_fork, 0));
    precond_qr_q_kernel<T><<<1, 1024, qsmem, P->side>>>(k, w.qv, w.qg);
    CKL("precond_qr_q");
    CK(cudaEventRecord(P->ev_join, P->side));
    const T eps = (sizeof(T) == 4) ? T(5.9604645e-8) : T(1.1102230246251565e-16);
    const T tol = (sizeof(T) == 4) ? T(4) * sqrt(T(k)) * eps : T(k) * eps;
    if ((rc = launch_jacobi<T>(st, P, w.t1, (const T *)nullptr, w.us, S, w.t1, w.ctl, tol))) return rc;
    CK(cudaStreamWaitEvent(st, P->ev_join, 0));
    if ((rc = launch_gemm<T>(st, P, ws, k, k, k, w.qg, k, true, w.t1, k, true, w.vs, k))) return rc;
  }
  return 0;
}

// Alg. 9 after the small SVD: a11 (U = Q_t U_s, V = V' V_s, the sign rule),
// the pivot tail and the report.
template <typename T>
int run_post(ffsrqr_plan_s *P, const T *A, int64_t lda, T *U, int64_t ldu, T *V, int64_t ldv, int32_t *piv,
             unsigned char *ws, cudaStream_t st, ffsrqr_info_t *info) {
  const int64_t m = P->m, n = P->n;
  const int k = P->k;
  const int64_t ldk = P->ldk;
  WsPtrs<T> w = ws_ptrs<T>(P, ws);
  const int nsm = P->num_sms;
  const bool tc = use_tc<T>(P, A, lda);
  int rc;
  MARK(11);
  // a11: U = Q_t U_s, V = V' V_s, sign rule
  if (tc) {
    const TcBufs tb = tc_bufs(P, ws);
    if ((rc = tc_split_t(st, (const float *)w.us, k, k, k, tb.sh, tb.sl, ldk))) return rc;
    if ((rc = tc_mul(st, P, ws, (const float *)w.yt, ldk, m, k, k, (float *)U, ldu))) return rc;
    if ((rc = tc_split_t(st, (const float *)w.vs, k, k, k, tb.sh, tb.sl, ldk))) return rc;
    if ((rc = tc_mul(st, P, ws, (const float *)w.vp, ldk, n, k, k, (float *)V, ldv))) return rc;
  } else {
    if ((rc = launch_gemm<T>(st, P, ws, (int)m, k, k, w.yt, ldk, false, w.us, k, true, U, ldu))) return rc;
    if ((rc = launch_gemm<T>(st, P, ws, (int)n, k, k, w.vp, ldk, false, w.vs, k, true, V, ldv))) return rc;
  }
  sign_partial_kernel<T><<<P->nblk_sign, 256, 0, st>>>(U, ldu, m, k, w.sgnv, w.sgni);
  CKL("sign_partial");
  sign_final_kernel<T><<<(unsigned)cdiv((int64_t)k * 32, 256), 256, 0, st>>>(U, ldu, k, w.sgnv, w.sgni, P->nblk_sign, w.sgn);
  CKL("sign_final");
  scale_cols_kernel<T><<<(unsigned)std::min<int64_t>(cdiv(m * k, 256), 8 * nsm), 256, 0, st>>>(U, ldu, m, k,
                                                                                              w.sgn);
  scale_cols_kernel<T><<<(unsigned)std::min<int64_t>(cdiv(n * k, 256), 8 * nsm), 256, 0, st>>>(V, ldv, n, k,
                                                                                              w.sgn);
  CKL("scale_cols");
  piv_rest_kernel<<<1, 1024, 0, st>>>(w.sel, n, k, piv);
  CKL("piv_rest");
  ffsrqr_info_t *dinfo = reinterpret_cast<ffsrqr_info_t *>(ws + P->off_info);
  info_kernel<<<1, 32, 0, st>>>(w.ctl, w.dctl, dinfo);
  MARK(12);
  CKL("info");
  if (info) CK(cudaMemcpyAsync(info, dinfo, sizeof(ffsrqr_info_t), cudaMemcpyDeviceToHost, st));
  return 0;
}

template <typename T>
int run_impl(ffsrqr_plan_s *P, const T *A, int64_t lda, uint64_t seed, T *U, int64_t ldu, T *S, T *V,
             int64_t ldv, int32_t *piv, unsigned char *ws, cudaStream_t st, ffsrqr_info_t *info) {
  int rc;
  if ((rc = run_pre<T>(P, A, lda, seed, piv, ws, st))) return rc;
  if ((rc = run_small_svd<T>(P, S, ws, st))) return rc;
  return run_post<T>(P, A, lda, U, ldu, V, ldv, piv, ws, st, info);
}

// Alg. 9 with SRQR depth l = P->k above the target rank kout: the depth-l
// U, S, V go to the workspace and their leading kout columns to the caller.
template <typename T>
int run_truncated(ffsrqr_plan_s *P, const T *A, int64_t lda, uint64_t seed, T *U, int64_t ldu, T *S, T *V,
                  int64_t ldv, int32_t *piv, unsigned char *ws, cudaStream_t st, ffsrqr_info_t *info) {
  const int64_t m = P->m, n = P->n;
  const int l = P->k, k = P->kout, nsm = P->num_sms;
  T *uo = reinterpret_cast<T *>(ws + P->off_uo);
  T *so = reinterpret_cast<T *>(ws + P->off_so);
  T *vo = reinterpret_cast<T *>(ws + P->off_vo);
  int rc;
  if ((rc = run_impl<T>(P, A, lda, seed, uo, l, so, vo, l, piv, ws, st, info))) return rc;
  copy2d_kernel<T><<<(unsigned)std::min<int64_t>(cdiv(m * k, 256), 8 * nsm), 256, 0, st>>>(uo, l, U, ldu, m, k,
                                                                                          nullptr);
  CKL("copy_u");
  copy2d_kernel<T><<<(unsigned)std::min<int64_t>(cdiv(n * k, 256), 8 * nsm), 256, 0, st>>>(vo, l, V, ldv, n, k,
                                                                                          nullptr);
  CKL("copy_v");
  CK(cudaMemcpyAsync(S, so, (size_t)k * sizeof(T), cudaMemcpyDeviceToDevice, st));
  return 0;
}

// Approximate SVD by randomized subspace iteration (the paper's appendix
// algorithm) on this plan's kernels, with l = P->k = kout + p columns:
//   Omega (n x l);  Q = orth(A Omega);  q times: V' = orth(A^T Q), Q = orth(A V');
//   A^T Q = V' R_z  (so Q^T A = R_z^T V'^T);  svd(R_z^T) = W S Z^T;
//   U = Q W, V = V' Z, the leading kout triplets.
// orth() is CholeskyQR2; the passes and products are the Flip-Flop SRQR ones.
template <typename T>
int run_rsi(ffsrqr_plan_s *P, const T *A, int64_t lda, uint64_t seed, T *U, int64_t ldu, T *S, T *V,
            int64_t ldv, unsigned char *ws, cudaStream_t st, ffsrqr_info_t *info) {
  const int64_t m = P->m, n = P->n, ldk = P->ldk;
  const int l = P->k, k = P->kout, nsm = P->num_sms;
  WsPtrs<T> w = ws_ptrs<T>(P, ws);
  int rc;
  CK(cudaMemsetAsync(ws + P->off_ctl, 0, CTL_WORDS * sizeof(int), st));
  CK(cudaMemsetAsync(ws + P->off_dctl, 0, D_WORDS * sizeof(double), st));
  init_ctl_kernel<<<1, 32, 0, st>>>(w.ctl, w.dctl);
  CKL("init_ctl");
  // Omega, n x l row-major (element (i, j) is draw i l + j), into V'
  {
    const int64_t nq = cdiv(n * l, 4);
    omega_kernel<T><<<(unsigned)std::min<int64_t>(cdiv(nq, 256), 8 * nsm), 256, 0, st>>>(w.vp, (int)n, l, ldk,
                                                                                         seed);
    CKL("omega");
  }
  const bool tc = use_tc<T>(P, A, lda);
  auto right = [&](const T *X, T *C) -> int {  // C (m x l) = A X, X n x l
    if (tc) return tc_thin_pass(st, P, ws, false, (const float *)A, lda, (const float *)X, n, (float *)C);
    return launch_gemm<T>(st, P, ws, (int)m, l, (int)n, A, lda, false, X, ldk, true, C, ldk);
  };
  auto left = [&](const T *X, T *C) -> int {  // C (n x l) = A^T X, X m x l
    if (tc) return tc_thin_pass(st, P, ws, true, (const float *)A, lda, (const float *)X, m, (float *)C);
    return launch_gemm<T>(st, P, ws, (int)n, l, (int)m, A, lda, true, X, ldk, true, C, ldk);
  };
  auto orth = [&](const T *X, int64_t rows, T *Q, T *R) -> int {  // Q = X R^{-1}
    if (tc) return cholqr2_tc(st, P, ws, (const float *)X, rows, (float *)Q, (float *)R);
    copy2d_kernel<T><<<(unsigned)std::min<int64_t>(cdiv(rows * l, 256), 8 * nsm), 256, 0, st>>>(X, ldk, Q, ldk,
                                                                                               rows, l, nullptr);
    CKL("copy_orth");
    return cholqr2<T>(st, P, ws, Q, ldk, rows, R);
  };
  if ((rc = right(w.vp, w.tmp)) || (rc = orth(w.tmp, m, w.yt, nullptr))) return rc;
  for (int it = 0; it < P->rsi_q; ++it) {
    if ((rc = left(w.yt, w.gt)) || (rc = orth(w.gt, n, w.vp, nullptr))) return rc;
    if ((rc = right(w.vp, w.tmp)) || (rc = orth(w.tmp, m, w.yt, nullptr))) return rc;
  }
  if ((rc = left(w.yt, w.gt)) || (rc = orth(w.gt, n, w.vp, w.rz))) return rc;
  // M = R_z^T (l x l): Q^T A = M V'^T
  transpose_kernel<T><<<dim3((unsigned)cdiv(l, 32), (unsigned)cdiv(l, 32)), dim3(32, 8), 0, st>>>(w.rz, l, l, l,
                                                                                                  w.mt, l);
  CKL("transpose_rz");
  // outputs at full width l: to the caller's buffers when kout = l
  T *uo = (k < l) ? reinterpret_cast<T *>(ws + P->off_uo) : U;
  T *so = (k < l) ? reinterpret_cast<T *>(ws + P->off_so) : S;
  T *vo = (k < l) ? reinterpret_cast<T *>(ws + P->off_vo) : V;
  const int64_t lduo = (k < l) ? l : ldu, ldvo = (k < l) ? l : ldv;
  if constexpr (sizeof(T) == 4) {
    // the small SVD of the Flip-Flop SRQR pipeline (column-block cluster Jacobi)
    CK(launch_jacobi_blk(st, (const float *)w.mt, l, l, (float *)w.us, (float *)so, (float *)w.vs, w.ctl));
    ++g_launches;
  } else {
    // the small SVD of the Flip-Flop SRQR pipeline: QR of M^T, Jacobi on R^T,
    // Q of the small QR formed on the side stream
    const size_t qsmem = precond_qr_smem(l, sizeof(T));
    precond_qr_r_kernel<T><<<1, 1024, qsmem, st>>>(w.mt, l, w.t1, w.qv);
    CKL("precond_qr_r");
    CK(cudaEventRecord(P->ev_fork, st));
    CK(cudaStreamWaitEvent(P->side, P->ev_fork, 0));
    precond_qr_q_kernel<T><<<1, 1024, qsmem, P->side>>>(l, w.qv, w.qg);
    CKL("precond_qr_q");
    CK(cudaEventRecord(P->ev_join, P->side));
    const T eps = (sizeof(T) == 4) ? T(5.9604645e-8) : T(1.1102230246251565e-16);
    const T tol = (sizeof(T) == 4) ? T(4) * sqrt(T(l)) * eps : T(l) * eps;
    if ((rc = launch_jacobi<T>(st, P, w.t1, (const T *)nullptr, w.us, so, w.t1, w.ctl, tol))) return rc;
    CK(cudaStreamWaitEvent(st, P->ev_join, 0));
    if ((rc = launch_gemm<T>(st, P, ws, l, l, l, w.qg, l, true, w.t1, l, true, w.vs, l))) return rc;
  }
  if (tc) {
    const TcBufs tb = tc_bufs(P, ws);
    if ((rc = tc_split_t(st, (const float *)w.us, l, l, l, tb.sh, tb.sl, ldk))) return rc;
    if ((rc = tc_mul(st, P, ws, (const float *)w.yt, ldk, m, l, l, (float *)uo, lduo))) return rc;
    if ((rc = tc_split_t(st, (const float *)w.vs, l, l, l, tb.sh, tb.sl, ldk))) return rc;
    if ((rc = tc_mul(st, P, ws, (const float *)w.vp, ldk, n, l, l, (float *)vo, ldvo))) return rc;
  } else {
    if ((rc = launch_gemm<T>(st, P, ws, (int)m, l, l, w.yt, ldk, false, w.us, l, true, uo, lduo))) return rc;
    if ((rc = launch_gemm<T>(st, P, ws, (int)n, l, l, w.vp, ldk, false, w.vs, l, true, vo, ldvo))) return rc;
  }
  sign_partial_kernel<T><<<P->nblk_sign, 256, 0, st>>>(uo, lduo, m, l, w.sgnv, w.sgni);
  CKL("sign_partial");
  sign_final_kernel<T><<<(unsigned)cdiv((int64_t)l * 32, 256), 256, 0, st>>>(uo, lduo, l, w.sgnv, w.sgni, P->nblk_sign, w.sgn);
  CKL("sign_final");
  scale_cols_kernel<T><<<(unsigned)std::min<int64_t>(cdiv(m * l, 256), 8 * nsm), 256, 0, st>>>(uo, lduo, m, l,
                                                                                              w.sgn);
  scale_cols_kernel<T><<<(unsigned)std::min<int64_t>(cdiv(n * l, 256), 8 * nsm), 256, 0, st>>>(vo, ldvo, n, l,
                                                                                              w.sgn);
  CKL("scale_cols");
  if (k < l) {
    copy2d_kernel<T><<<(unsigned)std::min<int64_t>(cdiv(m * k, 256), 8 * nsm), 256, 0, st>>>(uo, l, U, ldu, m, k,
                                                                                            nullptr);
    CKL("copy_u");
    copy2d_kernel<T><<<(unsigned)std::min<int64_t>(cdiv(n * k, 256), 8 * nsm), 256, 0, st>>>(vo, l, V, ldv, n, k,
                                                                                            nullptr);
    CKL("copy_v");
    CK(cudaMemcpyAsync(S, so, (size_t)k * sizeof(T), cudaMemcpyDeviceToDevice, st));
  }
  ffsrqr_info_t *dinfo = reinterpret_cast<ffsrqr_info_t *>(ws + P->off_info);
  info_kernel<<<1, 32, 0, st>>>(w.ctl, w.dctl, dinfo);
  CKL("info");
  if (info) CK(cudaMemcpyAsync(info, dinfo, sizeof(ffsrqr_info_t), cudaMemcpyDeviceToHost, st));
  return 0;
}

template <typename T>
void layout(ffsrqr_plan_s *P) {
  const int64_t m = P->m, n = P->n;
  const int k = P->k, s = P->s;
  const int64_t ldm = P->ldm, lds = P->lds, ldk = P->ldk;
  const int nsm = P->num_sms;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align256(off + std::max<size_t>(bytes, 1));
    return o;
  };
  const size_t E = sizeof(T);
  P->off_ctl = take(CTL_WORDS * sizeof(int));
  P->off_dctl = take(D_WORDS * sizeof(double));
  P->off_info = take(sizeof(ffsrqr_info_t));
  P->off_om = take((size_t)s * ldm * E);
  P->off_bt = take((size_t)n * lds * E);
  P->off_sel = take((size_t)n * sizeof(int));
  P->off_s11 = take((size_t)k * k * E);
  P->off_cval = take((size_t)4 * P->qrcp_grid * E);  // [2][2][G]: bests and bounds
  P->off_cidx = take((size_t)2 * P->qrcp_grid * sizeof(int));
  P->off_ccol = take((size_t)2 * P->qrcp_grid * lds * E);
  P->off_q1 = take((size_t)m * ldk * E);
  P->off_w = take((size_t)k * k * E);
  P->off_rc1 = take((size_t)k * k * E);
  P->off_rc2 = take((size_t)k * k * E);
  P->off_gt = take((size_t)n * ldk * E);
  P->off_r11 = take((size_t)k * k * E);
  P->off_rinv = take((size_t)k * k * E);
  P->off_zt = take((size_t)n * ldk * E);
  P->off_bjt = take((size_t)k * lds * E);
  P->off_cbt = take((size_t)n * lds * E);
  P->off_r = take((size_t)n * E);
  P->nblk_tn = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, 8), 2 * nsm));
  P->off_bv = take((size_t)P->nblk_tn * E);
  P->off_bi = take((size_t)P->nblk_tn * sizeof(int));
  P->off_avec = take((size_t)k * E);
  P->off_z = take((size_t)m * E);
  P->nblk_res = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(m, 64), nsm));
  P->off_hpart = take((size_t)(P->nblk_res + 1) * k * E);  // block partials of h, then h
  P->off_npart = take((size_t)P->nblk_res * E);
  P->off_vp = take((size_t)n * ldk * E);
  P->off_rz = take((size_t)k * k * E);
  P->off_tmp = take((size_t)m * ldk * E);
  P->off_yt = take((size_t)m * ldk * E);
  P->off_rt = take((size_t)k * k * E);
  P->off_t1 = take((size_t)k * k * E);
  P->off_mt = take((size_t)k * k * E);
  P->off_us = take((size_t)k * k * E);
  P->off_vs = take((size_t)k * k * E);
  P->off_qv = take(((size_t)k + 1) * round_up(k, 16 / (int)E) * E);  // reflectors + tau of the QR of M_t^T
  P->off_qg = take((size_t)k * k * E);  // Q of the QR of M_t^T
  P->off_rowk = take((size_t)n * E);
  P->off_qk = take((size_t)m * E);
  P->off_rot = take((size_t)2 * k * E);
  P->off_rd = take((size_t)k * k * E);
  P->off_xinv = take((size_t)k * k * E);
  P->off_swpart = take((size_t)P->swap_grid * std::max<int64_t>(n, k + 1) * E);
  P->off_swbv = take((size_t)P->swap_grid * E);
  P->off_swbi = take((size_t)P->swap_grid * sizeof(int));
  P->nblk_sign = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(std::max(m, n), 64), nsm));
  P->off_sgnv = take((size_t)P->nblk_sign * k * E);
  P->off_sgni = take((size_t)P->nblk_sign * k * sizeof(int));
  P->off_sgn = take((size_t)k * E);
  P->part_cap = (size_t)std::max<int64_t>((int64_t)k * k * 64, (int64_t)4 * 1024 * 1024 / E);
  P->off_part = take(P->part_cap * E);
  P->off_omb = 0;
  if (tc_mode(P->mode)) {
    const int64_t ldmax = std::max(round_up(m, 8), round_up(n, 8));
    if (P->mode == FFSRQR_MIXED_BF16X3) P->off_omb = take((size_t)s * round_up(m, 8) * 2);  // BF16 Omega
    P->off_tcpart = take((size_t)2 * nsm * TC_BM * 256 * sizeof(float));
    P->off_tt = take((size_t)k * ldmax * sizeof(float));
    P->off_bh = take((size_t)k * ldmax * sizeof(float));
    P->off_bl = take((size_t)k * ldmax * sizeof(float));
    P->off_sinv = take((size_t)k * ldk * sizeof(float));
    P->off_sh = take((size_t)256 * ldk * sizeof(float));
    P->off_sl = take((size_t)256 * ldk * sizeof(float));
    P->off_scr = take((size_t)std::max(m, n) * ldk * sizeof(float));
  } else {
    P->off_tcpart = P->off_tt = P->off_bh = P->off_bl = 0;
    P->off_sinv = P->off_sh = P->off_sl = P->off_scr = 0;
  }
  if (P->kout < k) {
    P->off_uo = off;
    off = align256(off + (size_t)m * k * E);
    P->off_so = off;
    off = align256(off + (size_t)k * E);
    P->off_vo = off;
    off = align256(off + (size_t)n * k * E);
  }
  P->ws_bytes = off;
  auto item = [&](int i, size_t o, int64_t r, int64_t c, int64_t ld) {
    P->items[i].off = o;
    P->items[i].rows = r;
    P->items[i].cols = c;
    P->items[i].ld = ld;
    P->items[i].elem = (int)E;
  };
  item(0, P->off_om, s, m, ldm);
  item(1, P->off_bt, n, s, lds);
  item(2, P->off_s11, k, k, k);
  item(3, P->off_q1, m, k, ldk);
  item(4, P->off_gt, n, k, ldk);
  item(5, P->off_vp, n, k, ldk);
  item(6, P->off_tmp, m, k, ldk);
  item(7, P->off_r, n, 1, 1);
  item(8, P->off_mt, k, k, k);
  P->items[9].off = P->off_ctl;  // the control words (int32)
  P->items[9].rows = 1;
  P->items[9].cols = CTL_WORDS;
  P->items[9].ld = CTL_WORDS;
  P->items[9].elem = 4;
}

// The QR kernels of the small SVD and the shape of the Jacobi cluster: the
// first (blocks, lanes per pair) of the list below whose slab fits the
// per-lane registers, whose blocks stay within 512 threads and whose cluster
// the device can hold.
template <typename T>
int plan_jacobi(ffsrqr_plan_s *P) {
  const int k = P->k;
  const int vn = 16 / (int)sizeof(T);
  const size_t qsmem = precond_qr_smem(k, sizeof(T));
  if (qsmem > (size_t)P->smem_optin) return FFSRQR_STATUS_UNSUPPORTED;
  // the caps are per kernel, shared by every plan: set them to the device
  // maximum less the kernel's static shared memory
  {
    const void *fns[5] = {(const void *)precond_qr_r_kernel<T>, (const void *)precond_qr_q_kernel<T>,
                          (const void *)jacobi_cluster_kernel<T, 2>, (const void *)jacobi_cluster_kernel<T, 4>,
                          (const void *)jacobi_cluster_kernel<T, 8>};
    for (const void *fn : fns) {
      CK(smem_cap_max(fn));
    }
  }
  if constexpr (sizeof(T) == 4) {
    // single precision runs the column-block cluster Jacobi
    if (jb_smem_bytes(k) + 1024 > (size_t)P->smem_optin) return FFSRQR_STATUS_UNSUPPORTED;
    CK(smem_cap_max((const void *)jacobi_blk_kernel));
    int nc = 0;
    if (launch_jacobi_blk(nullptr, nullptr, k, k, nullptr, nullptr, nullptr, nullptr, true, &nc) != cudaSuccess ||
        nc < 1) {
      (void)cudaGetLastError();
      return FFSRQR_STATUS_UNSUPPORTED;
    }
  }
  P->jac_cluster = 0;
  P->jac_lpp = 0;
  const int cand[7][2] = {{8, 2}, {8, 4}, {4, 4}, {2, 4}, {2, 8}, {4, 8}, {8, 8}};
  for (int ci = 0; ci < 7 && !P->jac_cluster; ++ci) {
    const int C = cand[ci][0], lpp = cand[ci][1];
    const JacGeom g = jac_geom(k, C, vn);
    if (cdiv(g.hb / vn, lpp) > JAC_NVL) continue;
    if (round_up((int64_t)g.npair * lpp, 32) > 512) continue;
    if (jac_cluster_smem(k, C, sizeof(T), lpp) + 1024 > (size_t)P->smem_optin) continue;
    int nc = 0;
    if (launch_jacobi_any<T>(nullptr, C, lpp, k, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, T(0), true,
                             &nc) == cudaSuccess &&
        nc >= 1) {
      P->jac_cluster = C;
      P->jac_lpp = lpp;
    } else {
      (void)cudaGetLastError();
    }
  }
  return P->jac_cluster ? 0 : FFSRQR_STATUS_UNSUPPORTED;
}

// Switch the SRQR test between the exact g2 (d = 0) and the d-row estimate,
// resizing the swap kernel's shared memory for it.
template <typename T>
int plan_g2_rows(ffsrqr_plan_s *P, int d) {
  const size_t bytes = swap_smem_bytes(P->k, d, sizeof(T));
  if (bytes > (size_t)P->smem_optin) return FFSRQR_STATUS_UNSUPPORTED;
  int per_sm = 0;
  CK(smem_cap_max((const void *)srqr_swap_kernel<T>));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, srqr_swap_kernel<T>, 512, bytes));
  if (per_sm < 1) return FFSRQR_STATUS_UNSUPPORTED;
  P->swap_smem = bytes;
  P->g2_rows = d;
  return 0;
}

template <typename T>
int plan_qrcp(ffsrqr_plan_s *P) {
  const int s = P->s;
  P->qrcp_threads = 512;
  P->qrcp_spad = (int)round_up(s, 4);
  int dev_smem = 0;
  CK(cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device));
  P->smem_optin = dev_smem;
  const size_t budget = (size_t)dev_smem - 2048;
  // slab width per block so that the slab fits; at least 16 columns per block
  int64_t grid = std::min<int64_t>(P->num_sms, std::max<int64_t>(1, cdiv(P->n, 16)));
  for (;;) {
    const int64_t cols = cdiv(P->n, grid);
    // slab, reflector, norms; single precision adds the second reflector and
    // the candidate columns of the two-pivot steps (16-byte aligned)
    const size_t need = ((size_t)cols * P->qrcp_spad + cols + P->qrcp_spad) * sizeof(T) +
                        (sizeof(T) == 4 ? (size_t)qrcp_pair_extra(P->qrcp_spad) * sizeof(T) + 16 : 0);
    if (need <= budget) {
      P->qrcp_cols = (int)cols;
      P->qrcp_smem = need;
      break;
    }
    if (grid >= P->num_sms) return FFSRQR_STATUS_UNSUPPORTED;  // sketch too large for on-chip slabs
    grid = std::min<int64_t>(P->num_sms, grid * 2);
  }
  int per_sm = 0;
  CK(smem_cap_max((const void *)qrcp_kernel<T>));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qrcp_kernel<T>, P->qrcp_threads, P->qrcp_smem));
  if (per_sm < 1) return FFSRQR_STATUS_UNSUPPORTED;
  P->qrcp_grid = (int)grid;
  // swap loop: one co-resident block of 512 threads per SM
  P->swap_smem = swap_smem_bytes(P->k, P->g2_rows, sizeof(T));
  CK(smem_cap_max((const void *)srqr_swap_kernel<T>));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, srqr_swap_kernel<T>, 512, P->swap_smem));
  if (per_sm < 1) return FFSRQR_STATUS_UNSUPPORTED;
  P->swap_grid = P->num_sms;
  return 0;
}

// The plan for checked arguments: SRQR depth k, returned rank kout, TRQRCP
// block size b (the sketch has b + p rows).
int plan_create(ffsrqr_plan_t *plan, int64_t m, int64_t n, int32_t kout, int32_t k, int32_t b, int32_t p,
                int32_t mode, const ffsrqr_opts_t *opts, size_t *workspace_bytes) {
  const int elem = (mode == FFSRQR_FP64) ? 8 : 4;
  // the k x k factors live in one block's shared memory, and the row solves
  // hold at most 7 x 32 columns per lane group
  if ((size_t)k * k * elem > 200 * 1024 || k > 224) return FFSRQR_STATUS_UNSUPPORTED;
  ffsrqr_plan_s *P = new (std::nothrow) ffsrqr_plan_s();
  if (!P) return FFSRQR_STATUS_WORKSPACE;
  P->m = m;
  P->n = n;
  P->k = k;
  P->kout = kout;
  P->rsi_q = -1;  // Flip-Flop SRQR unless ffsrqr_plan_rsi says otherwise
  P->p = p;
  P->s = b + p;
  P->blk = b;
  P->mode = mode;
  P->g = opts ? opts->g : 2.0;
  P->max_swaps = opts ? opts->max_swaps : 4 * k;
  P->flags = opts ? opts->flags : 0;
  P->elem = elem;
  P->ldm = round_up(m, 4);
  P->ldn = round_up(n, 4);
  P->lds = round_up(P->s, 4);
  P->ldk = round_up(k, 4);
  if (!cuda_ok(cudaGetDevice(&P->device), "cudaGetDevice") ||
      !cuda_ok(cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device),
               "cudaDeviceGetAttribute")) {
    delete P;
    return FFSRQR_STATUS_CUDA;
  }
  int rc = (elem == 8) ? plan_qrcp<double>(P) : plan_qrcp<float>(P);
  if (!rc) rc = (elem == 8) ? plan_jacobi<double>(P) : plan_jacobi<float>(P);
  if (!rc && !(cuda_ok(cudaStreamCreateWithFlags(&P->side, cudaStreamNonBlocking), "cudaStreamCreate") &&
               cuda_ok(cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming), "cudaEventCreate") &&
               cuda_ok(cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming), "cudaEventCreate")))
    rc = FFSRQR_STATUS_CUDA;
  if (rc) {
    if (P->side) cudaStreamDestroy(P->side);
    if (P->ev_fork) cudaEventDestroy(P->ev_fork);
    if (P->ev_join) cudaEventDestroy(P->ev_join);
    delete P;
    return rc;
  }
  P->ev_ok = false;
  if (P->flags & FFSRQR_FLAG_PHASE_TIMES) {
    bool ok = true;
    for (int e = 0; e < 2; ++e) {
      for (int i = 0; i < 13 && ok; ++i) ok = cuda_ok(cudaEventCreate(&P->ev[e][i]), "cudaEventCreate");
      for (int i = 0; i < 6 && ok; ++i)
        ok = cuda_ok(cudaEventCreate(&P->ev_tc[e][i / 2][i % 2]), "cudaEventCreate");
    }
    if (!ok) {
      ffsrqr_destroy(P);
      return FFSRQR_STATUS_CUDA;
    }
    P->ev_ok = true;
  }
  if (elem == 8) layout<double>(P);
  else layout<float>(P);
  *workspace_bytes = P->ws_bytes;
  *plan = P;
  return 0;
}

}  // namespace

extern "C" {

int ffsrqr_plan(ffsrqr_plan_t *plan, int64_t m, int64_t n, int32_t k, int32_t p, int32_t mode,
                const ffsrqr_opts_t *opts, size_t *workspace_bytes) {
  return ffsrqr_plan_l(plan, m, n, k, k, p, mode, opts, workspace_bytes);
}

int ffsrqr_plan_blocked(ffsrqr_plan_t *plan, int64_t m, int64_t n, int32_t k, int32_t b, int32_t p, int32_t mode,
                        const ffsrqr_opts_t *opts, size_t *workspace_bytes) {
  if (!plan) return -1;
  *plan = nullptr;
  if (m < 1 || m > (int64_t)INT32_MAX) return -2;
  if (n < 1 || n > (int64_t)INT32_MAX) return -3;
  if (k < 1 || k > n || k > m) return -4;
  if (b < 1 || b > k || (b < k && b % 8 != 0)) return -5;
  if (p < 0 || (int64_t)b + p > m || b + p > 256) return -6;
  if (mode != FFSRQR_PLAIN_FP32 && mode != FFSRQR_MIXED && mode != FFSRQR_MIXED_BF16X3 && mode != FFSRQR_FP64)
    return -7;
  if (opts && !(opts->g > 1.0)) return -8;
  if (opts && opts->max_swaps < 0) return -8;
  if (!workspace_bytes) return -9;
  return plan_create(plan, m, n, k, k, b, p, mode, opts, workspace_bytes);
}

int ffsrqr_plan_l(ffsrqr_plan_t *plan, int64_t m, int64_t n, int32_t kout, int32_t k, int32_t p, int32_t mode,
                  const ffsrqr_opts_t *opts, size_t *workspace_bytes) {
  // here k is Alg. 9's SRQR depth l and kout its target rank; the checks
  // below use ffsrqr_plan's argument numbers, shifted by one after kout
  if (!plan) return -1;
  *plan = nullptr;
  if (kout < 1 || kout > k) {
    if (k >= 1 && kout > k) return -5;
    return -4;
  }
  if (m < 1 || m > (int64_t)INT32_MAX) return -2;
  if (n < 1 || n > (int64_t)INT32_MAX) return -3;
  const int sh = (kout == k) ? 0 : 1;  // ffsrqr_plan has no l argument
  if (k < 1 || k > n || k > m) return -4 - sh;
  if (p < 0 || (int64_t)k + p > m || k + p > 256) return -5 - sh;
  if (mode != FFSRQR_PLAIN_FP32 && mode != FFSRQR_MIXED && mode != FFSRQR_MIXED_BF16X3 && mode != FFSRQR_FP64)
    return -6 - sh;
  if (opts && !(opts->g > 1.0)) return -7 - sh;
  if (opts && opts->max_swaps < 0) return -7 - sh;
  if (!workspace_bytes) return -8 - sh;
  return plan_create(plan, m, n, kout, k, k, p, mode, opts, workspace_bytes);
}

int ffsrqr_run(ffsrqr_plan_t plan, const void *A, int64_t lda, uint64_t seed, void *U, int64_t ldu,
               void *S, void *V, int64_t ldv, int32_t *piv, void *workspace, void *stream,
               ffsrqr_info_t *info) {
  if (!plan) return -1;
  if (!A) return -2;
  if (lda < plan->n) return -3;
  if (!U) return -5;
  if (ldu < plan->kout) return -6;
  if (!S) return -7;
  if (!V) return -8;
  if (ldv < plan->kout) return -9;
  if (!piv) return -10;
  if (!workspace || ((uintptr_t)workspace & 255u)) return -11;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  unsigned char *ws = reinterpret_cast<unsigned char *>(workspace);
  g_launches = 0;
  plan->evset = (int)(plan->runs & 1);
  ++plan->runs;
  int rc;
  if (plan->rsi_q >= 0) {
    if (plan->elem == 8)
      rc = run_rsi<double>(plan, (const double *)A, lda, seed, (double *)U, ldu, (double *)S, (double *)V, ldv, ws,
                           st, info);
    else
      rc = run_rsi<float>(plan, (const float *)A, lda, seed, (float *)U, ldu, (float *)S, (float *)V, ldv, ws, st,
                          info);
  } else if (plan->kout < plan->k) {
    // depth l > k: the pipeline runs at depth l into the workspace, and the
    // leading k singular triplets (S is descending) are copied out
    if (plan->elem == 8)
      rc = run_truncated<double>(plan, (const double *)A, lda, seed, (double *)U, ldu, (double *)S, (double *)V,
                                 ldv, piv, ws, st, info);
    else
      rc = run_truncated<float>(plan, (const float *)A, lda, seed, (float *)U, ldu, (float *)S, (float *)V, ldv,
                                piv, ws, st, info);
  } else if (plan->elem == 8) {
    rc = run_impl<double>(plan, (const double *)A, lda, seed, (double *)U, ldu, (double *)S, (double *)V,
                          ldv, piv, ws, st, info);
  } else {
    rc = run_impl<float>(plan, (const float *)A, lda, seed, (float *)U, ldu, (float *)S, (float *)V, ldv,
                         piv, ws, st, info);
  }
  plan->launches = g_launches;
  return rc;
}

int ffsrqr_plan_set_g2_rows(ffsrqr_plan_t plan, int32_t d) {
  if (!plan) return -1;
  if (d < 0 || d > G2EST_MAX_D) return -2;
  if (plan->rsi_q >= 0) return FFSRQR_STATUS_UNSUPPORTED;
  return plan->mode == FFSRQR_FP64 ? plan_g2_rows<double>(plan, d) : plan_g2_rows<float>(plan, d);
}

int ffsrqr_plan_tune(ffsrqr_plan_t plan, const void *A, int64_t lda, uint64_t seed, void *U, int64_t ldu,
                     void *S, void *V, int64_t ldv, int32_t *piv, void *workspace, void *stream,
                     int32_t *config, float *ms_best) {
  if (!plan) return -1;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return FFSRQR_STATUS_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return FFSRQR_STATUS_CUDA;
  }
  // one warm-up and two timed runs per configuration
  auto time_runs = [&](float *ms) -> int {
    int rc = ffsrqr_run(plan, A, lda, seed, U, ldu, S, V, ldv, piv, workspace, stream, nullptr);
    if (rc) return rc;
    if (cudaEventRecord(e0, st) != cudaSuccess) return FFSRQR_STATUS_CUDA;
    for (int r = 0; r < 2 && !rc; ++r) rc = ffsrqr_run(plan, A, lda, seed, U, ldu, S, V, ldv, piv, workspace, stream,
                                                       nullptr);
    if (rc) return rc;
    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
      return FFSRQR_STATUS_CUDA;
    *ms *= 0.5f;
    return 0;
  };
  int rc = 0;
  float best = 0.f;
  for (int site = 0; site < 4; ++site) plan->tc_stages[site] = plan->tc_grid[site] = plan->tc_sk[site] = 0;
  rc = time_runs(&best);
  // coordinate descent over the sites: for each pass over A the schedule
  // (data-parallel tiles first, or all stream-K) and the pipeline depth (all
  // the stages its shared memory holds, or one or two fewer), and the
  // stream-K grid of the Grams (all SMs, a half, a quarter); a candidate is
  // kept only when the whole run got faster
  for (int site = 0; site < 3 && !rc; ++site) {
    plan->tc_sk[site] = 1;
    float t = 0.f;
    rc = time_runs(&t);
    if (!rc && t < best) best = t;
    else plan->tc_sk[site] = 0;
  }
  for (int site = 0; site < 4 && !rc; ++site) {
    for (int c = 1; c <= 2 && !rc; ++c) {
      const int keep_s = plan->tc_stages[site], keep_g = plan->tc_grid[site];
      if (site < 3) {
        const int d = plan->tc_stages_fit[site];
        if (d - c < 2) break;
        plan->tc_stages[site] = d - c;
      } else {
        plan->tc_grid[site] = std::max(1, plan->num_sms >> c);
      }
      float t = 0.f;
      rc = time_runs(&t);
      if (!rc && t < best) {
        best = t;
      } else {
        plan->tc_stages[site] = keep_s;
        plan->tc_grid[site] = keep_g;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) {
    for (int site = 0; site < 4; ++site) plan->tc_stages[site] = plan->tc_grid[site] = plan->tc_sk[site] = 0;
    return rc;
  }
  if (config) {
    for (int site = 0; site < 3; ++site) config[site] = plan->tc_stages[site];
    config[3] = plan->tc_grid[3];
    for (int site = 0; site < 3; ++site) config[4 + site] = plan->tc_sk[site];
  }
  if (ms_best) *ms_best = best;
  return 0;
}

}  // extern "C"

namespace {

template <typename T>
int project_impl(ffsrqr_plan_s *P, const T *A, int64_t lda, const T *X, int64_t ldx, T *Gt, int64_t ldg,
                 unsigned char *ws, cudaStream_t st) {
  WsPtrs<T> w = ws_ptrs<T>(P, ws);
  const int64_t m = P->m, n = P->n, ldk = P->ldk;
  const int k = P->k, nsm = P->num_sms;
  int rc;
  CK(cudaMemsetAsync(ws + P->off_ctl, 0, CTL_WORDS * sizeof(int), st));
  copy2d_kernel<T><<<(unsigned)std::min<int64_t>(cdiv(m * k, 256), 8 * nsm), 256, 0, st>>>(X, ldx, w.q1, ldk, m,
                                                                                          k, nullptr);
  CKL("copy_x");
  if (use_tc<T>(P, A, lda)) {
    if ((rc = tc_thin_pass(st, P, ws, true, (const float *)A, lda, (const float *)w.q1, m, (float *)w.gt)))
      return rc;
    copy2d_kernel<T><<<(unsigned)std::min<int64_t>(cdiv(n * k, 256), 8 * nsm), 256, 0, st>>>(w.gt, ldk, Gt, ldg,
                                                                                            n, k, nullptr);
    CKL("copy_gt");
    return 0;
  }
  return launch_gemm<T>(st, P, ws, (int)n, k, (int)m, A, lda, true, w.q1, ldk, true, Gt, ldg);
}

}  // namespace

// Gt (n x k, leading dimension ldg) = A^T X for A (m x n, lda) and X (m x k,
// ldx) with the plan's pass-2 product: the three-product TF32 split on the
// tensor cores in FFSRQR_MIXED when A is TMA-addressable, the CUDA cores
// otherwise.  The mode products of the HOSVD core (Alg. 5) use it.  Writes
// the number of kernels enqueued to *launches.
int ffq_project(ffsrqr_plan_t P, const void *A, int64_t lda, const void *X, int64_t ldx, void *Gt, int64_t ldg,
                void *workspace, cudaStream_t st, int *launches) {
  g_launches = 0;
  unsigned char *ws = reinterpret_cast<unsigned char *>(workspace);
  int rc;
  if (P->elem == 8)
    rc = project_impl<double>(P, (const double *)A, lda, (const double *)X, ldx, (double *)Gt, ldg, ws, st);
  else
    rc = project_impl<float>(P, (const float *)A, lda, (const float *)X, ldx, (float *)Gt, ldg, ws, st);
  *launches = g_launches;
  return rc;
}

// X (m x n, ldx) = U V^T over the first r columns of U (m x r, ldu) and V
// (n x r, ldv), on the CUDA cores (r <= the plan's k), for the singular value
// thresholding step of the robust PCA driver (Alg. 7).  Writes the number of
// kernels enqueued to *launches.
int ffq_gemm_nt(ffsrqr_plan_t P, int64_t m, int64_t n, int r, const void *U, int64_t ldu, const void *V,
                int64_t ldv, void *X, int64_t ldx, void *workspace, cudaStream_t st, int *launches) {
  g_launches = 0;
  unsigned char *ws = reinterpret_cast<unsigned char *>(workspace);
  int rc;
  if (P->elem == 8)
    rc = launch_gemm<double>(st, P, ws, (int)m, (int)n, r, (const double *)U, ldu, false, (const double *)V, ldv,
                             false, (double *)X, ldx);
  else
    rc = launch_gemm<float>(st, P, ws, (int)m, (int)n, r, (const float *)U, ldu, false, (const float *)V, ldv,
                            false, (float *)X, ldx);
  *launches = g_launches;
  return rc;
}

// Phase-batched runs.  A batch graph or a server group runs part 1 (everything
// before the small SVD) of several problems, one launch of their small SVDs,
// then part 2.  Only plans whose small SVD is the single-precision cluster
// Jacobi take part (FP32 arithmetic, SRQR depth l = k, not the subspace
// iteration); every result is bitwise the one ffsrqr_run gives.
bool ffq_phase_batchable(ffsrqr_plan_t P) { return P && P->elem == 4 && P->rsi_q < 0 && P->kout == P->k; }

int ffq_run_pre(ffsrqr_plan_t P, const void *A, int64_t lda, uint64_t seed, int32_t *piv, void *workspace,
                cudaStream_t st) {
  if (!ffq_phase_batchable(P)) return -1;
  if (!A || lda < P->n || !piv || !workspace || ((uintptr_t)workspace & 255u)) return -2;
  P->evset = (int)(P->runs & 1);
  ++P->runs;
  return run_pre<float>(P, (const float *)A, lda, seed, piv, reinterpret_cast<unsigned char *>(workspace), st);
}

int ffq_run_post(ffsrqr_plan_t P, const void *A, int64_t lda, void *U, int64_t ldu, void *V, int64_t ldv,
                 int32_t *piv, void *workspace, cudaStream_t st, ffsrqr_info_t *info) {
  if (!ffq_phase_batchable(P)) return -1;
  if (!A || !U || ldu < P->k || !V || ldv < P->k || !piv || !workspace) return -2;
  return run_post<float>(P, (const float *)A, lda, (float *)U, ldu, (float *)V, ldv, piv,
                         reinterpret_cast<unsigned char *>(workspace), st, info);
}

// The small SVDs of count phase-batchable problems (after their part 1, in
// stream order): one jacobi_blk_batch_kernel launch per cluster size and
// JB_BATCH_MAX problems.  S[i] is problem i's singular-value output.  Writes
// the number of launches to *launches.
int ffq_small_svd_batched(const ffsrqr_plan_t *plans, void *const *workspaces, void *const *S, int count,
                          cudaStream_t st, int *launches) {
  int nl = 0;
  std::vector<char> done(count, 0);
  for (int i0 = 0; i0 < count; ++i0) {
    if (done[i0]) continue;
    const int C = jb_cluster_for(plans[i0]->k);
    std::vector<int> grp;
    for (int i = i0; i < count; ++i)
      if (!done[i] && jb_cluster_for(plans[i]->k) == C) {
        grp.push_back(i);
        done[i] = 1;
      }
    for (size_t g0 = 0; g0 < grp.size(); g0 += JB_BATCH_MAX) {
      const int ng = (int)std::min<size_t>(JB_BATCH_MAX, grp.size() - g0);
      JbBatch jb{};
      jb.count = ng;
      jb.max_sweeps = JB_MAX_SWEEPS;
      int nw = 1;
      size_t smem = 0;
      for (int e = 0; e < ng; ++e) {
        ffsrqr_plan_s *P = plans[grp[g0 + e]];
        if (!ffq_phase_batchable(P)) return -1;
        const int k = P->k;
        WsPtrs<float> w = ws_ptrs<float>(P, reinterpret_cast<unsigned char *>(workspaces[grp[g0 + e]]));
        JbProblem &q = jb.p[e];
        q.M = w.mt;
        q.U = w.us;
        q.S = reinterpret_cast<float *>(S[grp[g0 + e]]);
        q.V = w.vs;
        q.ctl = w.ctl;
        q.k = k;
        q.ldm = k;
        q.tol = 4.f * sqrtf((float)k) * 5.9604645e-8f;  // as launch_jacobi_blk
        nw = std::max(nw, jb_geom(k, C).nw);
        smem = std::max(smem, jb_smem_bytes(k));
      }
      CK(smem_cap_max((const void *)jacobi_blk_batch_kernel));
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = (unsigned)C;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3((unsigned)(ng * C));
      cfg.blockDim = dim3((unsigned)(32 * nw));
      cfg.dynamicSmemBytes = smem;
      cfg.stream = st;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      CK(cudaLaunchKernelEx(&cfg, jacobi_blk_batch_kernel, jb));
      ++nl;
    }
  }
  if (launches) *launches = nl;
  return 0;
}

extern "C" {

int ffsrqr_plan_rsi(ffsrqr_plan_t *plan, int64_t m, int64_t n, int32_t k, int32_t p, int32_t q, int32_t mode,
                    const ffsrqr_opts_t *opts, size_t *workspace_bytes) {
  if (!plan) return -1;
  *plan = nullptr;
  if (m < 1 || m > (int64_t)INT32_MAX) return -2;
  if (n < 1 || n > (int64_t)INT32_MAX) return -3;
  if (k < 1 || k > n || k > m) return -4;
  if (p < 0 || (int64_t)k + p > std::min(m, n)) return -5;
  if (q < 0) return -6;
  if (mode != FFSRQR_PLAIN_FP32 && mode != FFSRQR_MIXED && mode != FFSRQR_MIXED_BF16X3 && mode != FFSRQR_FP64)
    return -7;
  if (opts && (!(opts->g > 1.0) || opts->max_swaps < 0)) return -8;
  if (!workspace_bytes) return -9;
  // a plan at width l = k + p (no sketch oversampling of its own) whose
  // outputs are cut to k columns
  const int rc = ffsrqr_plan_l(plan, m, n, k, k + p, 0, mode, opts, workspace_bytes);
  if (rc < 0) return -5;
  if (rc > 0) return rc;
  (*plan)->rsi_q = q;
  return 0;
}

int ffsrqr_plan_depth(ffsrqr_plan_t plan) {
  if (!plan) return -1;
  return plan->k;
}

int ffsrqr_plan_shape(ffsrqr_plan_t plan, int64_t *m, int64_t *n, int32_t *k, int32_t *p, int32_t *mode) {
  if (!plan) return -1;
  if (m) *m = plan->m;
  if (n) *n = plan->n;
  if (k) *k = plan->kout;
  if (p) *p = plan->p;
  if (mode) *mode = plan->mode;
  return 0;
}

int ffsrqr_destroy(ffsrqr_plan_t plan) {
  if (!plan) return -1;
  if (plan->side) {
    cudaStreamSynchronize(plan->side);
    cudaStreamDestroy(plan->side);
  }
  if (plan->ev_fork) cudaEventDestroy(plan->ev_fork);
  if (plan->ev_join) cudaEventDestroy(plan->ev_join);
  if (plan->ev_ok) {
    for (int e = 0; e < 2; ++e) {
      for (int i = 0; i < 13; ++i) cudaEventDestroy(plan->ev[e][i]);
      for (int i = 0; i < 6; ++i) cudaEventDestroy(plan->ev_tc[e][i / 2][i % 2]);
    }
  }
  delete plan;
  return 0;
}

const char *ffsrqr_status_string(int code) {
  switch (code) {
    case 0: return "ok";
    case FFSRQR_STATUS_RANK_DEFICIENT: return "rank deficient (zero pivot norm or singular factor)";
    case FFSRQR_STATUS_SWAP_CAP: return "SRQR swap cap reached with g2 > g";
    case FFSRQR_STATUS_TIMEOUT: return "bounded device wait expired";
    case FFSRQR_STATUS_NONFINITE: return "input contains Inf or NaN";
    case FFSRQR_STATUS_WORKSPACE: return "workspace too small or admission refused";
    case FFSRQR_STATUS_CUDA: return "CUDA API error";
    case FFSRQR_STATUS_UNSUPPORTED: return "size not supported by this build";
    default: break;
  }
  if (code < 0) return "invalid argument";
  return "unknown status";
}

const char *ffsrqr_last_cuda_error(void) { return g_last_cuda_error.c_str(); }

int ffsrqr_phase_times_back(ffsrqr_plan_t plan, int32_t back, float *ms, int32_t cap) {
  if (!plan) return -1;
  if (!plan->ev_ok) return -2;
  if (back < 0 || back > 1 || plan->runs <= back) return -3;
  if (!ms && cap > 0) return -4;
  const int e = (int)((plan->runs - 1 - back) & 1);
  // host wait for that run's last event (the next run may still execute)
  if (cudaEventSynchronize(plan->ev[e][12]) != cudaSuccess) return FFSRQR_STATUS_CUDA;
  int cnt = 0;
  for (int i = 0; i < 12 && cnt < cap; ++i, ++cnt) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, plan->ev[e][i], plan->ev[e][i + 1]) != cudaSuccess) t = -1.f;
    ms[cnt] = t;
  }
  for (int i = 0; i < 3 && cnt < cap; ++i, ++cnt) {
    float t = -1.f;
    if (tc_mode(plan->mode) &&
        cudaEventElapsedTime(&t, plan->ev_tc[e][i][0], plan->ev_tc[e][i][1]) != cudaSuccess)
      t = -1.f;
    ms[cnt] = t;
  }
  return cnt;
}

int ffsrqr_phase_times(ffsrqr_plan_t plan, float *ms, int32_t cap) {
  if (!plan) return -1;
  if (!plan->ev_ok) return -2;
  if (plan->runs < 1) return -3;
  return ffsrqr_phase_times_back(plan, 0, ms, cap);
}

int ffsrqr_launch_count(ffsrqr_plan_t plan) {
  if (!plan) return -1;
  return plan->launches;
}

int ffsrqr_workspace_item(ffsrqr_plan_t plan, int32_t what, size_t *offset, int64_t *rows,
                          int64_t *cols, int64_t *ld, int32_t *elem_bytes) {
  if (!plan) return -1;
  if (what < 0 || what > 9) return -2;
  const Item &it = plan->items[what];
  if (offset) *offset = it.off;
  if (rows) *rows = it.rows;
  if (cols) *cols = it.cols;
  if (ld) *ld = it.ld;
  if (elem_bytes) *elem_bytes = it.elem;
  return 0;
}

int ffsrqr_philox4x32_10(const uint32_t *ctr_key, uint32_t *out, int32_t count, void *stream) {
  if (!ctr_key) return -1;
  if (!out) return -2;
  if (count < 0) return -3;
  if (count == 0) return 0;
  philox_raw_kernel<<<(unsigned)cdiv(count, 128), 128, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      ctr_key, out, count);
  CKL("philox_raw");
  return 0;
}

}  // extern "C"
