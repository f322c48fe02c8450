/*
 * ffsrqr.h -- C ABI of the GB300 (sm_103a) Flip-Flop SRQR library.
 *
 * Flip-Flop Spectrum-Revealing QR (Feng, Xiao & Gu, arXiv 1803.01982,
 * Alg. 9) computes a rank-k approximate SVD  A ~= U diag(S) V^T  of a dense
 * m x n matrix:
 *   sketch B = Omega A                       (Alg. 2, Omega ~ N(0,1)^{(k+p) x m})
 *   partial QRCP of B for k steps -> Pi      (Alg. 1 on the sketch, Alg. 2)
 *   QR of the pivoted panel A Pi(:,1:k)      (Alg. 2)
 *   (R11 R12) = Q1^T A Pi                    (Eq. RRQR)
 *   SRQR test / swaps on R11^{-1}R12 and the trailing norms (Alg. 4)
 *   QR of (R11 R12)^T -> Qhat1              (Alg. 9)
 *   tmp = A Pi Qhat1, svd(tmp) -> U, S, V    (Alg. 9)
 * All entry points take plain pointers and sizes; no C++ or framework types.
 *
 * Conventions
 *   - Matrices are row-major.  A is m x n with leading dimension lda >= n.
 *   - Device pointers are CUDA device addresses on the plan's device; host
 *     pointers are ordinary (preferably pinned) host memory.
 *   - Return codes: 0 = success; -i = argument i is invalid (LAPACK style);
 *     positive codes are the FFSRQR_STATUS_* values below (numerical status,
 *     reported through ffsrqr_info_t once the stream has been synchronised).
 *   - Nothing here allocates device memory except where stated: the caller
 *     owns A, the outputs and the workspace.
 */
#ifndef FFSRQR_H
#define FFSRQR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ffsrqr_plan_s *ffsrqr_plan_t;

/* Arithmetic modes (the precision layer).
 *   FFSRQR_PLAIN_FP32:   every product in FP32 on the CUDA cores (FFMA).
 *   FFSRQR_MIXED_TF32X3: the sketch B = Omega A on the tensor cores in TF32
 *                        (one product; the sketch only chooses pivots), the
 *                        two accuracy-bearing passes (Q1^T A and A Pi Qhat1)
 *                        on the tensor cores as a three-product TF32 split
 *                        that recovers FP32 accuracy; everything else FP32.
 *                        FFSRQR_MIXED is the same value.
 *   FFSRQR_MIXED_BF16X3: the sketch in BF16 (one product), the two passes as
 *                        a three-product split-BF16 (head x head + head x
 *                        tail + tail x head, FP32 accumulate: about 2^-16
 *                        per product, random, so sigma stays within the FP32
 *                        tolerances); BF16 runs the tensor cores at twice the
 *                        TF32 rate, so the passes are bound by HBM, not by
 *                        the three products.  The Grams and small products
 *                        stay three-product TF32.
 *   FFSRQR_FP64:         everything in FP64 on the CUDA cores (A, U, S, V are
 *                        double). */
#define FFSRQR_PLAIN_FP32 0
#define FFSRQR_MIXED_TF32X3 1
#define FFSRQR_MIXED 1
#define FFSRQR_MIXED_BF16X3 2
#define FFSRQR_FP64 3

/* Numerical status codes (ffsrqr_info_t.status and positive return codes). */
#define FFSRQR_STATUS_OK 0
#define FFSRQR_STATUS_RANK_DEFICIENT 1 /* zero pivot norm / singular R11; results still written */
#define FFSRQR_STATUS_SWAP_CAP 2       /* Alg. 4's swap loop hit max_swaps with g2 > g */
#define FFSRQR_STATUS_TIMEOUT 3        /* a bounded device-side wait expired */
#define FFSRQR_STATUS_NONFINITE 4      /* A contains Inf/NaN */
#define FFSRQR_STATUS_WORKSPACE 5      /* workspace too small / admission refused */
#define FFSRQR_STATUS_CUDA 6           /* a CUDA API call failed (see ffsrqr_last_cuda_error) */
#define FFSRQR_STATUS_UNSUPPORTED 7    /* size outside what this build supports */

/* Options (NULL -> defaults g = 2.0, max_swaps = 4k, flags = 0).
 * g is the SRQR tolerance for g2 (Alg. 4, "a small number greater than one,
 * like 2.0" in Sec. 2.2); max_swaps caps Alg. 4's while loop. */
typedef struct {
  double g;
  int32_t max_swaps;
  int32_t flags;
} ffsrqr_opts_t;

/* opts.flags bits */
#define FFSRQR_FLAG_CHECK_FINITE 1 /* scan A for Inf/NaN first (one extra read of A) */
#define FFSRQR_FLAG_PHASE_TIMES 2  /* record CUDA events between pipeline phases */
/* Failure injection for testing the device-side failure detection: the grid
 * barrier of the sketch QRCP's last step waits for one block more than the
 * grid holds, so that wait expires (after about a second) and the run
 * reports FFSRQR_STATUS_TIMEOUT; the outputs of such a run are not
 * meaningful.  Nothing faults or hangs: every later kernel still runs to its
 * own bounds, and the next run on the same context is unaffected. */
#define FFSRQR_FLAG_TEST_STALL 4

/* Per-run report, written by a device->host copy enqueued at the end of
 * ffsrqr_run; valid after the stream has been synchronised.
 *   g2_first / g2_final: g2 = |alpha| ||Rtilde^{-T}||_{1,2} (Eq. for g1, g2 in
 *   Sec. 2.2) before and after the swap loop; cand_first: original index of the
 *   first SRQR candidate column; alpha_first: its residual norm. */
typedef struct {
  int32_t status;
  int32_t swaps;
  double g2_first;
  double g2_final;
  int32_t cand_first;
  int32_t jacobi_sweeps;
  double alpha_first;
} ffsrqr_info_t;

/* Create a plan for m x n inputs, target rank k and oversampling p (the sketch
 * has s = k + p rows; the paper's block size b = k and SRQR depth l = k).
 * Requirements: 1 <= k <= n, k <= m, p >= 0, k + p <= m, k + p <= 256.
 * mode is one of FFSRQR_*; opts may be NULL.  On success *workspace_bytes is
 * the size of the device workspace ffsrqr_run needs (256-byte aligned).
 * The plan holds only host metadata; it is bound to the current CUDA device.
 * Errors: -1 plan NULL, -2 m, -3 n, -4 k, -5 p, -6 mode, -7 opts, -8
 * workspace_bytes NULL; FFSRQR_STATUS_UNSUPPORTED for sizes this build does
 * not handle (the k x k factors live in one block's shared memory: k <= 224
 * in FP32 and the mixed mode, k <= 160 in FP64); FFSRQR_STATUS_CUDA if the
 * device query fails. */
int ffsrqr_plan(ffsrqr_plan_t *plan, int64_t m, int64_t n, int32_t k, int32_t p, int32_t mode,
                const ffsrqr_opts_t *opts, size_t *workspace_bytes);

/* The same with Alg. 9's SRQR depth l >= k as an argument (Sec. 3.2: "l is
 * usually a little larger than k, like l = k + 5"): SRQR runs to l steps on
 * the sketch of l + p rows, V' has l columns, the SVD of A Pi Qhat_1 (m x l)
 * is computed, and its leading k singular triplets are returned.  ffsrqr_plan
 * is this with l = k.  Requirements as ffsrqr_plan's with l in place of k,
 * and 1 <= k <= l.  The workspace adds the depth-l U, S and V.  Errors: -1
 * plan NULL, -2 m, -3 n, -4 k, -5 l, -6 p, -7 mode, -8 opts, -9
 * workspace_bytes NULL, and the statuses of ffsrqr_plan. */
int ffsrqr_plan_l(ffsrqr_plan_t *plan, int64_t m, int64_t n, int32_t k, int32_t l, int32_t p, int32_t mode,
                  const ffsrqr_opts_t *opts, size_t *workspace_bytes);

/* The same with TRQRCP's block size b (Alg. 2) as an argument: the sketch has
 * b + p rows, and the k pivots are chosen block by block.  For the block at
 * positions jb..jb+bb-1 (bb = min(b, k - jb)): partial QRCP (Alg. 1) for bb
 * steps on the current sample, the columns selected earlier excluded; the
 * block's columns of A, orthogonalised against the earlier blocks' Q1 and
 * factored ("QR on A(j:m, j:j+b-1)"); one pass over A for that block's rows
 * of R = Q1^T A Pi; and, except after the last block, the sample update
 * ("Update B(:, j+b:n)") B <- B - B(:, J) R_JJ^{-1} R(J, :), which keeps the
 * sample equal to Omega (I - Q1 Q1^T) A.  The SRQR test, the swap loop and
 * the rest of Alg. 9 are as in ffsrqr_plan (whose case is b = k); A is read
 * 1 + ceil(k / b) + 1 times instead of three.  Requirements: those of
 * ffsrqr_plan with b + p in place of k + p, 1 <= b <= k, and b a multiple of
 * 8 when b < k (each block's first column keeps 32-byte row alignment).
 * Errors: -1 plan NULL, -2 m, -3 n, -4 k, -5 b, -6 p, -7 mode, -8 opts, -9
 * workspace_bytes NULL, and the statuses of ffsrqr_plan. */
int ffsrqr_plan_blocked(ffsrqr_plan_t *plan, int64_t m, int64_t n, int32_t k, int32_t b, int32_t p, int32_t mode,
                        const ffsrqr_opts_t *opts, size_t *workspace_bytes);

/* A plan that ffsrqr_run executes as approximate SVD by randomized subspace
 * iteration (the paper's appendix algorithm, the method Sec. 3.2 compares
 * against) with l = k + p columns and q iterations, on the same kernels:
 * Omega (n x l, Philox stream 0, element (i, j) = draw i l + j), Q = orth(A
 * Omega); q times V' = orth(A^T Q), Q = orth(A V'); then A^T Q = V' R,
 * svd(R^T) = W S Z^T, U = Q W, V = V' Z, the leading k triplets (sign rule as
 * Alg. 9).  orth() is CholeskyQR2, exact in exact arithmetic for any full-rank
 * input and reliable in FP32 up to cond(A Omega) of about 1e4.  piv is not
 * written.  Requirements: 1 <= k, k + p <= min(m, n), q >= 0, k + p <= 224
 * (FP32) / 160 (FP64).  Errors: -1 plan NULL, -2 m, -3 n, -4 k, -5 p, -6 q,
 * -7 mode, -8 opts, -9 workspace_bytes NULL, and ffsrqr_plan's statuses. */
int ffsrqr_plan_rsi(ffsrqr_plan_t *plan, int64_t m, int64_t n, int32_t k, int32_t p, int32_t q, int32_t mode,
                    const ffsrqr_opts_t *opts, size_t *workspace_bytes);

/* SRQR depth l of a plan (k for plans made by ffsrqr_plan); -1 for NULL. */
int ffsrqr_plan_depth(ffsrqr_plan_t plan);

/* Run Alg. 9 on A (device, m x n, row-major, lda >= n; FP32, or FP64 in
 * FFSRQR_FP64 mode) and write
 *   U   (device, m x k, row-major, ldu >= k),
 *   S   (device, k, descending),
 *   V   (device, n x k, row-major, ldv >= k),
 *   piv (device, int32[n]): piv[0:l] = the final selected columns of A (0-based,
 *        in R order; l = k unless planned by ffsrqr_plan_l); piv[l:n] = the
 *        remaining columns in ascending order.
 * Omega is generated on the device from seed (Philox4x32-10, stream 0).
 * workspace: device, >= the size reported by ffsrqr_plan, 256-byte aligned.
 * stream: a cudaStream_t (NULL = legacy default stream).  The call only
 * enqueues work; A is read-only.  info (may be NULL): host pointer, filled by
 * an asynchronous copy (use pinned memory), valid after stream sync.
 * Errors: -1 plan, -2 A, -3 lda, -5 U, -6 ldu, -7 S, -8 V, -9 ldv, -10 piv,
 * -11 workspace; FFSRQR_STATUS_CUDA if a launch fails. */
int ffsrqr_run(ffsrqr_plan_t plan, const void *A, int64_t lda, uint64_t seed, void *U, int64_t ldu,
               void *S, void *V, int64_t ldv, int32_t *piv, void *workspace, void *stream,
               ffsrqr_info_t *info);

/* Destroy a plan (host memory only).  Returns 0, or -1 for NULL. */
int ffsrqr_destroy(ffsrqr_plan_t plan);

/* Static description of a return / status code. */
const char *ffsrqr_status_string(int code);

/* Text of the last CUDA error seen by this library on the calling thread. */
const char *ffsrqr_last_cuda_error(void);

/* The strong rank-revealing test's g2 = |alpha| ||Rtilde^{-T}||_{1,2} (Alg. 4,
 * Rtilde = [[R11, a], [0, alpha]] of order l + 1): d = 0 (the default)
 * computes it exactly; 1 <= d <= 32 uses Alg. 4's random estimate
 * |alpha| / sqrt(d) ||Omega_t Rtilde^{-T}||_{1,2}, with Omega_t in
 * N(0,1)^{d x (l+1)} drawn afresh for every test t of a run (t = 0 for the
 * first test, t = s after the s-th swap): element (r, j) of Omega_t is element
 * (t d + r)(l + 1) + j of Philox stream 1 under the run's seed (the stream
 * definition of Omega, stream 0, with counter word 2 = 1).  The swap of
 * Alg. 4 takes the argmax of the estimated column norms.  Column l + 1 of
 * Rtilde^{-T} is e_{l+1} / alpha, whose term is exactly 1; the estimate is
 * taken over columns 1..l and floored at 1 like the exact value.  The
 * estimate costs d triangular solves with R11 instead of R11^{-1}.  Applies
 * to the later runs of the plan; not for randomized-subspace-iteration plans.
 * Errors: -1 plan NULL, -2 d outside [0, 32]; FFSRQR_STATUS_UNSUPPORTED for
 * an RSISVD plan or when the swap kernel's shared memory does not fit;
 * FFSRQR_STATUS_CUDA if the device query fails. */
int ffsrqr_plan_set_g2_rows(ffsrqr_plan_t plan, int32_t d);

/* Autotuner of the tensor-core launches (mixed modes): runs the pipeline on
 * the given problem (arguments as ffsrqr_run; outputs hold the last run)
 * while trying, site by site, the schedule of each pass over A (whole tiles
 * data-parallel first, the default, or all stream-K), its pipeline depth
 * (the stages its shared memory holds, or one or two fewer) and the
 * stream-K grid of the Cholesky-QR Grams (all SMs, a half, a quarter),
 * keeping a choice only when the whole run got faster (one warm-up and two
 * timed runs each).  The plan keeps the chosen configuration for its later
 * runs.  config (int32[7], may be NULL) receives the stages of passes 1-3,
 * the Gram grid (0: the default) and, for passes 1-3, 1 where all stream-K
 * was chosen; *ms_best (may be NULL) the best milliseconds per run.
 * Returns as ffsrqr_run. */
int ffsrqr_plan_tune(ffsrqr_plan_t plan, const void *A, int64_t lda, uint64_t seed, void *U, int64_t ldu,
                     void *S, void *V, int64_t ldv, int32_t *piv, void *workspace, void *stream,
                     int32_t *config, float *ms_best);

/* Location of an intermediate inside the workspace after ffsrqr_run, for
 * step-by-step checks.  what: 0 Omega (s x m), 1 B^T (n x s), 2 S11 (k x k,
 * R factor of the sketched pivot columns), 3 Q1 (m x k), 4 G^T = A^T Q1
 * (n x k, original column order), 5 V' = Pi Qhat1 (n x k), 6 tmp = A V'
 * (m x k), 7 trailing estimates r (n), 8 M_t (k x k, tmp = Q_t M_t), 9 the
 * device control words (1 x 40 int32: status, counters; words 14 and 15
 * count the second Cholesky-QR sweeps that took the first-order expansion of
 * their factor and the exact factorization; word 38 the grid barriers of the
 * single-precision sketch QRCP).
 * Writes the byte offset, row/column counts and leading dimension (elements)
 * and the element size in bytes.  Returns 0 or -2 for an unknown item. */
int ffsrqr_workspace_item(ffsrqr_plan_t plan, int32_t what, size_t *offset, int64_t *rows,
                          int64_t *cols, int64_t *ld, int32_t *elem_bytes);

/* Per-phase device times (milliseconds) of the last ffsrqr_run of a plan
 * created with FFSRQR_FLAG_PHASE_TIMES, measured by CUDA events recorded on
 * the run's stream between phases; call after that stream is synchronised.
 * Phases: 0 Omega, 1 pass 1 (sketch), 2 QRCP of the sketch, 3 panel QR,
 * 4 pass 2 (R12), 5 SRQR trailing norms and test, 6 swap loop, 7 QR of
 * (R11 R12)^T, 8 pass 3 (A Pi Qhat1), 9 QR of tmp, 10 small SVD, 11 U, V and
 * outputs; then 12..14 the tensor-core kernels of passes 1, 2, 3 alone (-1
 * outside FFSRQR_MIXED).  Writes min(cap, 15) values; returns the number
 * written, -1 for a NULL plan, -2 if the plan was made without the flag. */
int ffsrqr_phase_times(ffsrqr_plan_t plan, float *ms, int32_t cap);

/* The same for the last run (back = 0) or the run before it (back = 1): a
 * plan keeps two sets of events and alternate runs record into alternate
 * sets, so the times of run i can be read while run i + 1 is already
 * enqueued.  Waits on the host until that run's last event has completed.
 * Returns the count written, -1 NULL plan,
 * -2 plan without FFSRQR_FLAG_PHASE_TIMES, -3 back outside [0, 1] or no
 * such run yet, -4 NULL ms, FFSRQR_STATUS_CUDA if the wait fails. */
int ffsrqr_phase_times_back(ffsrqr_plan_t plan, int32_t back, float *ms, int32_t cap);

/* Number of kernels the last ffsrqr_run of this plan enqueued (-1 for NULL). */
int ffsrqr_launch_count(ffsrqr_plan_t plan);

/* Raw Philox4x32-10 blocks (Salmon et al., SC'11), the counter-based generator
 * behind Omega (Alg. 2's Gaussian test matrix): for t < count, reads
 * ctr_key[6t .. 6t+5] = (c0, c1, c2, c3, k0, k1) and writes the four output
 * words to out[4t .. 4t+3].  Both pointers are device memory; the call only
 * enqueues a kernel on stream.  Returns 0, -1/-2 for NULL pointers, -3 for
 * count < 0, FFSRQR_STATUS_CUDA on launch failure. */
int ffsrqr_philox4x32_10(const uint32_t *ctr_key, uint32_t *out, int32_t count, void *stream);

/* Partial QR with column pivoting of a sketch B (s x n), k steps: Alg. 1
 * applied to B as in Alg. 2 -- the step ffsrqr_run performs after pass 1 --
 * for callers that cannot allocate device memory at the point of the call.
 * The entry point itself has no counterpart in the paper: it only places the
 * step's scratch (candidate columns, control words, selection flags) in a
 * fixed device array of this library instead of a caller workspace.
 *   Bt     device, n x lds row-major FP32: B^T (column i of B is row i).
 *   piv    device, k int32 out: the pivots (original column indices, in
 *          pivot order; greedy largest trailing norm, ties to the lowest
 *          index).
 *   S11    device, k x k row-major FP32 out: the R factor of the pivoted
 *          columns, rows flipped so that its diagonal is non-negative.
 *   status device int32 out or NULL: the largest of the codes met --
 *          0; FFSRQR_STATUS_RANK_DEFICIENT (a winner with zero trailing
 *          norm; outputs complete); FFSRQR_STATUS_TIMEOUT (a bounded grid
 *          wait expired: piv and S11 are written only for the steps before
 *          it); FFSRQR_STATUS_NONFINITE (no column with a finite trailing
 *          norm was left at some step, e.g. NaN in Bt: that step and the
 *          later ones are skipped, so piv[j] and column j of S11 keep
 *          what the caller had there for every skipped step j, up to the
 *          sign of each row, which the non-negative-diagonal normalisation
 *          of the completed rows may flip).
 * Limits of the static scratch: n <= 65536, lds <= 256 (so s <= 256 and
 * k <= 256), and the sketch slabs must fit the blocks' shared memory (else
 * FFSRQR_STATUS_UNSUPPORTED).  Nothing is allocated: the scratch's device
 * address is looked up on every call with the calling device current (the
 * first call on a device also loads the module: make it outside any stream
 * capture), and the words that must start at zero are cleared with
 * cudaMemsetAsync on stream.  Calls on one device share the scratch, so
 * calls that may execute at the same time race: order them on one stream or
 * with events.  Enqueues only; results valid after the stream is
 * synchronised.  Returns 0, -i for an invalid i-th argument (1 Bt, 2 n,
 * 3 s, 4 lds < s, 5 k outside [1, min(s, n)], 6 piv, 7 S11),
 * FFSRQR_STATUS_UNSUPPORTED beyond the limits, FFSRQR_STATUS_CUDA on a CUDA
 * error. */
int ffsrqr_qrcp_static(const float *Bt, int64_t n, int32_t s, int64_t lds, int32_t k, int32_t *piv,
                       float *S11, int32_t *status, void *stream);


/* ------------------------------------------------------------------------ */
/* Batched problems (many uneven rank-k approximations as one graph launch) */
/* ------------------------------------------------------------------------ */
/* Not a step of the paper's algorithm: a way to run Alg. 9 on many matrices
 * at once (e.g. the mode unfoldings of a Tucker decomposition or the iterates
 * of singular-value thresholding, the paper's applications). */
typedef struct ffsrqr_batch_s *ffsrqr_batch_t;

/* One problem's device buffers, as in ffsrqr_run. */
typedef struct {
  const void *A;
  int64_t lda;
  uint64_t seed;
  void *U;
  int64_t ldu;
  void *S;
  void *V;
  int64_t ldv;
  int32_t *piv;
} ffsrqr_problem_t;

/* Plans count problems (sizes m[i] x n[i], rank k[i], oversampling p[i], one
 * mode and opts for all) and lays their workspaces out in one buffer of
 * *workspace_bytes (256-byte aligned slices).  streams (1..64): concurrent
 * streams the batch graph uses.  Returns 0, -1 NULL batch, -2 count < 1,
 * -3 NULL size arrays, -8 streams outside [1, 64], -9 NULL workspace_bytes,
 * or the ffsrqr_plan code of the first problem that fails to plan. */
int ffsrqr_batch_create(ffsrqr_batch_t *batch, int32_t count, const int64_t *m, const int64_t *n,
                        const int32_t *k, const int32_t *p, int32_t mode, const ffsrqr_opts_t *opts,
                        int32_t streams, size_t *workspace_bytes);

/* Runs every problem (probs[count], infos[count] pinned host or NULL).  On
 * the first call, or when probs / workspace / infos / the stream count
 * differ from the previous call, the pipelines of all problems are captured
 * into one CUDA graph (stream forked into the batch's streams, problems in
 * decreasing m*n round-robin over them, joined back); the graph is then
 * launched on stream.  Later calls with the same arguments only launch it.
 * Returns 0, -1 NULL batch, -2 NULL probs, -3 NULL or unaligned workspace,
 * the ffsrqr_run code of a problem, or FFSRQR_STATUS_CUDA. */
int ffsrqr_batch_run(ffsrqr_batch_t batch, const ffsrqr_problem_t *probs, void *workspace, void *stream,
                     ffsrqr_info_t *infos);

/* Autotuner: times the batch graph (3 launches after a warm-up) with 1, 2,
 * 4 and 8 streams, plain and phase-batched, on stream and keeps the fastest;
 * writes its stream count to *chosen and its milliseconds per launch to
 * *ms_best (either may be NULL; ffsrqr_batch_phased reports the other
 * choice).  The batch's outputs hold the results of the last timed launch.
 * Returns as ffsrqr_batch_run. */
int ffsrqr_batch_tune(ffsrqr_batch_t batch, const ffsrqr_problem_t *probs, void *workspace, void *stream,
                      ffsrqr_info_t *infos, int32_t *chosen, float *ms_best);

/* Current stream count of the batch (-1 for NULL). */
int ffsrqr_batch_streams(ffsrqr_batch_t batch);

/* Phase-batched graph (phased = 1): the streams run every problem up to its
 * small SVD (Alg. 9, "svd(tmp)"), join, one launch per cluster size takes the
 * small SVDs of all single-precision problems whose SRQR depth is k together
 * (the column-block Jacobi of each problem on its own thread-block cluster),
 * then the streams fork again for the rest.  Results are bitwise those of the
 * plain graph (phased = 0, the default).  The next ffsrqr_batch_run
 * re-captures.  Returns 0, -1 NULL batch, -2 phased not 0 or 1. */
int ffsrqr_batch_set_phased(ffsrqr_batch_t batch, int32_t phased);

/* 1 if the batch builds phase-batched graphs, 0 if not, -1 for NULL. */
int ffsrqr_batch_phased(ffsrqr_batch_t batch);

/* Batched small-SVD launches in the captured graph (0 or more), -1 for NULL,
 * before the first capture, or when the graph is not phase-batched. */
int ffsrqr_batch_small_svd_launches(ffsrqr_batch_t batch);

/* Byte offset of problem i's workspace slice and its plan (for
 * ffsrqr_workspace_item).  Returns 0, -1 NULL batch, -2 i out of range. */
int ffsrqr_batch_workspace_offset(ffsrqr_batch_t batch, int32_t i, size_t *offset, ffsrqr_plan_t *plan);

int ffsrqr_batch_destroy(ffsrqr_batch_t batch);

/* ------------------------------------------------------------------------ */
/* Host-buffer pipeline                                                      */
/* ------------------------------------------------------------------------ */
/* Not a step of the paper's algorithm: problems of one plan's shape whose A
 * and outputs live in host memory.  The copy of problem i+1's A to the device
 * overlaps the computation of problem i, and problem i's outputs return while
 * problem i+1 computes (two device buffer sets, one stream per direction). */
typedef struct ffsrqr_pipe_s *ffsrqr_pipe_t;

/* One problem in host memory (pinned memory lets the copies overlap): A
 * (m x n, row-major, lda >= n), outputs U (m x k, ldu >= k), S (k), V (n x k,
 * ldv >= k), piv (int32[n]), as in ffsrqr_run. */
typedef struct {
  const void *A;
  int64_t lda;
  uint64_t seed;
  void *U;
  int64_t ldu;
  void *S;
  void *V;
  int64_t ldv;
  int32_t *piv;
} ffsrqr_host_problem_t;

/* Creates a pipeline for plan (which it does not own) and writes the device
 * memory it needs beside the plan's workspace: two inputs and two output sets
 * (256-byte aligned).  Returns 0, -1 NULL pipe, -2 NULL plan, -3 NULL
 * device_bytes, FFSRQR_STATUS_CUDA if its streams or events cannot be made. */
int ffsrqr_pipe_create(ffsrqr_pipe_t *pipe, ffsrqr_plan_t plan, size_t *device_bytes);

/* Enqueues count problems: for each, host A -> device buffer (H2D stream),
 * ffsrqr_run on stream, outputs -> host (D2H stream).  device_mem: device,
 * the size ffsrqr_pipe_create reported, 256-byte aligned; workspace: the
 * plan's.  stream (NULL = legacy stream) waits for the last output copy, so a
 * synchronisation of stream makes every output valid.  infos: pinned host
 * array of count reports, or NULL.  Returns 0, -1 NULL pipe, -2 NULL probs or
 * a problem with a NULL buffer or a leading dimension below n (A) or k,
 * -3 device_mem, -4 count < 0, the ffsrqr_run code of a failing problem, or
 * FFSRQR_STATUS_CUDA. */
int ffsrqr_pipe_run(ffsrqr_pipe_t pipe, const ffsrqr_host_problem_t *probs, int32_t count, void *device_mem,
                    void *workspace, void *stream, ffsrqr_info_t *infos);

int ffsrqr_pipe_destroy(ffsrqr_pipe_t pipe);

/* Shape of a plan: m, n, k (the rank returned), p, mode (any pointer may be
 * NULL).  Returns 0, or -1 for a NULL plan. */
int ffsrqr_plan_shape(ffsrqr_plan_t plan, int64_t *m, int64_t *n, int32_t *k, int32_t *p, int32_t *mode);

/* ------------------------------------------------------------------------ */
/* Request server (admission under a memory budget, continuous batching)    */
/* ------------------------------------------------------------------------ */
/* Not a step of the paper's algorithm: a serving loop for streams of
 * truncated-SVD requests such as the singular-value-thresholding iterates of
 * the paper's robust PCA and matrix completion applications. */
typedef struct ffsrqr_server_s *ffsrqr_server_t;

/* One request: sizes and mode as in ffsrqr_plan, buffers as in ffsrqr_run
 * (device memory owned by the caller until the request is finished). */
typedef struct {
  int64_t m, n;
  int32_t k, p;
  int32_t mode;
  int32_t reserved;
  const void *A;
  int64_t lda;
  uint64_t seed;
  void *U;
  int64_t ldu;
  void *S;
  void *V;
  int64_t ldv;
  int32_t *piv;
} ffsrqr_request_t;

/* Creates a server on the current device: one device arena of budget_bytes
 * (the only device memory it allocates; request workspaces are carved from
 * it first-fit), slots concurrent streams (1..64), options for every plan
 * (NULL for the defaults), and a scheduler thread.  The scheduler admits
 * queued requests in arrival order whenever a slot is free and the arena has
 * room, and retires finished ones, so requests that arrive while others run
 * start as resources free up and overlap on the device.  Returns 0, -1 NULL
 * server, -2 budget below 4096, -3 slots outside [1, 64],
 * FFSRQR_STATUS_WORKSPACE if the arena cannot be allocated, FFSRQR_STATUS_CUDA. */
int ffsrqr_server_create(ffsrqr_server_t *server, size_t budget_bytes, int32_t slots, const ffsrqr_opts_t *opts);

/* Queues a request; writes its ticket.  Returns 0, -1 NULL server, -2 NULL
 * request or buffer, -3 NULL ticket, the ffsrqr_plan code for invalid sizes,
 * or FFSRQR_STATUS_WORKSPACE when its workspace exceeds the whole budget
 * (admission refused). */
int ffsrqr_server_submit(ffsrqr_server_t server, const ffsrqr_request_t *req, int64_t *ticket);

/* Non-blocking status of a ticket: 1 while queued or running; once finished
 * writes its report and latency (seconds from submission to completion) and
 * returns 0 (or the request's error code) -- a finished ticket is reported
 * once, after which it is unknown (-2). */
int ffsrqr_server_poll(ffsrqr_server_t server, int64_t ticket, ffsrqr_info_t *info, double *latency_s);

/* Blocks until the ticket is finished; then as ffsrqr_server_poll. */
int ffsrqr_server_wait(ffsrqr_server_t server, int64_t ticket, ffsrqr_info_t *info, double *latency_s);

/* Counters: requests admitted, finished, still queued, and free arena bytes
 * (any pointer may be NULL). */
int ffsrqr_server_stats(ffsrqr_server_t server, int64_t *admitted, int64_t *completed, int64_t *queued,
                        size_t *arena_free);

/* Same-phase batching (on = 1; 0, the default, turns it off): the requests
 * admitted in one pass of the scheduler whose small SVD (Alg. 9,
 * "svd(tmp)") is the single-precision column-block Jacobi (FP32 and mixed
 * modes, SRQR depth k) run up to the small SVD on their slot streams; one
 * launch per thread-block-cluster size then takes all their small SVDs, and
 * each request finishes on its own stream.  Results are bitwise those of the
 * request run alone.  Returns 0, -1 NULL server, -2 on not 0 or 1. */
int ffsrqr_server_set_phase_batch(ffsrqr_server_t server, int32_t on);

/* paused = 1 holds admission (requests queue; running ones go on), 0 resumes
 * it, so that requests submitted while paused are admitted in one pass (and,
 * with same-phase batching, share their small-SVD launches).  Returns 0, -1
 * NULL server, -2 paused not 0 or 1. */
int ffsrqr_server_pause(ffsrqr_server_t server, int32_t paused);

/* Same-phase batching counters: batched small-SVD launches so far and the
 * requests they covered (either pointer may be NULL). */
int ffsrqr_server_phase_stats(ffsrqr_server_t server, int64_t *small_svd_launches, int64_t *grouped_requests);

/* Stops the scheduler (running requests finish first) and frees the arena. */
int ffsrqr_server_destroy(ffsrqr_server_t server);

/* ------------------------------------------------------------------------ */
/* Tucker approximations: ST-HOSVD (Alg. 6) and HOSVD (Alg. 5) on Alg. 9      */
/* ------------------------------------------------------------------------ */
/* A rank-(k_1, ..., k_d) Tucker approximation X ~= G x_1 U_1 ... x_d U_d of a
 * dense tensor (Sec. 3.1), with Alg. 9 as the approximate rank-k_r SVD of
 * every unfolding:
 *   FFSRQR_TUCKER_STHOSVD (Alg. 6): for each mode r in the processing order,
 *     U S V^T ~= G_(r) of the current core, U_r = U, and the core is replaced
 *     by the tensor whose mode-r unfolding is diag(S) V^T (it shrinks along
 *     mode r to k_r);
 *   FFSRQR_TUCKER_HOSVD (Alg. 5): U_r from the unfolding X_(r) of the input
 *     for every mode, then G = X x_1 U_1^T ... x_d U_d^T.
 *
 * Layout: the tensor X (I_1 x ... x I_d) and the core G (k_1 x ... x k_d) are
 * dense and row-major over their modes (the last index fastest).  The
 * unfolding of mode r has the mode-r index as its row and, as its column, the
 * row-major linear index of the other indices in increasing mode order.  U_r
 * is I_r x k_r row-major (leading dimension k_r).  FP32 in FFSRQR_PLAIN_FP32
 * and FFSRQR_MIXED, FP64 in FFSRQR_FP64. */
typedef struct ffsrqr_tucker_s *ffsrqr_tucker_t;

#define FFSRQR_TUCKER_STHOSVD 0
#define FFSRQR_TUCKER_HOSVD 1

/* Plans the steps for method (FFSRQR_TUCKER_*), 2 <= d <= 8 modes: dims[d] =
 * I_r >= 1, ranks[d] = k_r in [1, I_r], order[d] = the ST-HOSVD processing
 * order (a permutation of 0..d-1; NULL = 0, 1, ..., d-1; ignored by the
 * HOSVD, which factors the modes in order), oversampling p and mode for every
 * Alg. 9 run, opts as in ffsrqr_plan.  Factor step j runs Alg. 9 on an
 * m_j x n_j unfolding: m_j = I_r for r = order[j], n_j = the product of the
 * other modes' current sizes (k_x for the modes the ST-HOSVD has already
 * processed, I_x otherwise); each must meet ffsrqr_plan's requirements
 * (k_r + p <= m_j, k_r <= n_j, k_r <= 224 in FP32).  Writes the device
 * workspace size.  Returns 0, -1 NULL handle, -2 method, -3 d, -4 dims,
 * -5 ranks, -6 order, -7 p, -8 mode, -10 NULL workspace_bytes, -11 a step's
 * unfolding that ffsrqr_plan rejects, FFSRQR_STATUS_UNSUPPORTED (k_r above
 * ffsrqr_plan's limit) or FFSRQR_STATUS_CUDA. */
int ffsrqr_tucker_plan(ffsrqr_tucker_t *plan, int32_t method, int32_t d, const int64_t *dims,
                       const int32_t *ranks, const int32_t *order, int32_t p, int32_t mode,
                       const ffsrqr_opts_t *opts, size_t *workspace_bytes);

/* Enqueues the method on stream.  X: device tensor (read-only).  Factor step j
 * draws its Omega from seed + j.  U: host array of d device pointers, U[r] the
 * I_r x k_r factor of mode r.  S: NULL, or a host array of d device pointers
 * (each may be NULL) that receive the k_r singular values Alg. 9 returns for
 * mode r.  core: device, k_1 x ... x k_d.  workspace: device, the planned size,
 * 256-byte aligned.  infos: NULL or a pinned host array of d reports, one per
 * factor step, valid after the stream is synchronised.  Returns 0, -1 NULL
 * plan, -2 X, -4 U, -6 core, -7 workspace, an ffsrqr_run code, or
 * FFSRQR_STATUS_CUDA if a launch fails. */
int ffsrqr_tucker_run(ffsrqr_tucker_t plan, const void *X, uint64_t seed, void *const *U, void *const *S,
                      void *core, void *workspace, void *stream, ffsrqr_info_t *infos);

/* Kernels the last ffsrqr_tucker_run enqueued (-1 for NULL). */
int ffsrqr_tucker_launch_count(ffsrqr_tucker_t plan);

int ffsrqr_tucker_destroy(ffsrqr_tucker_t plan);

/* ------------------------------------------------------------------------ */
/* Robust PCA by IALM (Alg. 7) on Alg. 9                                     */
/* ------------------------------------------------------------------------ */
/* min ||X||_* + lambda ||E||_1 subject to M = X + E (Sec. 3.2), by the
 * inexact augmented Lagrange multiplier iteration of Alg. 7 with Alg. 9 as
 * the truncated SVD of M - E + Y/mu at a predicted rank sv.  Start:
 * J = max(||M||_2, ||M||_max) (||M||_2 = the first singular value of Alg. 9
 * on M at rank sv0), Y = M / J, E = 0, mu = 1.25 / ||M||_2.  Per iteration:
 * X = U S_{1/mu}(S) V^T over the svp singular values above 1/mu;
 * E = S_{lambda/mu}(M - X + Y/mu); Y += mu (M - X - E); mu = min(rho mu,
 * mu_bar), mu_bar = mu_bar_ratio * mu0; stop when ||M - X - E||_F <
 * tol ||M||_F, or when it stalls (falls by less than 10 % in an iteration)
 * below 100 tol: the rounding floor of the FP32 truncated SVD lies near
 * 1e-6 ||M||_F at 2000 x 2000.  Predicted rank: sv0 at first; then svp + 1 if svp < sv, else
 * svp + round(0.05 n); at most kmax. */
typedef struct ffsrqr_rpca_s *ffsrqr_rpca_t;

/* Options; a field <= 0 takes its default: mode as given (FFSRQR_*; NULL
 * options = FFSRQR_MIXED), p = 10, sv0 = 10, max_iter = 100, kmax = the
 * largest rank the mode supports (224 FP32, 160 FP64, and at most
 * min(n, m - p)), lambda = 1/sqrt(max(m, n)), rho = 1.5 (values <= 1 take it
 * too), mu_bar_ratio = 1e7, tol = 1e-6 in the FP32 modes and 1e-7 in FP64
 * (an FP32 residual does not resolve 1e-7 of ||M||_F). */
typedef struct {
  int32_t mode;
  int32_t p;
  int32_t sv0;
  int32_t max_iter;
  int32_t kmax;
  int32_t reserved;
  double lambda;
  double rho;
  double mu_bar_ratio;
  double tol;
} ffsrqr_rpca_opts_t;

/* Result of a run: status 0 (converged) or FFSRQR_STATUS_SWAP_CAP (the
 * iteration cap was reached), iterations, rank of X (svp of the last
 * iteration), the relative residual ||M - X - E||_F / ||M||_F, the nonzeros
 * of E, ||M||_2 and lambda as used. */
typedef struct {
  int32_t status;
  int32_t iters;
  int32_t rank;
  int32_t reserved;
  double rel_residual;
  int64_t nnz_e;
  double norm2;
  double lambda;
} ffsrqr_rpca_info_t;

/* Plans a solver for m x n inputs (m, n >= 2) and writes the device
 * workspace size (the largest Alg. 9 plan's workspace plus Y, Z (m x n each),
 * U, S, V, piv).  Alg. 9 plans for other ranks are made on first use and
 * cached.  Returns 0, -1 NULL handle, -2 m, -3 n, -4 options (mode, negative
 * values, or no admissible rank), -5 NULL workspace_bytes, or the
 * ffsrqr_plan status for the largest rank. */
int ffsrqr_rpca_create(ffsrqr_rpca_t *solver, int64_t m, int64_t n, const ffsrqr_rpca_opts_t *opts,
                       size_t *workspace_bytes);

/* Solves for M (device, m x n row-major, ldm >= n; FP32, FP64 in FFSRQR_FP64)
 * into X and E (device, m x n, ldx, lde >= n).  Blocking: the host reads the
 * singular values and the residual back every iteration (the rank rule and
 * the stopping test need them) and returns when the iteration ends.  Alg. 9
 * run i draws its Omega from seed + i (run 0 estimates ||M||_2).  info (host,
 * may be NULL) receives the result.  Returns 0, -1 NULL solver, -2 M, -3 ldm,
 * -4 X, -5 ldx, -6 E, -7 lde, -9 workspace, an ffsrqr_plan / ffsrqr_run code,
 * FFSRQR_STATUS_TIMEOUT or FFSRQR_STATUS_NONFINITE when an Alg. 9 run
 * reports it, or FFSRQR_STATUS_CUDA. */
int ffsrqr_rpca_run(ffsrqr_rpca_t solver, const void *M, int64_t ldm, void *X, int64_t ldx, void *E,
                    int64_t lde, uint64_t seed, void *workspace, void *stream, ffsrqr_rpca_info_t *info);

/* Kernels the last ffsrqr_rpca_run enqueued (-1 for NULL). */
int ffsrqr_rpca_launch_count(ffsrqr_rpca_t solver);

int ffsrqr_rpca_destroy(ffsrqr_rpca_t solver);

#ifdef __cplusplus
}
#endif
#endif /* FFSRQR_H */
