/*
 * ffsrqr_oracle.c -- plain, slow FP64 CPU oracle for Flip-Flop SRQR
 * (Feng, Xiao & Gu, "Low-Rank Matrix Approximations with Flip-Flop
 * Spectrum-Revealing QR Factorization", arXiv 1803.01982).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, __graft_entry__.smoke() and the CPU-baseline
 * leg of bench.py use it.  It shares no code, header or constant table with
 * the CUDA library: the Philox generator below is written a second time, from
 * its published definition (Salmon, Moraes, Dror & Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), independently of the device one.
 *
 * Every routine follows the paper's algorithm steps in the paper's order, with
 * no blocking, fusion or reordering beyond plain loop order:
 *   Alg. 1  (partial QRCP)                      -> oracle_qrcp
 *   Alg. 2  (TRQRCP, one block b = k, or b < k) -> oracle_srqr_x, first half
 *   Alg. 4  (SRQR test and swap loop)           -> oracle_srqr_x, second half
 *   Alg. 9  (Flip-Flop SRQR)                    -> oracle_ffsrqr_x
 * Readings of points the paper leaves open:
 *   - one TRQRCP block (b = k) by default, SRQR depth l = k; with b < k
 *     (blocked_pivots) the sketch has b + p rows and each block's pivots come
 *     from QRCP on the sample updated by the earlier blocks;
 *   - the trailing-norm estimate of Alg. 4 uses the updated sample
 *     B2 - B1 R11^{-1} R12 (the sample of A(l+1:m, l+1:n) that TRQRCP's
 *     "update B" step produces), divided by b + p;
 *   - g2 = |alpha| * ||Rtilde^{-T}||_{1,2} is computed exactly (closed form)
 *     by default; with d >= 1 (oracle_srqr_x, oracle_ffsrqr_x) it is Alg. 4's
 *     d-row random estimate |alpha|/sqrt(d) * ||Omega_t Rtilde^{-T}||_{1,2},
 *     Omega_t in N(0,1)^{d x (l+1)} drawn afresh for every test t (0 for the
 *     first, s after the s-th swap) from Philox stream 1: element (i, j) is
 *     stream element (t d + i)(l+1) + j.  Column l+1 of Rtilde^{-T} is
 *     e_{l+1}/alpha, so its term is exactly 1 and is not estimated; only
 *     columns 1..l are, and the estimate is max(1, max_{i<=l} ...) like the
 *     exact value;
 *   - every argmax breaks ties toward the lowest ORIGINAL column index;
 *   - "Round Robin rotation" = cyclic shift that moves the leaving column to
 *     position l+1, followed by Givens re-triangularisation;
 *   - the final small SVD is a cyclic one-sided Jacobi SVD; singular vectors
 *     are made unique by the sign rule "largest-|.| entry of each U column is
 *     positive (lowest row on ties)".
 * All matrices are row-major.  All arithmetic is IEEE double.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define ORACLE_OK 0
#define ORACLE_RANK_DEFICIENT 1
#define ORACLE_SWAP_CAP 2

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the two-multiplier     */
/* S-box, Weyl sequence on the key between rounds.                           */
/* ------------------------------------------------------------------------ */
static void philox_round(uint32_t c[4], const uint32_t key[2])
{
    const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ key[0];
    const uint32_t n2 = hi0 ^ c[3] ^ key[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        philox_round(c, k);
    }
    out[0] = c[0];
    out[1] = c[1];
    out[2] = c[2];
    out[3] = c[3];
}

/* Element e of a Gaussian stream: counter (q_lo, q_hi, stream, 0) with
 * q = floor(e/4), key = (seed_lo, seed_hi); outputs (x0,x1) and (x2,x3) feed
 * two Box-Muller pairs (Box & Muller 1958): e%4 = 0,1 -> cos/sin of the first
 * pair, e%4 = 2,3 -> cos/sin of the second.  u = (x + 1/2) 2^-32 in (0,1). */
double oracle_normal(uint64_t seed, uint32_t stream, uint64_t e)
{
    const uint64_t q = e >> 2;
    const int r = (int)(e & 3u);
    const uint32_t ctr[4] = {(uint32_t)q, (uint32_t)(q >> 32), stream, 0u};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t x[4];
    oracle_philox4x32_10(ctr, key, x);
    const uint32_t a = x[(r >> 1) * 2], b = x[(r >> 1) * 2 + 1];
    const double u1 = ((double)a + 0.5) * 0x1p-32;
    const double u2 = ((double)b + 0.5) * 0x1p-32;
    const double rad = sqrt(-2.0 * log(u1));
    const double ang = 2.0 * M_PI * u2;
    return (r & 1) ? rad * sin(ang) : rad * cos(ang);
}

/* Omega in N(0,1)^{s x m} (Alg. 2, first line), row-major, element (i,j) is
 * stream element e = i*m + j of stream 0. */
void oracle_omega(uint64_t seed, int64_t s, int64_t m, double *Omega)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < s; ++i)
        for (int64_t j = 0; j < m; ++j)
            Omega[i * m + j] = oracle_normal(seed, 0u, (uint64_t)(i * m + j));
}

/* ------------------------------------------------------------------------ */
/* Dense helpers (plain loops).                                               */
/* ------------------------------------------------------------------------ */

/* C (r x c) = X (r x t) * Y (t x c); Y has leading dimension ldy. Parallel
 * over column blocks of C so that a row piece of Y is reused from cache. */
static void mat_mul(const double *X, const double *Y, int64_t ldy, double *C, int64_t r, int64_t t,
                    int64_t c)
{
    const int64_t JB = 256;
    const int64_t nb = (c + JB - 1) / JB;
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nb; ++b) {
        const int64_t j0 = b * JB, j1 = (j0 + JB < c) ? j0 + JB : c;
        for (int64_t i = 0; i < r; ++i)
            for (int64_t j = j0; j < j1; ++j) C[i * c + j] = 0.0;
        for (int64_t l = 0; l < t; ++l) {
            const double *yrow = Y + l * ldy;
            for (int64_t i = 0; i < r; ++i) {
                const double w = X[i * t + l];
                if (w == 0.0) continue;
                double *crow = C + i * c;
                for (int64_t j = j0; j < j1; ++j) crow[j] += w * yrow[j];
            }
        }
    }
}

/* dlarfg-style Householder reflector for x (length len, stride inc):
 * H = I - tau v v^T, v(0) = 1, H x = beta e1 with beta = -sign(x0) ||x||.
 * On return x(0) holds beta and x(1:) holds v(1:). Returns tau. */
static double householder(double *x, int64_t len, int64_t inc)
{
    double alpha = x[0], ss = 0.0;
    for (int64_t t = 1; t < len; ++t) ss += x[t * inc] * x[t * inc];
    if (ss == 0.0) return 0.0; /* H = I; x(0) stays alpha */
    const double normx = sqrt(alpha * alpha + ss);
    const double beta = (alpha >= 0.0) ? -normx : normx;
    const double tau = (beta - alpha) / beta;
    const double scal = 1.0 / (alpha - beta);
    for (int64_t t = 1; t < len; ++t) x[t * inc] *= scal;
    x[0] = beta;
    return tau;
}

/* Householder QR without pivoting of X (m x k, leading dim ldx, k <= m):
 * X = Q R with Q (m x k, explicit, orthonormal columns) and R (k x k, upper
 * triangular, diagonal made >= 0 by flipping rows of R / columns of Q). */
void oracle_house_qr(const double *X, int64_t m, int64_t k, int64_t ldx, double *Q, double *R)
{
    double *W = (double *)malloc(sizeof(double) * (size_t)(m * k));
    double *tau = (double *)malloc(sizeof(double) * (size_t)k);
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < k; ++j) W[i * k + j] = X[i * ldx + j];
    for (int64_t j = 0; j < k; ++j) {
        tau[j] = householder(W + j * k + j, m - j, k);
        /* apply H_j to trailing columns j+1..k-1 */
        for (int64_t c = j + 1; c < k; ++c) {
            double w = W[j * k + c];
            for (int64_t t = j + 1; t < m; ++t) w += W[t * k + j] * W[t * k + c];
            w *= tau[j];
            W[j * k + c] -= w;
            for (int64_t t = j + 1; t < m; ++t) W[t * k + c] -= w * W[t * k + j];
        }
    }
    for (int64_t i = 0; i < k; ++i)
        for (int64_t j = 0; j < k; ++j) R[i * k + j] = (j >= i) ? W[i * k + j] : 0.0;
    /* Q = H_0 H_1 ... H_{k-1} applied to the first k columns of I */
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < k; ++j) Q[i * k + j] = (i == j) ? 1.0 : 0.0;
    for (int64_t j = k - 1; j >= 0; --j) {
        if (tau[j] == 0.0) continue;
        for (int64_t c = 0; c < k; ++c) {
            double w = Q[j * k + c];
            for (int64_t t = j + 1; t < m; ++t) w += W[t * k + j] * Q[t * k + c];
            w *= tau[j];
            Q[j * k + c] -= w;
            for (int64_t t = j + 1; t < m; ++t) Q[t * k + c] -= w * W[t * k + j];
        }
    }
    for (int64_t j = 0; j < k; ++j) {
        if (R[j * k + j] < 0.0) {
            for (int64_t c = j; c < k; ++c) R[j * k + c] = -R[j * k + c];
            for (int64_t t = 0; t < m; ++t) Q[t * k + j] = -Q[t * k + j];
        }
    }
    free(W);
    free(tau);
}

/* ------------------------------------------------------------------------ */
/* Alg. 1: partial QRCP for k steps, applied to the sketch B (s x n).         */
/* B is overwritten with the factored matrix in pivot order; perm[i] is the   */
/* original column at position i.  Column norms are recomputed exactly at     */
/* every step (the "update r_s" line of Alg. 1).                              */
/* ------------------------------------------------------------------------ */
int oracle_qrcp(double *B, int64_t s, int64_t n, int32_t k, int32_t *perm)
{
    int status = ORACLE_OK;
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t j = 0; j < k; ++j) {
        /* r_i = ||B(j:s, i)||^2 for the trailing columns */
        for (int64_t i = j; i < n; ++i) {
            double v = 0.0;
            for (int64_t t = j; t < s; ++t) v += B[t * n + i] * B[t * n + i];
            r[i] = v;
        }
        int64_t best = j;
        for (int64_t i = j + 1; i < n; ++i)
            if (r[i] > r[best] || (r[i] == r[best] && perm[i] < perm[best])) best = i;
        if (r[best] == 0.0) status = ORACLE_RANK_DEFICIENT;
        if (best != j) {
            for (int64_t t = 0; t < s; ++t) {
                double tmp = B[t * n + j];
                B[t * n + j] = B[t * n + best];
                B[t * n + best] = tmp;
            }
            int32_t tp = perm[j];
            perm[j] = perm[best];
            perm[best] = tp;
        }
        const double tau = householder(B + j * n + j, s - j, n);
        if (tau != 0.0) {
            for (int64_t c = j + 1; c < n; ++c) {
                double w = B[j * n + c];
                for (int64_t t = j + 1; t < s; ++t) w += B[t * n + j] * B[t * n + c];
                w *= tau;
                B[j * n + c] -= w;
                for (int64_t t = j + 1; t < s; ++t) B[t * n + c] -= w * B[t * n + j];
            }
        }
        for (int64_t t = j + 1; t < s; ++t) B[t * n + j] = 0.0; /* keep only R */
    }
    free(r);
    return status;
}

/* Solve R11 x = b for upper-triangular R11 (k x k, leading dim ldr). */
static void upper_solve(const double *R, int64_t ldr, int64_t k, double *x)
{
    for (int64_t i = k - 1; i >= 0; --i) {
        double v = x[i];
        for (int64_t j = i + 1; j < k; ++j) v -= R[i * ldr + j] * x[j];
        x[i] = v / R[i * ldr + i];
    }
}

/* ------------------------------------------------------------------------ */
/* Alg. 4 (SRQR) with Alg. 2 (TRQRCP, b = k) as its initialisation.          */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t status;
    int32_t swaps;
    double g2_first;
    double g2_final;
    int32_t cand_first; /* original index of the first SRQR candidate (-1: none) */
    double alpha_first;
} oracle_srqr_info;

/* State of the (l+1)-step factorisation A Pi(:, 0:l+1) = Qx Rx(:, 0:l+1). */
typedef struct {
    const double *A;
    int64_t m, n, lda;
    int32_t k;
    double *Qx; /* m x (k+1) */
    double *Rx; /* (k+1) x n, pivot order */
    int32_t *perm;
    double *r; /* trailing squared-norm estimates, pivot order */
} srqr_state;

static void swap_cols(srqr_state *S, int64_t a, int64_t b, int64_t rows)
{
    if (a == b) return;
    const int64_t n = S->n;
    for (int64_t t = 0; t < rows; ++t) {
        double v = S->Rx[t * n + a];
        S->Rx[t * n + a] = S->Rx[t * n + b];
        S->Rx[t * n + b] = v;
    }
    int32_t p = S->perm[a];
    S->perm[a] = S->perm[b];
    S->perm[b] = p;
    double v = S->r[a];
    S->r[a] = S->r[b];
    S->r[b] = v;
}

/* argmax of r over positions l..n-1, ties -> lowest original column index */
static int64_t argmax_trailing(const srqr_state *S, int64_t l)
{
    int64_t best = l;
    for (int64_t i = l + 1; i < S->n; ++i)
        if (S->r[i] > S->r[best] || (S->r[i] == S->r[best] && S->perm[i] < S->perm[best])) best = i;
    return best;
}

/* One-step QR of the trailing matrix at position l = k: the column at
 * position k is orthogonalised against Q1 = Qx(:, 0:k) (Gram-Schmidt applied
 * twice, in FP64), alpha = its residual norm, q = residual / alpha becomes
 * Qx(:, k), and row k of R becomes q^T A Pi for the trailing positions; the
 * trailing estimates are downdated r_i -= R(k, i)^2 (Alg. 4). Returns alpha. */
static double one_step_qr(srqr_state *S)
{
    const int64_t m = S->m, n = S->n, lda = S->lda, k = S->k, kp = k + 1;
    const int64_t c = S->perm[k];
    double *z = (double *)malloc(sizeof(double) * (size_t)m);
    double *h = (double *)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
    for (int64_t t = 0; t < m; ++t) z[t] = S->A[t * lda + c];
    for (int pass = 0; pass < 2; ++pass) {
        for (int64_t j = 0; j < k; ++j) {
            double v = 0.0;
            for (int64_t t = 0; t < m; ++t) v += S->Qx[t * kp + j] * z[t];
            h[j] = v;
        }
        for (int64_t t = 0; t < m; ++t) {
            double v = z[t];
            for (int64_t j = 0; j < k; ++j) v -= S->Qx[t * kp + j] * h[j];
            z[t] = v;
        }
    }
    double a2 = 0.0;
    for (int64_t t = 0; t < m; ++t) a2 += z[t] * z[t];
    const double alpha = sqrt(a2);
    for (int64_t t = 0; t < m; ++t) S->Qx[t * kp + k] = (alpha > 0.0) ? z[t] / alpha : 0.0;
    for (int64_t i = 0; i < k; ++i) S->Rx[k * n + i] = 0.0;
    S->Rx[k * n + k] = alpha;
#pragma omp parallel for schedule(static)
    for (int64_t i = k + 1; i < n; ++i) {
        const int64_t col = S->perm[i];
        double v = 0.0;
        for (int64_t t = 0; t < m; ++t) v += S->Qx[t * kp + k] * S->A[t * lda + col];
        S->Rx[k * n + i] = v;
    }
    for (int64_t i = k + 1; i < n; ++i) S->r[i] -= S->Rx[k * n + i] * S->Rx[k * n + i];
    free(z);
    free(h);
    return alpha;
}

/* g2 = |alpha| * ||Rtilde^{-T}||_{1,2} with Rtilde = [[R11, a], [0, alpha]]
 * (Eq. for g1, g2 in Sec. 2.2).  Row i <= k of Rtilde^{-1} is
 * [e_i^T R11^{-1}, -(R11^{-1} a)_i / alpha] and row k+1 is [0, 1/alpha], so
 * g2 = max(1, max_i sqrt(alpha^2 ||e_i^T R11^{-1}||^2 + (R11^{-1} a)_i^2)).
 * Also returns the maximising row index (the leaving column of Alg. 4). */
static double g2_exact(const srqr_state *S, double alpha, int64_t *imax, int *singular)
{
    const int64_t n = S->n, k = S->k;
    double *Rinv = (double *)calloc((size_t)(k * k), sizeof(double));
    double *u = (double *)malloc(sizeof(double) * (size_t)k);
    *singular = 0;
    for (int64_t i = 0; i < k; ++i)
        if (S->Rx[i * n + i] == 0.0) *singular = 1;
    double g2 = 1.0;
    *imax = -1;
    if (!*singular) {
        /* columns of R11^{-1}: solve R11 x = e_j */
        for (int64_t j = 0; j < k; ++j) {
            double *x = (double *)calloc((size_t)k, sizeof(double));
            x[j] = 1.0;
            upper_solve(S->Rx, n, k, x);
            for (int64_t i = 0; i < k; ++i) Rinv[i * k + j] = x[i];
            free(x);
        }
        for (int64_t i = 0; i < k; ++i) u[i] = S->Rx[i * n + k];
        upper_solve(S->Rx, n, k, u);
        for (int64_t i = 0; i < k; ++i) {
            double rn = 0.0;
            for (int64_t j = 0; j < k; ++j) rn += Rinv[i * k + j] * Rinv[i * k + j];
            const double v = sqrt(alpha * alpha * rn + u[i] * u[i]);
            if (v > g2) {
                g2 = v;
                *imax = i;
            }
        }
    }
    free(Rinv);
    free(u);
    return g2;
}

/* Alg. 4's d-row estimate of g2 for test t: form Rtilde = [[R11, a],
 * [0, alpha]] ((k+1) x (k+1), a = R(0:k, k) of the candidate), draw Omega_t
 * (d x (k+1), Philox stream 1), solve Rtilde Y^T = Omega_t^T one row of
 * Omega_t at a time (Y = Omega_t Rtilde^{-T}), and take
 * |alpha|/sqrt(d) * (2-norm of column i of Y) for i < k; column k's term is
 * exactly 1 (see the header).  alpha = 0 makes Rtilde singular: the
 * estimate's limit |alpha| Y(:, i) -> -(R11^{-1} a)_i Omega_t(:, k) is used. */
static double g2_estimate(const srqr_state *S, double alpha, int32_t d, uint64_t seed, int64_t t,
                          int64_t *imax, int *singular)
{
    const int64_t n = S->n, k = S->k, kp = k + 1;
    *singular = 0;
    for (int64_t i = 0; i < k; ++i)
        if (S->Rx[i * n + i] == 0.0) *singular = 1;
    double g2 = 1.0;
    *imax = -1;
    if (*singular) return g2;
    double *Rt = (double *)calloc((size_t)(kp * kp), sizeof(double));
    for (int64_t i = 0; i < k; ++i)
        for (int64_t j = i; j < kp; ++j) Rt[i * kp + j] = S->Rx[i * n + j];
    Rt[k * kp + k] = alpha;
    double *colsq = (double *)calloc((size_t)kp, sizeof(double));
    double *y = (double *)malloc(sizeof(double) * (size_t)kp);
    for (int64_t r = 0; r < d; ++r) {
        for (int64_t j = 0; j < kp; ++j)
            y[j] = oracle_normal(seed, 1u, (uint64_t)((t * d + r) * kp + j));
        if (alpha != 0.0) {
            upper_solve(Rt, kp, kp, y); /* y = Rtilde^{-1} omega_r^T, row r of Y */
            for (int64_t i = 0; i < k; ++i) colsq[i] += (alpha * y[i]) * (alpha * y[i]);
        } else {
            const double wk = y[k];
            for (int64_t i = 0; i < k; ++i) y[i] = S->Rx[i * n + k];
            upper_solve(S->Rx, n, k, y);
            for (int64_t i = 0; i < k; ++i) colsq[i] += (y[i] * wk) * (y[i] * wk);
        }
    }
    for (int64_t i = 0; i < k; ++i) {
        const double v = sqrt(colsq[i] / (double)d);
        if (v > g2) {
            g2 = v;
            *imax = i;
        }
    }
    free(Rt);
    free(colsq);
    free(y);
    return g2;
}

static double g2_test(const srqr_state *S, double alpha, int32_t d, uint64_t seed, int64_t t,
                      int64_t *imax, int *singular)
{
    return (d > 0) ? g2_estimate(S, alpha, d, seed, t, imax, singular)
                   : g2_exact(S, alpha, imax, singular);
}

/* Alg. 2 (TRQRCP) with block size b < k: the pivots of the block starting at
 * position jb come from bb = min(b, k - jb) steps of partial QRCP (Alg. 1) on
 * the current sample, restricted to the columns not selected yet; the block's
 * columns of A are then orthogonalised against the earlier blocks' Q
 * (projected twice) and factored by Householder QR without pivoting ("QR on
 * A(j:m, j:j+b-1)"), G_j = Q_j^T A is formed (one pass over A per block), and
 * the sample is updated ("Update B(:, j+b:n)"):
 *   B <- B - B(:, J_j) R_jj^{-1} G_j,   R_jj = upper triangle of G_j(:, J_j),
 * which keeps B = Omega (I - Q Q^T) A, the sample of the trailing matrix.
 * perm[0:k] receives the pivots in order, perm[k:n] the other columns in
 * ascending order.  The QR factors themselves are recomputed by the caller
 * (the QR of A(:, perm[0:k]) with a positive diagonal is unique, and block
 * Gram-Schmidt with positive diagonals produces the same factors). */
static int blocked_pivots(const double *A, int64_t m, int64_t n, int64_t lda, const double *B0,
                          int64_t s, int32_t k, int32_t b, int32_t *perm)
{
    int status = ORACLE_OK;
    double *B = (double *)malloc(sizeof(double) * (size_t)(s * n));
    memcpy(B, B0, sizeof(double) * (size_t)(s * n));
    int *sel = (int *)calloc((size_t)n, sizeof(int));
    double *Q = (double *)calloc((size_t)(m * k), sizeof(double));
    double *Bc = (double *)malloc(sizeof(double) * (size_t)(s * n));
    int32_t *map = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *pc = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    double *G = (double *)malloc(sizeof(double) * (size_t)(b * n));
    double *Qt = (double *)malloc(sizeof(double) * (size_t)(b * m));
    double *h = (double *)malloc(sizeof(double) * (size_t)k);
    double *x = (double *)malloc(sizeof(double) * (size_t)b);
    for (int32_t jb = 0; jb < k; jb += b) {
        const int32_t bb = (k - jb < b) ? k - jb : b;
        /* partial QRCP on the unselected columns (ascending original order) */
        int64_t nu = 0;
        for (int64_t i = 0; i < n; ++i)
            if (!sel[i]) map[nu++] = (int32_t)i;
        for (int64_t t = 0; t < s; ++t)
            for (int64_t c = 0; c < nu; ++c) Bc[t * nu + c] = B[t * n + map[c]];
        if (oracle_qrcp(Bc, s, nu, bb, pc) != ORACLE_OK) status = ORACLE_RANK_DEFICIENT;
        for (int32_t t = 0; t < bb; ++t) {
            perm[jb + t] = map[pc[t]];
            sel[map[pc[t]]] = 1;
        }
        /* the block's columns, projected twice against Q(:, 0:jb), then QR */
        double *Y = (double *)malloc(sizeof(double) * (size_t)(m * bb));
        double *Qj = (double *)malloc(sizeof(double) * (size_t)(m * bb));
        double *Rj = (double *)malloc(sizeof(double) * (size_t)(bb * bb));
        for (int64_t t = 0; t < m; ++t)
            for (int32_t c = 0; c < bb; ++c) Y[t * bb + c] = A[t * lda + perm[jb + c]];
        for (int pass = 0; pass < 2 && jb > 0; ++pass) {
            for (int32_t c = 0; c < bb; ++c) {
                for (int32_t i = 0; i < jb; ++i) {
                    double v = 0.0;
                    for (int64_t t = 0; t < m; ++t) v += Q[t * k + i] * Y[t * bb + c];
                    h[i] = v;
                }
                for (int64_t t = 0; t < m; ++t) {
                    double v = Y[t * bb + c];
                    for (int32_t i = 0; i < jb; ++i) v -= Q[t * k + i] * h[i];
                    Y[t * bb + c] = v;
                }
            }
        }
        oracle_house_qr(Y, m, bb, bb, Qj, Rj);
        for (int64_t t = 0; t < m; ++t)
            for (int32_t c = 0; c < bb; ++c) Q[t * k + jb + c] = Qj[t * bb + c];
        if (jb + bb < k) {
            /* G_j = Q_j^T A (bb x n) */
            for (int64_t t = 0; t < m; ++t)
                for (int32_t c = 0; c < bb; ++c) Qt[c * m + t] = Qj[t * bb + c];
            mat_mul(Qt, A, lda, G, bb, m, n);
            /* B <- B - B(:, J_j) R_jj^{-1} G_j, column by column, from the
             * block's columns before the update */
            double *BJ = (double *)malloc(sizeof(double) * (size_t)(s * bb));
            for (int64_t t = 0; t < s; ++t)
                for (int32_t c = 0; c < bb; ++c) BJ[t * bb + c] = B[t * n + perm[jb + c]];
            for (int64_t i = 0; i < n; ++i) {
                for (int32_t c = 0; c < bb; ++c) x[c] = G[c * n + i];
                for (int32_t r = bb - 1; r >= 0; --r) { /* x = R_jj^{-1} G_j(:, i) */
                    double v = x[r];
                    for (int32_t c = r + 1; c < bb; ++c) v -= G[r * n + perm[jb + c]] * x[c];
                    x[r] = v / G[r * n + perm[jb + r]];
                }
                for (int64_t t = 0; t < s; ++t) {
                    double v = 0.0;
                    for (int32_t c = 0; c < bb; ++c) v += BJ[t * bb + c] * x[c];
                    B[t * n + i] -= v;
                }
            }
            free(BJ);
        }
        free(Y);
        free(Qj);
        free(Rj);
    }
    int64_t pos = k;
    for (int64_t i = 0; i < n; ++i)
        if (!sel[i]) perm[pos++] = (int32_t)i;
    free(B);
    free(sel);
    free(Q);
    free(Bc);
    free(map);
    free(pc);
    free(G);
    free(Qt);
    free(h);
    free(x);
    return status;
}

/* Run SRQR (Alg. 4, initialised by TRQRCP with b = k, Alg. 2) to depth l = k.
 * Inputs: A (m x n, lda), the sketch B = Omega A (s x n).
 * Outputs: perm (n), Q1 (m x k), R (k x n, pivot order), initial QRCP pivots
 * perm0 (n, may be NULL), trailing estimates r0 (n, pivot order of perm0 after
 * the candidate swap, may be NULL). */
int oracle_srqr_x(const double *A, int64_t m, int64_t n, int64_t lda, const double *B, int64_t s,
                  int32_t k, int32_t b, double g, int32_t max_swaps, int32_t d, uint64_t seed,
                  int32_t *perm, double *Q1, double *R, int32_t *perm0, double *r0,
                  oracle_srqr_info *info)
{
    const int64_t kp = k + 1;
    oracle_srqr_info inf;
    memset(&inf, 0, sizeof inf);
    inf.cand_first = -1;
    /* Alg. 2: partial QRCP on B to obtain the k pivots (one block, b >= k),
     * or the blocked TRQRCP selection */
    int status;
    if (b >= k) {
        double *Bw = (double *)malloc(sizeof(double) * (size_t)(s * n));
        memcpy(Bw, B, sizeof(double) * (size_t)(s * n));
        status = oracle_qrcp(Bw, s, n, k, perm);
        free(Bw);
    } else {
        status = blocked_pivots(A, m, n, lda, B, s, k, b, perm);
    }
    if (perm0) memcpy(perm0, perm, sizeof(int32_t) * (size_t)n);

    /* Alg. 2: QR (no pivoting) of the pivoted panel A(:, perm[0:k]) */
    double *P = (double *)malloc(sizeof(double) * (size_t)(m * k));
    double *R11 = (double *)malloc(sizeof(double) * (size_t)(k * k));
    double *Qp = (double *)malloc(sizeof(double) * (size_t)(m * k));
    for (int64_t t = 0; t < m; ++t)
        for (int64_t j = 0; j < k; ++j) P[t * k + j] = A[t * lda + perm[j]];
    oracle_house_qr(P, m, k, k, Qp, R11);
    free(P);
    free(R11);

    srqr_state S;
    S.A = A;
    S.m = m;
    S.n = n;
    S.lda = lda;
    S.k = k;
    S.Qx = (double *)calloc((size_t)(m * kp), sizeof(double));
    S.Rx = (double *)calloc((size_t)(kp * n), sizeof(double));
    S.perm = perm;
    S.r = (double *)calloc((size_t)n, sizeof(double));
    for (int64_t t = 0; t < m; ++t)
        for (int64_t j = 0; j < k; ++j) S.Qx[t * kp + j] = Qp[t * k + j];
    free(Qp);
    /* R = Q1^T A Pi (rows 0..k-1): R11 and R12 of Eq. (RRQR) */
    {
        double *Q1t = (double *)malloc(sizeof(double) * (size_t)(k * m));
        for (int64_t t = 0; t < m; ++t)
            for (int64_t j = 0; j < k; ++j) Q1t[j * m + t] = S.Qx[t * kp + j];
        double *Rk = (double *)malloc(sizeof(double) * (size_t)(k * n)); /* Q1^T A, original order */
        mat_mul(Q1t, A, lda, Rk, k, m, n);
        for (int64_t j = 0; j < k; ++j)
            for (int64_t i = 0; i < n; ++i) S.Rx[j * n + i] = Rk[j * n + perm[i]];
        free(Rk);
        free(Q1t);
    }

    int singular = 0;
    for (int64_t i = 0; i < k; ++i)
        if (S.Rx[i * n + i] == 0.0) singular = 1;
    if (singular) status = ORACLE_RANK_DEFICIENT;

    if (!singular && k < n) {
        /* Alg. 4: r_i = ||(B2 - B1 R11^{-1} R12)_{:,i}||^2 / (b+p), i > l */
        double *x = (double *)malloc(sizeof(double) * (size_t)k);
        for (int64_t i = k; i < n; ++i) {
            for (int64_t j = 0; j < k; ++j) x[j] = S.Rx[j * n + i];
            upper_solve(S.Rx, n, k, x); /* x = R11^{-1} R12(:, i) */
            double acc = 0.0;
            for (int64_t t = 0; t < s; ++t) {
                double v = B[t * n + perm[i]];
                for (int64_t j = 0; j < k; ++j) v -= B[t * n + perm[j]] * x[j];
                acc += v * v;
            }
            S.r[i] = acc / (double)s;
        }
        free(x);
        /* candidate: argmax, swapped into position l+1 */
        int64_t c = argmax_trailing(&S, k);
        swap_cols(&S, k, c, k);
        if (r0) memcpy(r0, S.r, sizeof(double) * (size_t)n);
        inf.cand_first = S.perm[k];
        double alpha = one_step_qr(&S);
        inf.alpha_first = alpha;
        int64_t imax;
        int sing2;
        double g2 = g2_test(&S, alpha, d, seed, 0, &imax, &sing2);
        inf.g2_first = g2;
        int32_t swaps = 0;
        while (g2 > g && swaps < max_swaps) {
            /* cyclic shift: column imax -> position k, imax+1..k move left */
            {
                double *colR = (double *)malloc(sizeof(double) * (size_t)kp);
                for (int64_t t = 0; t < kp; ++t) colR[t] = S.Rx[t * n + imax];
                int32_t pv = S.perm[imax];
                double rv = S.r[imax];
                for (int64_t i = imax; i < k; ++i) {
                    for (int64_t t = 0; t < kp; ++t) S.Rx[t * n + i] = S.Rx[t * n + i + 1];
                    S.perm[i] = S.perm[i + 1];
                    S.r[i] = S.r[i + 1];
                }
                for (int64_t t = 0; t < kp; ++t) S.Rx[t * n + k] = colR[t];
                S.perm[k] = pv;
                S.r[k] = rv;
                free(colR);
            }
            /* Givens re-triangularisation of the Hessenberg part */
            for (int64_t j = imax; j < k; ++j) {
                const double a = S.Rx[j * n + j], b = S.Rx[(j + 1) * n + j];
                const double h = hypot(a, b);
                if (h == 0.0) continue;
                const double cs = a / h, sn = b / h;
                for (int64_t i = j; i < n; ++i) {
                    const double x0 = S.Rx[j * n + i], x1 = S.Rx[(j + 1) * n + i];
                    S.Rx[j * n + i] = cs * x0 + sn * x1;
                    S.Rx[(j + 1) * n + i] = -sn * x0 + cs * x1;
                }
                S.Rx[(j + 1) * n + j] = 0.0;
                for (int64_t t = 0; t < m; ++t) {
                    const double q0 = S.Qx[t * kp + j], q1 = S.Qx[t * kp + j + 1];
                    S.Qx[t * kp + j] = cs * q0 + sn * q1;
                    S.Qx[t * kp + j + 1] = -sn * q0 + cs * q1;
                }
            }
            /* r_{l+1} = R(l+1,l+1)^2, r_i += R(l+1,i)^2 */
            S.r[k] = S.Rx[k * n + k] * S.Rx[k * n + k];
            for (int64_t i = k + 1; i < n; ++i) S.r[i] += S.Rx[k * n + i] * S.Rx[k * n + i];
            /* new candidate, one-step QR, downdate, new g2 */
            c = argmax_trailing(&S, k);
            swap_cols(&S, k, c, k);
            alpha = one_step_qr(&S);
            ++swaps;
            g2 = g2_test(&S, alpha, d, seed, swaps, &imax, &sing2);
        }
        inf.swaps = swaps;
        inf.g2_final = g2;
        if (g2 > g) status = ORACLE_SWAP_CAP;
    } else {
        inf.g2_first = inf.g2_final = 1.0;
        if (r0) memset(r0, 0, sizeof(double) * (size_t)n);
    }

    for (int64_t t = 0; t < m; ++t)
        for (int64_t j = 0; j < k; ++j) Q1[t * k + j] = S.Qx[t * kp + j];
    for (int64_t j = 0; j < k; ++j)
        for (int64_t i = 0; i < n; ++i) R[j * n + i] = S.Rx[j * n + i];
    free(S.Qx);
    free(S.Rx);
    free(S.r);
    inf.status = status;
    if (info) *info = inf;
    return status;
}

/* oracle_srqr_x with one TRQRCP block (b = k) and the exact g2 (d = 0). */
int oracle_srqr(const double *A, int64_t m, int64_t n, int64_t lda, const double *B, int64_t s,
                int32_t k, double g, int32_t max_swaps, int32_t *perm, double *Q1, double *R,
                int32_t *perm0, double *r0, oracle_srqr_info *info)
{
    return oracle_srqr_x(A, m, n, lda, B, s, k, k, g, max_swaps, 0, 0, perm, Q1, R, perm0, r0, info);
}

/* ------------------------------------------------------------------------ */
/* Small SVD: cyclic one-sided Jacobi (Hestenes) on the columns of M (k x k). */
/* M V = U diag(sigma); sigma sorted descending (stable on ties).             */
/* ------------------------------------------------------------------------ */
int oracle_jacobi_svd(const double *M, int64_t k, double *U, double *sigma, double *V)
{
    double *X = (double *)malloc(sizeof(double) * (size_t)(k * k));
    double *J = (double *)malloc(sizeof(double) * (size_t)(k * k));
    memcpy(X, M, sizeof(double) * (size_t)(k * k));
    for (int64_t i = 0; i < k; ++i)
        for (int64_t j = 0; j < k; ++j) J[i * k + j] = (i == j) ? 1.0 : 0.0;
    const double tol = (double)k * 0x1p-53;
    int sweeps = 0;
    for (; sweeps < 100; ++sweeps) {
        int rotated = 0;
        for (int64_t p = 0; p < k - 1; ++p)
            for (int64_t q = p + 1; q < k; ++q) {
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int64_t t = 0; t < k; ++t) {
                    al += X[t * k + p] * X[t * k + p];
                    be += X[t * k + q] * X[t * k + q];
                    ga += X[t * k + p] * X[t * k + q];
                }
                if (ga == 0.0 || fabs(ga) <= tol * sqrt(al * be)) continue;
                rotated = 1;
                const double zeta = (be - al) / (2.0 * ga);
                const double tt = ((zeta >= 0.0) ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double cs = 1.0 / sqrt(1.0 + tt * tt), sn = cs * tt;
                for (int64_t t = 0; t < k; ++t) {
                    const double xp = X[t * k + p], xq = X[t * k + q];
                    X[t * k + p] = cs * xp - sn * xq;
                    X[t * k + q] = sn * xp + cs * xq;
                    const double jp = J[t * k + p], jq = J[t * k + q];
                    J[t * k + p] = cs * jp - sn * jq;
                    J[t * k + q] = sn * jp + cs * jq;
                }
            }
        if (!rotated) break;
    }
    /* sigma_j = ||X(:,j)||, order descending (stable) */
    double *nrm = (double *)malloc(sizeof(double) * (size_t)k);
    int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    for (int64_t j = 0; j < k; ++j) {
        double v = 0.0;
        for (int64_t t = 0; t < k; ++t) v += X[t * k + j] * X[t * k + j];
        nrm[j] = sqrt(v);
        ord[j] = j;
    }
    for (int64_t a = 1; a < k; ++a) { /* insertion sort, stable */
        int64_t v = ord[a], b = a - 1;
        while (b >= 0 && nrm[ord[b]] < nrm[v]) {
            ord[b + 1] = ord[b];
            --b;
        }
        ord[b + 1] = v;
    }
    for (int64_t j = 0; j < k; ++j) {
        const int64_t c = ord[j];
        sigma[j] = nrm[c];
        for (int64_t t = 0; t < k; ++t) {
            U[t * k + j] = (nrm[c] > 0.0) ? X[t * k + c] / nrm[c] : ((t == j) ? 1.0 : 0.0);
            V[t * k + j] = J[t * k + c];
        }
    }
    free(X);
    free(J);
    free(nrm);
    free(ord);
    return sweeps;
}

/* ------------------------------------------------------------------------ */
/* Alg. 9: Flip-Flop SRQR.                                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t status;
    int32_t swaps;
    double g2_first;
    double g2_final;
    int32_t cand_first;
    double alpha_first;
    int32_t jacobi_sweeps;
} oracle_info;

/* Optional intermediates (each pointer may be NULL). */
typedef struct {
    double *B;       /* s x n sketch Omega A */
    int32_t *perm0;  /* n, QRCP pivots before the SRQR swap loop */
    double *r0;      /* n, trailing estimates (pivot order perm0 with candidate at k) */
    double *Q1;      /* m x k, after SRQR */
    double *R;       /* k x n, after SRQR, pivot order of the final perm */
    double *Vp;      /* n x k, Pi Qhat1 (explicit) */
    double *Rhat;    /* k x k, R factor of (R11 R12)^T */
    double *tmp;     /* m x k, A Pi Qhat1 */
} oracle_trace;

static void sign_rule(double *U, double *V, int64_t m, int64_t n, int64_t k)
{
    for (int64_t j = 0; j < k; ++j) {
        int64_t best = 0;
        for (int64_t t = 1; t < m; ++t)
            if (fabs(U[t * k + j]) > fabs(U[best * k + j])) best = t;
        if (U[best * k + j] < 0.0) {
            for (int64_t t = 0; t < m; ++t) U[t * k + j] = -U[t * k + j];
            for (int64_t t = 0; t < n; ++t) V[t * k + j] = -V[t * k + j];
        }
    }
}

/* Alg. 9 with TRQRCP block size b (1 <= b <= k; the sketch has b + p rows)
 * and g2 exact (d = 0) or Alg. 4's d-row estimate (d >= 1, Omega_t from the
 * run's seed). */
int oracle_ffsrqr_x(const double *A, int64_t m, int64_t n, int64_t lda, int32_t k, int32_t b,
                    int32_t p, uint64_t seed, double g, int32_t max_swaps, int32_t d, double *U,
                    double *S, double *V, int32_t *piv, oracle_info *info, oracle_trace *trace)
{
    if (d < 0 || b < 1 || b > k) return -1;
    if (k < 1 || k > n || k > m || p < 0 || (int64_t)b + p > m || lda < n) return -1;
    const int64_t s = (int64_t)b + p;
    oracle_info inf;
    memset(&inf, 0, sizeof inf);

    /* Alg. 2: Omega and the sample B = Omega A */
    double *Om = (double *)malloc(sizeof(double) * (size_t)(s * m));
    double *B = (double *)malloc(sizeof(double) * (size_t)(s * n));
    oracle_omega(seed, s, m, Om);
    mat_mul(Om, A, lda, B, s, m, n);
    free(Om);
    if (trace && trace->B) memcpy(trace->B, B, sizeof(double) * (size_t)(s * n));

    /* Alg. 9: SRQR to l = k steps */
    double *Q1 = (double *)malloc(sizeof(double) * (size_t)(m * k));
    double *R = (double *)malloc(sizeof(double) * (size_t)(k * n));
    oracle_srqr_info si;
    oracle_srqr_x(A, m, n, lda, B, s, k, b, g, max_swaps, d, seed, piv, Q1, R,
                  trace ? trace->perm0 : NULL, trace ? trace->r0 : NULL, &si);
    free(B);
    inf.status = si.status;
    inf.swaps = si.swaps;
    inf.g2_first = si.g2_first;
    inf.g2_final = si.g2_final;
    inf.cand_first = si.cand_first;
    inf.alpha_first = si.alpha_first;
    if (trace && trace->Q1) memcpy(trace->Q1, Q1, sizeof(double) * (size_t)(m * k));
    if (trace && trace->R) memcpy(trace->R, R, sizeof(double) * (size_t)(k * n));
    free(Q1);

    /* Alg. 9: QRNP of (R11 R12)^T -> Qhat1 (n x k) */
    double *Rt = (double *)malloc(sizeof(double) * (size_t)(n * k));
    for (int64_t j = 0; j < k; ++j)
        for (int64_t i = 0; i < n; ++i) Rt[i * k + j] = R[j * n + i];
    free(R);
    double *Qh = (double *)malloc(sizeof(double) * (size_t)(n * k));
    double *Rh = (double *)malloc(sizeof(double) * (size_t)(k * k));
    oracle_house_qr(Rt, n, k, k, Qh, Rh);
    free(Rt);
    if (trace && trace->Rhat) memcpy(trace->Rhat, Rh, sizeof(double) * (size_t)(k * k));
    free(Rh);
    /* V' = Pi Qhat1: row perm[i] of V' is row i of Qhat1 */
    double *Vp = (double *)malloc(sizeof(double) * (size_t)(n * k));
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < k; ++j) Vp[(int64_t)piv[i] * k + j] = Qh[i * k + j];
    free(Qh);
    if (trace && trace->Vp) memcpy(trace->Vp, Vp, sizeof(double) * (size_t)(n * k));

    /* Alg. 9: tmp = A Pi Qhat1 (m x k) */
    double *T = (double *)malloc(sizeof(double) * (size_t)(m * k));
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < m; ++t) {
        for (int64_t j = 0; j < k; ++j) T[t * k + j] = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            const double a = A[t * lda + i];
            if (a == 0.0) continue;
            for (int64_t j = 0; j < k; ++j) T[t * k + j] += a * Vp[i * k + j];
        }
    }
    if (trace && trace->tmp) memcpy(trace->tmp, T, sizeof(double) * (size_t)(m * k));

    /* Alg. 9: svd(tmp) via Householder QR + Jacobi on R_t */
    double *Qt = (double *)malloc(sizeof(double) * (size_t)(m * k));
    double *Rtt = (double *)malloc(sizeof(double) * (size_t)(k * k));
    oracle_house_qr(T, m, k, k, Qt, Rtt);
    free(T);
    double *Us = (double *)malloc(sizeof(double) * (size_t)(k * k));
    double *Vs = (double *)malloc(sizeof(double) * (size_t)(k * k));
    inf.jacobi_sweeps = oracle_jacobi_svd(Rtt, k, Us, S, Vs);
    free(Rtt);
    mat_mul(Qt, Us, k, U, m, k, k);
    mat_mul(Vp, Vs, k, V, n, k, k);
    free(Qt);
    free(Us);
    free(Vs);
    free(Vp);
    sign_rule(U, V, m, n, k);
    if (info) *info = inf;
    return inf.status;
}

int oracle_ffsrqr(const double *A, int64_t m, int64_t n, int64_t lda, int32_t k, int32_t p,
                  uint64_t seed, double g, int32_t max_swaps, double *U, double *S, double *V,
                  int32_t *piv, oracle_info *info, oracle_trace *trace)
{
    return oracle_ffsrqr_x(A, m, n, lda, k, k, p, seed, g, max_swaps, 0, U, S, V, piv, info, trace);
}

/* Frobenius residual ||A - U diag(S) V^T||_F, accumulated in FP64 without
 * forming the product (used by tests and the benchmark's accuracy line). */
double oracle_residual_fro(const double *A, int64_t m, int64_t n, int64_t lda, const double *U,
                           const double *S, const double *V, int32_t k)
{
    double total = 0.0;
#pragma omp parallel for reduction(+ : total) schedule(static)
    for (int64_t t = 0; t < m; ++t) {
        double *us = (double *)malloc(sizeof(double) * (size_t)k);
        for (int64_t j = 0; j < k; ++j) us[j] = U[t * k + j] * S[j];
        double acc = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double v = A[t * lda + i];
            for (int64_t j = 0; j < k; ++j) v -= us[j] * V[i * k + j];
            acc += v * v;
        }
        free(us);
        total += acc;
    }
    return sqrt(total);
}
