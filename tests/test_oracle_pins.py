"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these tests re-types the oracle's formulas: each compares it with an
independent route (a library routine such as LAPACK via numpy/scipy, brute
force on tiny inputs, a closed form, or a bound proved in the paper).
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.stats

import oracle
from paper_1803_01982_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Philox4x32-10 and the Gaussian stream (Omega of Alg. 2)
# --------------------------------------------------------------------------
def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat())
def test_philox_known_answers(ctr, key, expect):
    assert list(oracle.philox(ctr, key)) == expect


def test_box_muller_pairs_come_from_one_philox_block():
    # z0^2 + z1^2 = -2 ln u1 and atan2(z1, z0) = 2 pi u2 (mod 2 pi) for the
    # pair built from outputs (x0, x1) of block q (counter = (q, 0, stream, 0)).
    seed, stream = 0x1234_5678_9ABC, 7
    for q in [0, 1, 5, 1 << 20, (1 << 33) + 3]:
        x = oracle.philox([q & 0xFFFFFFFF, q >> 32, stream, 0], [seed & 0xFFFFFFFF, seed >> 32])
        for half in range(2):
            u1 = (float(x[2 * half]) + 0.5) * 2.0 ** -32
            u2 = (float(x[2 * half + 1]) + 0.5) * 2.0 ** -32
            z0 = oracle.normal(seed, stream, 4 * q + 2 * half)
            z1 = oracle.normal(seed, stream, 4 * q + 2 * half + 1)
            assert math.isclose(z0 * z0 + z1 * z1, -2.0 * math.log(u1), rel_tol=1e-13)
            ang = math.atan2(z1, z0) % (2 * math.pi)
            assert math.isclose(ang, (2 * math.pi * u2) % (2 * math.pi), rel_tol=1e-12, abs_tol=1e-12)


def test_omega_is_standard_normal():
    Om = oracle.omega(0, 64, 4096)
    z = Om.ravel()
    n = z.size
    assert abs(z.mean()) < 5.0 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 5.0 * math.sqrt(2.0 / n)
    assert abs(scipy.stats.skew(z)) < 5.0 * math.sqrt(6.0 / n)
    assert abs(scipy.stats.kurtosis(z)) < 5.0 * math.sqrt(24.0 / n)
    assert scipy.stats.kstest(z, "norm").pvalue > 1e-4
    # rows are independent streams of one generator: no visible correlation
    C = np.corrcoef(Om[:8])
    assert np.max(np.abs(C - np.eye(8))) < 5.0 / math.sqrt(4096)


def test_omega_layout_and_seed():
    s, m = 5, 37
    Om = oracle.omega(11, s, m)
    for (i, j) in [(0, 0), (0, 36), (1, 0), (4, 36), (2, 17)]:
        assert Om[i, j] == oracle.normal(11, 0, i * m + j)
    assert not np.allclose(Om, oracle.omega(12, s, m))


def test_uniform_chi_square():
    # the raw 32-bit outputs, bucketed by their top 6 bits, are uniform
    counts = np.zeros(64)
    for q in range(4000):
        x = oracle.philox([q, 0, 0, 0], [0, 0])
        for v in x:
            counts[int(v) >> 26] += 1
    assert scipy.stats.chisquare(counts).pvalue > 1e-4


# --------------------------------------------------------------------------
# Alg. 1: partial QRCP (run on the sketch)
# --------------------------------------------------------------------------
def _greedy_pivots(B, k):
    """Brute force: pivot j = argmax_i dist(b_i, span(b_chosen))."""
    chosen = []
    n = B.shape[1]
    for _ in range(k):
        best, bestd = None, -1.0
        for i in range(n):
            if i in chosen:
                continue
            if chosen:
                C = B[:, chosen]
                coef, *_ = np.linalg.lstsq(C, B[:, i], rcond=None)
                d = np.linalg.norm(B[:, i] - C @ coef)
            else:
                d = np.linalg.norm(B[:, i])
            if d > bestd:
                best, bestd = i, d
        chosen.append(best)
    return chosen


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_qrcp_matches_greedy_definition(seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((9, 30)) * rng.uniform(0.2, 3.0, size=30)[None, :]
    perm, F, st = oracle.qrcp(B, 7)
    assert st == 0
    assert list(perm[:7]) == _greedy_pivots(B, 7)


@pytest.mark.parametrize("seed", [3, 4])
def test_qrcp_matches_lapack_geqp3(seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((25, 300)) * np.linspace(0.5, 2.0, 300)[None, :]
    k = 20
    perm, F, st = oracle.qrcp(B, k)
    _, R, P = scipy.linalg.qr(B, pivoting=True, mode="economic")
    assert list(perm[:k]) == list(P[:k])
    # |R11| agrees with LAPACK's (signs are convention)
    np.testing.assert_allclose(np.abs(np.triu(F[:k, :k])), np.abs(R[:k, :k]), rtol=1e-10,
                               atol=1e-12)


def test_qrcp_ties_go_to_lowest_original_index():
    B = np.zeros((4, 6))
    B[:, 2] = [1, 0, 0, 0]
    B[:, 5] = [0, 1, 0, 0]      # same norm as column 2
    B[:, 1] = [0, 0, 0.5, 0]
    perm, _, _ = oracle.qrcp(B, 2)
    assert list(perm[:2]) == [2, 5]


# --------------------------------------------------------------------------
# Householder QR (panel, (R11 R12)^T and tmp)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(40, 7), (9, 9), (200, 30)])
def test_house_qr_is_the_unique_positive_qr(shape):
    rng = np.random.default_rng(5)
    X = rng.standard_normal(shape)
    Q, R = oracle.house_qr(X)
    Qn, Rn = np.linalg.qr(X)
    d = np.sign(np.diag(Rn))
    np.testing.assert_allclose(Q, Qn * d[None, :], atol=1e-12)
    np.testing.assert_allclose(R, Rn * d[:, None], atol=1e-12)
    assert np.all(np.diag(R) >= 0)
    np.testing.assert_allclose(Q.T @ Q, np.eye(shape[1]), atol=1e-13)


# --------------------------------------------------------------------------
# Small SVD: one-sided Jacobi
# --------------------------------------------------------------------------
@pytest.mark.parametrize("k,grade", [(6, 1.0), (25, 1.0), (40, 1e-6)])
def test_jacobi_svd_matches_lapack(k, grade):
    rng = np.random.default_rng(k)
    M = rng.standard_normal((k, k)) * np.logspace(0, math.log10(grade), k)[None, :]
    U, S, V, sweeps = oracle.jacobi_svd(M)
    Ul, Sl, Vlt = np.linalg.svd(M)
    np.testing.assert_allclose(S, Sl, rtol=1e-12, atol=1e-14 * Sl[0])
    assert np.all(np.diff(S) <= 0)
    np.testing.assert_allclose(U @ np.diag(S) @ V.T, M, atol=1e-12 * Sl[0])
    np.testing.assert_allclose(V.T @ V, np.eye(k), atol=1e-13)
    # singular vectors agree with LAPACK's up to sign (distinct sigma)
    for j in range(k):
        sgn = np.sign(U[:, j] @ Ul[:, j])
        np.testing.assert_allclose(U[:, j] * sgn, Ul[:, j], atol=1e-8)
        np.testing.assert_allclose(V[:, j] * sgn, Vlt[j], atol=1e-8)


# --------------------------------------------------------------------------
# SRQR (Alg. 4 with TRQRCP initialisation)
# --------------------------------------------------------------------------
def _sketch(A, s, seed=0):
    return oracle.omega(seed, s, A.shape[0]) @ A


def test_srqr_factorisation_identity():
    A = synth.decayed(120, 90, 0.8 ** np.arange(90), 1e-3, seed=2, dtype=np.float64)
    k, p = 10, 5
    res = oracle.srqr(A, _sketch(A, k + p), k)
    Ap = A[:, res.perm]
    np.testing.assert_allclose(res.Q1.T @ res.Q1, np.eye(k), atol=1e-13)
    np.testing.assert_allclose(res.Q1 @ res.R[:, :k], Ap[:, :k], atol=1e-12)
    np.testing.assert_allclose(res.R, res.Q1.T @ Ap, atol=1e-12)
    assert np.allclose(np.tril(res.R[:, :k], -1), 0, atol=1e-12)
    assert sorted(res.perm) == list(range(90))


def test_trailing_estimate_is_sample_of_R22():
    # B2 - B1 R11^{-1} R12 = Omega Q2 R22, so r_i = ||Omega Q2 R22(:,i)||^2/(k+p):
    # compute the right-hand side from a full LAPACK QR of A Pi.
    A = synth.decayed(80, 60, 0.7 ** np.arange(60), 1e-4, seed=3, dtype=np.float64)
    k, p = 8, 4
    s = k + p
    Om = oracle.omega(0, s, 80)
    res = oracle.srqr(A, Om @ A, k, g=1e300)  # no swaps: r0 order = perm
    assert res.swaps == 0
    Qf, Rf = np.linalg.qr(A[:, res.perm], mode="complete")
    sample = Om @ Qf[:, k:] @ Rf[k:, k:]
    expect = np.sum(sample ** 2, axis=0) / s
    np.testing.assert_allclose(res.r0[k:], expect, rtol=1e-9, atol=1e-14)
    # the candidate is the argmax of the estimate
    assert res.cand_first == res.perm[k]
    assert res.r0[k] == pytest.approx(expect.max(), rel=1e-9)


def test_g2_closed_form_matches_explicit_inverse():
    A = synth.decayed(100, 70, 0.85 ** np.arange(70), 1e-3, seed=4, dtype=np.float64)
    k, p = 12, 5
    res = oracle.srqr(A, _sketch(A, k + p), k, g=1e300)
    R11 = res.R[:, :k]
    c = res.perm[k]
    a = res.R[:, k]
    z = A[:, c] - res.Q1 @ (res.Q1.T @ A[:, c])
    alpha = np.linalg.norm(z)
    assert alpha == pytest.approx(res.alpha_first, rel=1e-10)
    Rt = np.zeros((k + 1, k + 1))
    Rt[:k, :k] = R11
    Rt[:k, k] = a
    Rt[k, k] = alpha
    Rinv_T = np.linalg.inv(Rt).T
    g2 = alpha * np.max(np.linalg.norm(Rinv_T, axis=0))
    assert res.g2_first == pytest.approx(g2, rel=1e-9)


def test_swap_loop_on_kahan_matrix():
    n = 48
    K = synth.kahan(n, 0.285)
    # a tiny column perturbation breaks the exact ties of the Kahan matrix
    K = K * (1.0 + 1e-10 * np.arange(n))[None, :]
    k, p = 30, 6
    B = _sketch(K, k + p)
    res = oracle.srqr(K, B, k, g=1.05)
    assert res.g2_first > 1.05
    assert res.swaps > 0
    assert res.g2_final <= 1.05 or res.status == 2
    Ap = K[:, res.perm]
    np.testing.assert_allclose(res.Q1 @ res.R[:, :k], Ap[:, :k], atol=1e-12)
    np.testing.assert_allclose(res.R, res.Q1.T @ Ap, atol=1e-12)
    np.testing.assert_allclose(res.Q1.T @ res.Q1, np.eye(k), atol=1e-12)
    # each swap multiplies |det R11| by g2 > g (Gu-Eisenstat): volume grew
    _, R0 = np.linalg.qr(K[:, res.perm0[:k]])
    _, R1 = np.linalg.qr(K[:, res.perm[:k]])
    assert np.sum(np.log(np.abs(np.diag(R1)))) > np.sum(np.log(np.abs(np.diag(R0)))) + \
        res.swaps * math.log(1.05) - 1e-9


def test_swap_cap_status():
    n = 40
    K = synth.kahan(n, 0.3) * (1.0 + 1e-10 * np.arange(n))[None, :]
    res = oracle.srqr(K, _sketch(K, 30), 25, g=1.0 + 1e-12, max_swaps=1)
    if res.g2_final > 1.0 + 1e-12:
        assert res.status == 2 and res.swaps == 1


# --------------------------------------------------------------------------
# Alg. 2 (TRQRCP) with block size b < k
# --------------------------------------------------------------------------
@pytest.mark.parametrize("b", [1, 5, 8, 12])
def test_blocked_pivots_are_lapack_qrcp_of_the_trailing_sample(b):
    # block j's pivots = the first bb pivots of LAPACK's QRCP (geqp3) of the
    # sample of the trailing matrix, Omega (I - P_j P_j^T) A restricted to the
    # unselected columns, with P_j an orthonormal basis (numpy QR) of the
    # columns chosen by the earlier blocks
    rng = np.random.default_rng(b)
    m, n, k, p = 160, 120, 20, 6
    A = synth.decayed(m, n, 0.9 ** np.arange(n), 1e-3, seed=10 + b, dtype=np.float64)
    A = A * np.exp(0.3 * rng.standard_normal(n))[None, :]
    B = _sketch(A, b + p)
    res = oracle.srqr(A, B, k, g=1e300, b=b)
    Om = oracle.omega(0, b + p, m)
    for jb in range(0, k, b):
        bb = min(b, k - jb)
        chosen = list(res.perm0[:jb])
        rest = [i for i in range(n) if i not in chosen]
        T = A[:, rest]
        if chosen:
            P, _ = np.linalg.qr(A[:, chosen])
            T = T - P @ (P.T @ T)
        _, _, piv = scipy.linalg.qr(Om @ T, pivoting=True, mode="economic")
        assert [rest[i] for i in piv[:bb]] == list(res.perm0[jb:jb + bb]), jb
    # the unselected columns follow in ascending order
    assert list(res.perm0[k:]) == sorted(set(range(n)) - set(res.perm0[:k]))


@pytest.mark.parametrize("b", [1, 4, 7])
def test_blocked_ffsrqr_exact_on_rank_k(b):
    k = 9
    A = synth.rank_k(70, 55, k, seed=5)
    r = oracle.ffsrqr(A, k, 4, seed=3, b=b)
    s_true = np.linalg.svd(A, compute_uv=False)
    np.testing.assert_allclose(r.S, s_true[:k], rtol=1e-10)
    assert oracle.residual_fro(A, r.U, r.S, r.V) < 1e-11 * s_true[0]


def test_blocked_ffsrqr_equals_rayleigh_ritz_closed_form():
    A = synth.decayed(90, 70, 0.85 ** np.arange(70), 1e-3, seed=6, dtype=np.float64)
    k, p, b = 14, 5, 6
    r = oracle.ffsrqr(A, k, p, seed=2, b=b, g=1e300)
    U, S, V = _ritz(A, r.piv[:k], k)
    np.testing.assert_allclose(r.S, S, rtol=1e-10)
    np.testing.assert_allclose(np.abs(r.U.T @ U), np.eye(k), atol=1e-8)


# --------------------------------------------------------------------------
# Alg. 4's d-row random estimate of g2
# --------------------------------------------------------------------------
def _g2_omega(seed, t, d, kp):
    """Omega_t (d x (l+1)) of the estimate: element (r, j) is element
    (t d + r)(l+1) + j of Philox stream 1 (the stream is pinned above)."""
    return np.array([[oracle.normal(seed, 1, (t * d + r) * kp + j) for j in range(kp)]
                     for r in range(d)])


@pytest.mark.parametrize("d", [1, 3, 8])
def test_g2_estimate_on_orthogonal_columns(d):
    # A = Q diag(sigma) with orthonormal Q: R11 = diag(sigma of the pivots), a = 0
    # and alpha = sigma of the candidate, so column i of |alpha| Omega Rtilde^{-T}
    # is (alpha / R_ii) Omega(:, i): the estimate needs no inverse at all.
    rng = np.random.default_rng(5)
    m, n, k, p = 70, 40, 9, 4
    sig = 0.8 ** rng.permutation(n)
    Q, _ = np.linalg.qr(rng.standard_normal((m, n)))
    A = Q * sig[None, :]
    res = oracle.srqr(A, _sketch(A, k + p), k, g=1e300, g2_rows=d, seed=11)
    assert res.swaps == 0
    piv, c = res.perm[:k], res.cand_first
    Om = _g2_omega(11, 0, d, k + 1)
    terms = sig[c] / sig[piv] * np.linalg.norm(Om[:, :k], axis=0) / math.sqrt(d)
    assert res.alpha_first == pytest.approx(sig[c], rel=1e-12)
    assert res.g2_first == pytest.approx(max(1.0, terms.max()), rel=1e-10)


def test_g2_estimate_matches_explicit_inverse():
    A = synth.decayed(100, 70, 0.85 ** np.arange(70), 1e-3, seed=4, dtype=np.float64)
    k, p, d = 12, 5, 4
    res = oracle.srqr(A, _sketch(A, k + p), k, g=1e300, g2_rows=d, seed=3)
    Rt = np.zeros((k + 1, k + 1))
    Rt[:k, :k] = res.R[:, :k]
    Rt[:k, k] = res.R[:, k]
    Rt[k, k] = res.alpha_first
    Y = _g2_omega(3, 0, d, k + 1) @ np.linalg.inv(Rt).T
    est = res.alpha_first * np.linalg.norm(Y, axis=0) / math.sqrt(d)
    assert res.g2_first == pytest.approx(max(1.0, est[:k].max()), rel=1e-9)


def test_g2_estimate_converges_to_exact():
    # E ||Omega x||^2 = d ||x||^2: with many rows the estimate approaches the
    # exact g2 (relative spread about 1/sqrt(2d) per column)
    A = synth.decayed(100, 70, 0.85 ** np.arange(70), 1e-3, seed=4, dtype=np.float64)
    k, p = 12, 5
    B = _sketch(A, k + p)
    exact = oracle.srqr(A, B, k, g=1e300).g2_first
    est = oracle.srqr(A, B, k, g=1e300, g2_rows=20000, seed=1).g2_first
    assert exact > 1.1  # not the floor of 1
    assert est == pytest.approx(exact, rel=0.02)


def test_g2_estimate_is_scale_invariant():
    # g2 is homogeneous of degree 0 in A: alpha scales like R11, so the same
    # Omega_t gives the same estimate and the same swap decisions
    n = 48
    K = synth.kahan(n, 0.285) * (1.0 + 1e-10 * np.arange(n))[None, :]
    k, p = 30, 6
    B = _sketch(K, k + p)
    r1 = oracle.srqr(K, B, k, g=1.05, g2_rows=3, seed=2)
    r2 = oracle.srqr(1e3 * K, 1e3 * B, k, g=1.05, g2_rows=3, seed=2)
    assert r1.swaps == r2.swaps > 0
    assert list(r1.perm) == list(r2.perm)
    assert r2.g2_first == pytest.approx(r1.g2_first, rel=1e-11)
    assert r2.g2_final == pytest.approx(r1.g2_final, rel=1e-11)


@pytest.mark.parametrize("d", [1, 4])
def test_swap_loop_with_g2_estimate(d):
    n = 48
    K = synth.kahan(n, 0.285) * (1.0 + 1e-10 * np.arange(n))[None, :]
    k, p = 30, 6
    res = oracle.srqr(K, _sketch(K, k + p), k, g=1.05, g2_rows=d, seed=0)
    assert res.swaps > 0
    assert res.g2_final <= 1.05 or res.status == 2
    Ap = K[:, res.perm]
    np.testing.assert_allclose(res.Q1 @ res.R[:, :k], Ap[:, :k], atol=1e-12)
    np.testing.assert_allclose(res.R, res.Q1.T @ Ap, atol=1e-12)
    np.testing.assert_allclose(res.Q1.T @ res.Q1, np.eye(k), atol=1e-12)
    assert sorted(res.perm) == list(range(n))


# --------------------------------------------------------------------------
# Flip-Flop SRQR (Alg. 9)
# --------------------------------------------------------------------------
def _ritz(A, J, k):
    """Closed form given the pivot set J: rank-k SVD of A W, W = orth(A^T P), P = orth(A_J)."""
    P, _ = np.linalg.qr(A[:, J])
    W, _ = np.linalg.qr(A.T @ P)
    Ur, Sr, Vrt = np.linalg.svd(A @ W, full_matrices=False)
    return Ur[:, :k], Sr[:k], (W @ Vrt.T)[:, :k]


@pytest.mark.parametrize("shape,k,p", [((90, 70), 8, 5), ((60, 110), 10, 3), ((150, 150), 20, 10)])
def test_ffsrqr_equals_rayleigh_ritz_closed_form(shape, k, p):
    m, n = shape
    A = synth.decayed(m, n, 0.9 ** np.arange(min(m, n)), 1e-3, seed=7, dtype=np.float64)
    r = oracle.ffsrqr(A, k, p, seed=0)
    Ur, Sr, Vr = _ritz(A, r.piv[:k], k)
    np.testing.assert_allclose(r.S, Sr, rtol=1e-11)
    for j in range(k):
        sgn = np.sign(r.U[:, j] @ Ur[:, j])
        np.testing.assert_allclose(r.U[:, j], sgn * Ur[:, j], atol=1e-8)
        np.testing.assert_allclose(r.V[:, j], sgn * Vr[:, j], atol=1e-8)
    np.testing.assert_allclose(A @ r.V, r.U * r.S[None, :], atol=1e-11 * r.S[0])
    np.testing.assert_allclose(r.U.T @ r.U, np.eye(k), atol=1e-12)
    np.testing.assert_allclose(r.V.T @ r.V, np.eye(k), atol=1e-12)


def test_ffsrqr_exact_on_rank_k():
    k = 9
    A = synth.rank_k(70, 55, k, seed=5)
    r = oracle.ffsrqr(A, k, 4, seed=3)
    s_true = np.linalg.svd(A, compute_uv=False)
    np.testing.assert_allclose(r.S, s_true[:k], rtol=1e-10)
    assert oracle.residual_fro(A, r.U, r.S, r.V) < 1e-11 * s_true[0]


def test_ffsrqr_interlacing_and_eckart_young():
    A = synth.decayed(60, 50, 0.8 ** np.arange(50), 1e-2, seed=8, dtype=np.float64)
    k = 7
    r = oracle.ffsrqr(A, k, 5)
    sA = np.linalg.svd(A, compute_uv=False)
    assert np.all(r.S <= sA[:k] * (1 + 1e-12))          # sigma_j(A Pi Qhat1) <= sigma_j(A)
    res = oracle.residual_fro(A, r.U, r.S, r.V)
    assert res >= math.sqrt(np.sum(sA[k:] ** 2)) * (1 - 1e-12)   # Thm. 1.1 optimum
    np.testing.assert_allclose(res, np.linalg.norm(A - (r.U * r.S) @ r.V.T), rtol=1e-12)


@pytest.mark.parametrize("seed,decay", [(9, 0.75), (10, 0.9), (11, 0.97)])
def test_theorem_3_2_bounds(seed, decay):
    m, n, k, p = 80, 64, 8, 5
    A = synth.decayed(m, n, decay ** np.arange(min(m, n)), 1e-3, seed=seed, dtype=np.float64)
    r = oracle.ffsrqr(A, k, p)
    sA = np.linalg.svd(A, compute_uv=False)
    _, Rf = np.linalg.qr(A[:, r.piv], mode="complete")
    nR22 = np.linalg.norm(Rf[k:, k:], 2)
    lower = sA[:k] / (1 + 2 * nR22 ** 4 / r.S ** 4) ** 0.25
    assert np.all(r.S >= lower * (1 - 1e-12))
    err2 = np.linalg.norm(A - (r.U * r.S) @ r.V.T, 2)
    assert err2 <= sA[k] * (1 + 2 * (nR22 / sA[k]) ** 4) ** 0.25 * (1 + 1e-12)


def test_tuxv_equivalence_without_swaps():
    # Alg. 3 on the same pivots: svd of its final R equals Sigma (Alg. 9).
    A = synth.decayed(90, 80, 0.85 ** np.arange(80), 1e-3, seed=12, dtype=np.float64)
    k, p = 10, 5
    r = oracle.ffsrqr(A, k, p, g=1e300)
    assert r.swaps == 0
    Q, _ = np.linalg.qr(A[:, r.piv[:k]])
    Rk = Q.T @ A                      # R Pi^T, original column order
    V, _ = np.linalg.qr(Rk.T)
    _, Rz = np.linalg.qr(A @ V)
    np.testing.assert_allclose(np.linalg.svd(Rz, compute_uv=False), r.S, rtol=1e-11)


def test_config1_spectrum_and_bounds():
    A = synth.config1()
    k, p = 20, 5
    r = oracle.ffsrqr(A, k, p, seed=0, trace=True)
    true = 0.9 ** np.arange(1, 21)
    assert np.all(r.S <= true * (1 + 1e-12))
    assert np.all(r.S >= true * 0.5)
    res = oracle.residual_fro(A, r.U, r.S, r.V)
    opt = math.sqrt(np.sum(0.81 ** np.arange(21, 801)))
    assert opt <= res * (1 + 1e-12)
    assert res <= 3.0 * opt
    # the trace's B is Omega A with the same seeded Omega
    np.testing.assert_allclose(r.trace["B"], oracle.omega(0, k + p, 1000) @ A, rtol=1e-12,
                               atol=1e-12)


def test_sign_rule():
    A = synth.decayed(50, 40, 0.8 ** np.arange(40), 1e-3, seed=13, dtype=np.float64)
    r = oracle.ffsrqr(A, 6, 4)
    for j in range(6):
        i = np.argmax(np.abs(r.U[:, j]))
        assert r.U[i, j] > 0


def test_argument_checks():
    A = np.ones((10, 8))
    with pytest.raises(ValueError):
        oracle.ffsrqr(A, 0, 2)
    with pytest.raises(ValueError):
        oracle.ffsrqr(A, 9, 0)
    with pytest.raises(ValueError):
        oracle.ffsrqr(A, 6, 5)    # k + p > m


def test_depth_l_ritz_values_grow_with_the_subspace():
    """Alg. 9 with SRQR depth l > k: on the same sketch (l + p rows) and with no
    swaps, the first k pivots of the depth-l run are the depth-k run's (greedy
    QRCP), so span(V'_k) lies in span(V'_l) and the Ritz values of A on it can
    only grow (Rayleigh-Ritz monotonicity), while staying below the singular
    values of A (interlacing)."""
    A = synth.decayed(200, 160, 0.9 ** np.arange(160), 1e-3, seed=21, dtype=np.float64)
    k, l, p = 8, 14, 6
    rk = oracle.ffsrqr(A, k, p + l - k, seed=0)  # the depth-l run's sketch
    rl = oracle.ffsrqr(A, k, p, seed=0, l=l)
    full = oracle.ffsrqr(A, l, p, seed=0)
    assert rk.swaps == 0 and full.swaps == 0
    assert list(full.piv[:k]) == list(rk.piv[:k])
    sa = np.linalg.svd(A, compute_uv=False)[:k]
    assert np.all(rk.S <= rl.S * (1 + 1e-12)) and np.all(rl.S <= sa * (1 + 1e-12))
    assert np.any(rl.S > rk.S * (1 + 1e-6))
    # the depth-l result is the leading k triplets of the depth-l factorisation
    assert np.array_equal(rl.S, full.S[:k]) and np.array_equal(rl.U, full.U[:, :k])
    assert np.allclose(A @ rl.V, rl.U * rl.S, atol=1e-10)
