"""Pins of the FP64 randomized-subspace-iteration oracle (the paper's appendix
algorithm) against what the mathematics fixes:
* exact recovery of an exactly rank-k matrix (the range finder captures it);
* U S V^T is the rank-k truncation of Q Q^T A, with U, V orthonormal, and the
  Ritz values interlace: sigma_j(rsisvd) <= sigma_j(A);
* more iterations only help, and many iterations reach the truncated SVD
  (the power method's convergence at ratio (sigma_{k+p+1}/sigma_j)^(2q+1));
* the error is within the Halko-Martinsson-Tropp bound for the expected
  spectral error with q iterations, checked with a generous constant.
"""
import numpy as np

import oracle
from oracle import rsisvd as ors
from paper_1803_01982_gb300 import synth


def test_exact_rank_recovery():
    A = synth.rank_k(150, 120, 9, seed=4)
    U, S, V = ors.rsisvd(A, 9, p=5, q=0)
    sv = np.linalg.svd(A, compute_uv=False)[:9]
    assert np.allclose(S, sv, rtol=1e-12)
    assert np.linalg.norm(A - (U * S) @ V.T) <= 1e-11 * np.linalg.norm(A)


def test_projection_identity_and_interlacing():
    A = synth.decayed(200, 160, 0.85 ** np.arange(160), 1e-3, seed=5, dtype=np.float64)
    k, p, q = 10, 5, 1
    U, S, V = ors.rsisvd(A, k, p, q, seed=3)
    assert np.allclose(U.T @ U, np.eye(k), atol=1e-13) and np.allclose(V.T @ V, np.eye(k), atol=1e-13)
    # rebuild Q from the steps' definition and truncate Q Q^T A independently
    Om = oracle.omega(3, 160, k + p)
    Q = np.linalg.qr(A @ Om)[0]
    Q = np.linalg.qr(A.T @ Q)[0]
    Q = np.linalg.qr(A @ Q)[0]
    Uq, Sq, Vqt = np.linalg.svd(Q @ (Q.T @ A), full_matrices=False)
    assert np.allclose(S, Sq[:k], rtol=1e-11)
    assert np.allclose((U * S) @ V.T, (Uq[:, :k] * Sq[:k]) @ Vqt[:k], atol=1e-11 * S[0])
    sv = np.linalg.svd(A, compute_uv=False)
    assert np.all(S <= sv[:k] * (1 + 1e-12))


def test_iterations_converge_to_truncated_svd():
    A = synth.decayed(240, 200, 0.9 ** np.arange(200), 0.0, seed=6, dtype=np.float64)
    k = 12
    sv = np.linalg.svd(A, compute_uv=False)[:k]
    errs = []
    for q in (0, 1, 2, 8, 16):
        _, S, _ = ors.rsisvd(A, k, 5, q, seed=1)
        errs.append(np.max(np.abs(S - sv) / sv))
    assert errs[0] >= errs[1] >= errs[2] >= errs[3] >= errs[4]
    # the slowest Ritz value converges like (sigma_18/sigma_12)^(2(2q+1)) = 0.53^(2(2q+1))
    assert errs[3] < 1e-8 and errs[4] < 1e-13


def test_halko_martinsson_tropp_bound():
    """E||A - Q Q^T A|| <= [(1 + sqrt(k/(p-1))) sigma_{k+1}^{2q+1} + e sqrt(k+p)/p
    (sum_{j>k} sigma_j^{2(2q+1)})^{1/2}]^{1/(2q+1)} (HMT 2011, Cor. 10.10);
    one draw is checked against three times the bound."""
    m, n, k, p, q = 300, 250, 15, 6, 1
    s = 0.95 ** np.arange(n)
    A = synth.decayed(m, n, s, 0.0, seed=7, dtype=np.float64)
    U, S, V = ors.rsisvd(A, k + p, 0, q, seed=2)  # the whole l = k + p basis
    err = np.linalg.norm(A - (U * S) @ V.T, 2)
    e2 = 2 * q + 1
    bound = ((1 + np.sqrt(k / (p - 1))) * s[k] ** e2
             + np.e * np.sqrt(k + p) / p * np.sqrt(np.sum(s[k:] ** (2 * e2)))) ** (1.0 / e2)
    assert s[k + p] <= err <= 3 * bound
