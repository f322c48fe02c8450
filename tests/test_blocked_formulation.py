"""The device's formulation of TRQRCP with block size b < k (Alg. 2), replayed
in FP64 numpy on the CPU, against the oracle's.

The oracle takes each block's columns through Householder QR after projecting
them on the earlier blocks' Q, and updates the sample with B - B(:, J_j)
R_jj^{-1} G_j, G_j = Q_j^T A.  The device instead projects twice (block
classical Gram-Schmidt), preconditions by the R factor S11 of the block's
sketched columns (from its QRCP on the current sample) and runs CholeskyQR2;
it reads R_jj off G_j = Q_j^T A from the block's pass over A.  Both give the
QR factorization of A(:, J) with a positive diagonal, which is unique, so the
sample, the pivots and the final Q1 and R agree.
"""
import numpy as np
import pytest

import oracle
from paper_1803_01982_gb300 import synth


def _cholqr2(Y):
    Rs = []
    for _ in range(2):
        R = np.linalg.cholesky(Y.T @ Y).T
        Y = np.linalg.solve(R.T, Y.T).T
        Rs.append(R)
    return Y, Rs[1] @ Rs[0]


def _device_blocked(A, B, k, b):
    """Pivots and Q1 of the device's blocked path (FP64 replay)."""
    m, n = A.shape
    s = B.shape[0]
    smp = B.copy()
    sel = np.zeros(n, dtype=bool)
    piv = []
    Q = np.zeros((m, 0))
    for jb in range(0, k, b):
        bb = min(b, k - jb)
        # QRCP for bb steps on the current sample, selected columns masked
        rest = [i for i in range(n) if not sel[i]]
        perm, F, _ = oracle.qrcp(smp[:, rest], bb)
        J = [rest[i] for i in perm[:bb]]
        S11 = np.triu(F[:bb, :bb])
        S11 = S11 * np.sign(np.diag(S11))[:, None]  # rows with a positive diagonal
        # panel: project twice, precondition, CholeskyQR2
        Y = A[:, J].copy()
        for _ in range(2 if jb else 0):
            Y -= Q @ (Q.T @ Y)
        Y = np.linalg.solve(S11.T, Y.T).T
        Qj, _ = _cholqr2(Y)
        # the block's pass over A and the sample update
        Gj = Qj.T @ A
        if jb + bb < k:
            Rjj = np.triu(Gj[:, J])
            Z = np.linalg.solve(Rjj, Gj)  # R_jj^{-1} G_j
            smp = smp - smp[:, J] @ Z
        Q = np.hstack([Q, Qj])
        piv += J
        sel[J] = True
    return piv, Q


@pytest.mark.parametrize("b", [4, 6, 9])
def test_device_formulation_matches_oracle(b):
    rng = np.random.default_rng(b)
    m, n, k, p = 150, 110, 18, 5
    A = synth.decayed(m, n, 0.9 ** np.arange(n), 1e-3, seed=20 + b, dtype=np.float64)
    A = A * np.exp(0.4 * rng.standard_normal(n))[None, :]
    B = oracle.omega(3, b + p, m) @ A
    ref = oracle.srqr(A, B, k, g=1e300, b=b)
    piv, Q1 = _device_blocked(A, B, k, b)
    assert piv == list(ref.perm0[:k])
    # the same Q1 (the unique QR of A(:, J) with a positive diagonal)
    np.testing.assert_allclose(Q1, ref.Q1, atol=1e-9)
    np.testing.assert_allclose(Q1.T @ A[:, piv], np.triu(ref.R[:, :k]), atol=1e-9)
