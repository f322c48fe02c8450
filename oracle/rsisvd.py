"""FP64 approximate SVD by randomized subspace iteration (the paper's appendix
algorithm, after Halko, Martinsson & Tropp 2011, Alg. 4.4 and 5.1) -- TEST
INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module; the product library never loads it.

``rsisvd(A, k, p, q, seed)`` takes the appendix algorithm's steps in order,
with l = k + p:
  Omega (n x l) Gaussian;  B = A Omega;  Q = qr(B)
  q times:  B = A^T Q;  Q = qr(B);  B = A Q;  Q = qr(B)
  B = Q^T A;  [U~, S, V] = svd(B);  U = Q U~;  keep the leading k triplets.
Omega is the Philox Gaussian of Alg. 2's sketch laid out n x l (element
(i, j) is draw i l + j of stream 0, the row-major order of ``oracle.omega``).
The thin QR is the oracle's Householder QR (diag(R) >= 0) and the SVD of the
l x n matrix B is LAPACK's, with Alg. 9's sign rule on U.
"""
from __future__ import annotations

import numpy as np

from . import house_qr as _house_qr
from . import omega as _omega


def rsisvd(A, k: int, p: int = 5, q: int = 1, seed: int = 0):
    """Returns (U m x k, S k, V n x k)."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    l = k + p
    assert 1 <= k <= l <= min(m, n) and q >= 0
    Om = _omega(seed, n, l)
    Q, _ = _house_qr(A @ Om)
    for _ in range(q):
        Q, _ = _house_qr(A.T @ Q)
        Q, _ = _house_qr(A @ Q)
    Ub, S, Vt = np.linalg.svd(Q.T @ A, full_matrices=False)
    U = Q @ Ub[:, :k]
    V = Vt[:k].T.copy()
    for j in range(k):
        i = int(np.argmax(np.abs(U[:, j])))
        if U[i, j] < 0:
            U[:, j] = -U[:, j]
            V[:, j] = -V[:, j]
    return U, S[:k].copy(), V
