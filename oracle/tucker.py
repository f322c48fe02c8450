"""FP64 Tucker approximations: ST-HOSVD (Alg. 6) and HOSVD (Alg. 5), Sec. 3.1
-- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module; the product library never loads it.

Tensors are numpy arrays, row-major over their modes.  The unfolding G_(r)
has the mode-r index as its row and, as its column, the row-major index of
the other indices in increasing mode order (Sec. 3.1 leaves the column order
open; it only permutes the rows of V).

``sthosvd(X, ranks, order, p, seed, svd)`` follows Alg. 6 step by step:
  G <- X;  for j, r in enumerate(order):
      U S V^T  ~=  G_(r)   (rank k_r: Alg. 9 via ``oracle.ffsrqr`` with seed
                            seed + j, or the exact truncated SVD)
      U_r <- U;  G_(r) <- diag(S) V^T
and returns the core G, the factors U_r and the singular values S_r by mode.
``hosvd(X, ranks, p, seed, svd)`` follows Alg. 5: U_r from the rank-k_r SVD
of X_(r) (seed + r), then G = X x_1 U_1^T ... x_d U_d^T.
The exact-SVD variant uses the same sign rule as Alg. 9's outputs (the entry
of largest magnitude in each column of U is positive), so the two can be
compared entry by entry where the spectrum is exact.
"""
from __future__ import annotations

import numpy as np

from . import ffsrqr as _ffsrqr


def unfold(G: np.ndarray, r: int) -> np.ndarray:
    """Mode-r unfolding: rows = mode-r index, columns = the other modes, row-major."""
    return np.moveaxis(G, r, 0).reshape(G.shape[r], -1)


def fold(M: np.ndarray, r: int, shape) -> np.ndarray:
    """Inverse of ``unfold`` for a tensor of the given shape (mode r of size M.shape[0])."""
    rest = [shape[x] for x in range(len(shape)) if x != r]
    return np.moveaxis(M.reshape([M.shape[0]] + rest), 0, r)


def mode_product(G: np.ndarray, U: np.ndarray, r: int) -> np.ndarray:
    """G x_r U (Sec. 3.1): the mode-r unfolding becomes U G_(r)."""
    shape = list(G.shape)
    shape[r] = U.shape[0]
    return fold(U @ unfold(G, r), r, shape)


def tucker_full(G: np.ndarray, Us) -> np.ndarray:
    """G x_1 U_1 x_2 ... x_d U_d."""
    X = G
    for r, U in enumerate(Us):
        X = mode_product(X, U, r)
    return X


def _sign_rule(U, V):
    for j in range(U.shape[1]):
        i = int(np.argmax(np.abs(U[:, j])))
        if U[i, j] < 0:
            U[:, j] = -U[:, j]
            V[:, j] = -V[:, j]
    return U, V


def truncated_svd(M: np.ndarray, k: int):
    """Exact rank-k SVD (LAPACK), with Alg. 9's sign rule on U."""
    U, S, Vt = np.linalg.svd(M, full_matrices=False)
    U, V = _sign_rule(U[:, :k].copy(), Vt[:k].T.copy())
    return U, S[:k].copy(), V


def sthosvd(X, ranks, order=None, p: int = 5, seed: int = 0, svd: str = "ffsrqr"):
    """Alg. 6.  Returns (core, [U_r by mode], [S_r by mode], [report per step])."""
    G = np.asarray(X, dtype=np.float64)
    d = G.ndim
    order = list(range(d)) if order is None else list(order)
    assert sorted(order) == list(range(d)) and len(ranks) == d
    Us, Ss, reports = [None] * d, [None] * d, []
    for j, r in enumerate(order):
        k = int(ranks[r])
        U, S, V, rep = _svd(unfold(G, r), k, p, seed + j, svd)
        reports.append(rep)
        Us[r], Ss[r] = U, S
        shape = list(G.shape)
        shape[r] = k
        G = fold(S[:, None] * V.T, r, shape)
    return G, Us, Ss, reports


def _svd(M, k, p, seed, svd):
    if svd == "ffsrqr":
        res = _ffsrqr(M, k, p, seed=seed)
        return res.U, res.S, res.V, {"status": res.status, "swaps": res.swaps, "piv": res.piv}
    if svd == "exact":
        U, S, V = truncated_svd(M, k)
        return U, S, V, {"status": 0, "swaps": 0, "piv": None}
    raise ValueError(svd)


def hosvd(X, ranks, p: int = 5, seed: int = 0, svd: str = "ffsrqr"):
    """Alg. 5.  Returns (core, [U_r by mode], [S_r by mode], [report per mode])."""
    X = np.asarray(X, dtype=np.float64)
    d = X.ndim
    assert len(ranks) == d
    Us, Ss, reports = [], [], []
    for r in range(d):
        U, S, _, rep = _svd(unfold(X, r), int(ranks[r]), p, seed + r, svd)
        Us.append(U)
        Ss.append(S)
        reports.append(rep)
    G = X
    for r in range(d):
        G = mode_product(G, Us[r].T, r)
    return G, Us, Ss, reports
