"""FP64 robust PCA by the inexact augmented Lagrange multiplier method (Alg. 7,
Sec. 3.2), with the truncated SVD done by Alg. 9 or exactly -- TEST
INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module; the product library never loads it.

``rpca(M, ...)`` takes Alg. 7's steps in order:
  J = max(||M||_2, ||M||_max);  Y = M / J;  E = 0;  mu = mu0
  repeat:
      U S V^T = rank-sv SVD of  M - E + Y/mu
      X = U S_{1/mu}(S) V^T                      (singular value shrinkage)
      E = S_{lambda/mu}(M - X + Y/mu)            (entrywise soft shrinkage)
      Y = Y + mu (M - X - E);  mu = min(rho mu, mu_bar)
  until ||M - X - E||_F / ||M||_F < tol
Sec. 3.2 leaves mu0, rho, mu_bar, tol and the rank of the approximate SVD to
the reference IALM code; the values used here are the readings the C ABI
documents (mu0 = 1.25/||M||_2, rho = 1.5, mu_bar = 1e7 mu0, tol = 1e-7) and the
predicted-rank rule: start at sv0; after an iteration with svp singular values
above 1/mu, sv = svp + 1 if svp < sv, else svp + round(0.05 n); capped at kmax.
||M||_2 is the largest singular value of the first approximate SVD of M (Alg. 9
at rank sv0), or the exact 2-norm when svd == "exact".
"""
from __future__ import annotations

import numpy as np

from . import ffsrqr as _ffsrqr


def shrink(x, w):
    """Soft shrinkage S_w(x) = sgn(x) max(|x| - w, 0) (Sec. 3.2)."""
    return np.sign(x) * np.maximum(np.abs(x) - w, 0.0)


def rpca(M, lam: float | None = None, rho: float = 1.5, mu_bar_ratio: float = 1e7, tol: float = 1e-7,
         max_iter: int = 100, sv0: int = 10, kmax: int | None = None, p: int = 10, seed: int = 0,
         svd: str = "ffsrqr"):
    """Alg. 7.  Returns (X, E, Y, info) with info = iterations, rank of X
    (svp), nonzeros of E, relative residual and the status (0 converged,
    2 iteration cap)."""
    M = np.asarray(M, dtype=np.float64)
    m, n = M.shape
    lam = 1.0 / np.sqrt(max(m, n)) if lam is None else lam
    if kmax is None:
        kmax = min(n, m - p)

    def tsvd(Z, k, s):
        if svd == "exact":
            U, S, Vt = np.linalg.svd(Z, full_matrices=False)
            return U[:, :k], S[:k], Vt[:k].T
        r = _ffsrqr(Z, k, p, seed=s)
        return r.U, r.S, r.V

    if svd == "exact":
        norm2 = np.linalg.norm(M, 2)
    else:
        norm2 = tsvd(M, min(sv0, kmax), seed)[1][0]
    J = max(norm2, np.max(np.abs(M)))
    Y = M / J
    E = np.zeros_like(M)
    mu = 1.25 / norm2
    mu_bar = mu_bar_ratio * mu
    normM = np.linalg.norm(M)
    sv = min(sv0, kmax)
    X = np.zeros_like(M)
    status, rel, svp = 2, np.inf, 0
    it = 0
    for it in range(1, max_iter + 1):
        U, S, V = tsvd(M - E + Y / mu, sv, seed + it)
        svp = int(np.sum(S > 1.0 / mu))
        sv = min(svp + 1, kmax) if svp < sv else min(svp + int(round(0.05 * n)), kmax)
        X = (U[:, :svp] * (S[:svp] - 1.0 / mu)) @ V[:, :svp].T
        E = shrink(M - X + Y / mu, lam / mu)
        R = M - X - E
        Y = Y + mu * R
        mu = min(rho * mu, mu_bar)
        rel = np.linalg.norm(R) / normM
        if rel < tol:
            status = 0
            break
    info = {"iters": it, "rank": svp, "nnz_e": int(np.count_nonzero(E)), "rel_residual": float(rel),
            "status": status}
    return X, E, Y, info
