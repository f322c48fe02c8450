"""Pins of the FP64 robust PCA oracle (Alg. 7) against what the mathematics and
the paper fix:
* the soft shrinkage operator at known points;
* exact recovery of a low-rank plus sparse matrix (Candes, Li, Ma & Wright
  2011: rank 0.05 n, 5 % gross corruptions is well inside the recoverable
  regime), with the support of E found exactly;
* the optimality conditions of min ||X||_* + lambda ||E||_1, M = X + E, at the
  returned multiplier Y: |Y_ij| <= lambda with Y_ij = lambda sgn(E_ij) on the
  support of E, ||Y||_2 <= 1 and U^T Y V = I on X's singular subspaces;
* the paper's printed outcome at 1000 x 1000 (iterations, rank, nnz(E) and
  error of IALM_FFSRQR, tests/golden/rpca_ialm_ffsrqr_table.txt).
"""
import os

import numpy as np
import pytest

from oracle import rpca as orp
from paper_1803_01982_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rpca_ialm_ffsrqr_table.txt")


def test_shrink_values():
    x = np.array([3.0, -3.0, 0.5, -0.5, 1.0, 0.0])
    assert np.array_equal(orp.shrink(x, 1.0), np.array([2.0, -2.0, 0.0, 0.0, 0.0, 0.0]))


@pytest.fixture(scope="module")
def small():
    M, Xs, Es = synth.rpca_problem(200, 200, 10, 2000, seed=2, dtype=np.float64)
    return M, Xs, Es


@pytest.mark.parametrize("svd", ["exact", "ffsrqr"])
def test_exact_recovery(small, svd):
    M, Xs, Es = small
    X, E, Y, info = orp.rpca(M, svd=svd)
    assert info["status"] == 0 and info["iters"] < 60
    assert np.linalg.norm(X - Xs) <= 1e-5 * np.linalg.norm(Xs)
    assert info["rank"] == 10
    # the support of E* is found: entries above 1e-3 (E*'s smallest is far above it)
    assert np.min(np.abs(Es[Es != 0])) > 1e-2
    assert np.array_equal(np.abs(E) > 1e-3, Es != 0)
    assert np.linalg.norm(E - Es) <= 1e-5 * np.linalg.norm(Es)


def test_optimality_conditions(small):
    M, Xs, Es = small
    lam = 1.0 / np.sqrt(200)
    X, E, Y, info = orp.rpca(M, svd="exact")
    assert np.all(np.abs(Y) <= lam * (1 + 1e-9))
    on = E != 0
    assert np.allclose(Y[on], lam * np.sign(E[on]), rtol=1e-9, atol=0)
    U, s, Vt = np.linalg.svd(X)
    r = info["rank"]
    assert np.linalg.norm(Y, 2) <= 1 + 1e-3
    assert np.allclose(U[:, :r].T @ Y @ Vt[:r].T, np.eye(r), atol=1e-3)


def test_paper_table_1000():
    rows = [list(map(float, l.split())) for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    m, n, err_p, it_p, nnz_p, sv_p = rows[0]
    M, Xs, Es = synth.rpca_problem(int(m), int(n), int(m) // 10, int(0.05 * m * n), seed=1, dtype=np.float64)
    X, E, Y, info = orp.rpca(M, svd="ffsrqr")
    err = np.linalg.norm(X - Xs) / np.linalg.norm(Xs)
    assert info["status"] == 0
    assert info["rank"] == int(sv_p)
    assert abs(info["nnz_e"] - nnz_p) <= 0.002 * nnz_p
    assert abs(info["iters"] - it_p) <= 3
    assert err <= 1e-6 and err <= 5 * err_p
