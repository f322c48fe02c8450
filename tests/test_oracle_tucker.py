"""Pins of the FP64 ST-HOSVD oracle (Alg. 6) against facts the mathematics fixes.

* mode products agree with their index definition (Sec. 3.1), written out with
  einsum independently of the unfold/fold helpers;
* with exact truncated SVDs, the ST-HOSVD approximation is the orthogonal
  projection X x_1 P_1 ... x_d P_d (P_r = U_r U_r^T), so
  ||X - Xhat||^2 = ||X||^2 - ||G||^2, and its error is at most the sum over the
  modes of the energy the ORIGINAL unfoldings discard (Vannieuwenhoven,
  Vandebril & Meerbergen 2012, the T-HOSVD bound that ST-HOSVD also meets);
* a tensor of exact multilinear rank (k_1, ..., k_d) is reproduced exactly,
  in any processing order, with Alg. 9 as the SVD as well;
* for d = 2 the core is diag(sigma) up to signs: the matrix truncated SVD.
"""
import numpy as np
import pytest

import oracle
from oracle import tucker as st
from paper_1803_01982_gb300 import synth


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def test_mode_product_matches_index_definition():
    G = _rand((4, 5, 6), 0)
    U = _rand((7, 5), 1)
    Y = st.mode_product(G, U, 1)
    assert np.allclose(Y, np.einsum("ibl,jb->ijl", G, U), rtol=0, atol=1e-13)
    U0 = _rand((3, 4), 2)
    assert np.allclose(st.mode_product(G, U0, 0), np.einsum("abl,ia->ibl", G, U0), rtol=0, atol=1e-13)
    U2 = _rand((2, 6), 3)
    assert np.allclose(st.mode_product(G, U2, 2), np.einsum("abc,ic->abi", G, U2), rtol=0, atol=1e-13)
    M = st.unfold(G, 2)
    assert M.shape == (6, 20)
    assert M[4, 2 * 5 + 3] == G[2, 3, 4]  # columns: row-major over modes 0, 1
    assert np.array_equal(st.fold(M, 2, G.shape), G)


@pytest.mark.parametrize("order", [(0, 1, 2), (1, 2, 0), (2, 0, 1)])
def test_exact_sthosvd_is_a_projection_within_the_bound(order):
    X = _rand((9, 8, 7), 4)
    ranks = (4, 3, 5)
    G, Us, Ss, _ = st.sthosvd(X, ranks, order, svd="exact")
    assert G.shape == ranks
    for r, U in enumerate(Us):
        assert np.allclose(U.T @ U, np.eye(ranks[r]), atol=1e-13)
    Xh = st.tucker_full(G, Us)
    P = [U @ U.T for U in Us]
    Xp = np.einsum("abc,ia,jb,kc->ijk", X, P[0], P[1], P[2])
    assert np.allclose(Xh, Xp, rtol=0, atol=1e-12)
    err2 = np.linalg.norm(X - Xh) ** 2
    assert err2 == pytest.approx(np.linalg.norm(X) ** 2 - np.linalg.norm(G) ** 2, rel=1e-10)
    bound = 0.0
    for r in range(3):
        s = np.linalg.svd(np.moveaxis(X, r, 0).reshape(X.shape[r], -1), compute_uv=False)
        bound += np.sum(s[ranks[r]:] ** 2)
    assert err2 <= bound * (1 + 1e-12)
    # the first processed mode's factor is the leading left singular subspace of X_(r)
    r0 = order[0]
    Ux = np.linalg.svd(np.moveaxis(X, r0, 0).reshape(X.shape[r0], -1))[0][:, :ranks[r0]]
    assert np.allclose(np.abs(Ux.T @ Us[r0]), np.eye(ranks[r0]), atol=1e-10)


@pytest.mark.parametrize("svd", ["exact", "ffsrqr"])
@pytest.mark.parametrize("order", [(0, 1, 2), (2, 1, 0), (1, 0, 2)])
def test_exact_multilinear_rank_is_reproduced(svd, order):
    dims, core = (14, 12, 11), (3, 4, 2)
    X = synth.tucker(dims, core, None, 0.0, seed=5, dtype=np.float64)
    G, Us, Ss, rep = st.sthosvd(X, core, order, p=4, svd=svd)
    Xh = st.tucker_full(G, Us)
    assert np.linalg.norm(X - Xh) <= 1e-12 * np.linalg.norm(X)
    for r in range(3):
        Xr = np.moveaxis(X, r, 0).reshape(dims[r], -1)
        assert np.linalg.norm(Xr - Us[r] @ (Us[r].T @ Xr)) <= 1e-12 * np.linalg.norm(Xr)
    assert all(x["status"] == 0 for x in rep)


def test_order_two_reduces_to_matrix_svd():
    A = synth.decayed(60, 45, 0.8 ** np.arange(45), 0.0, seed=6, dtype=np.float64)
    k = 7
    G, Us, Ss, _ = st.sthosvd(A, (k, k), (0, 1), svd="exact")
    U, s, Vt = np.linalg.svd(A)
    assert np.allclose(np.abs(G), np.diag(s[:k]), atol=1e-12)
    assert np.allclose(np.abs(U[:, :k].T @ Us[0]), np.eye(k), atol=1e-10)
    assert np.allclose(np.abs(Vt[:k] @ Us[1]), np.eye(k), atol=1e-10)
    # with Alg. 9 as the SVD the second step sees a rank-k matrix: the core is
    # diag(S) of the first step, up to signs
    G, Us, Ss, rep = st.sthosvd(A, (k, k), (0, 1), p=5, svd="ffsrqr")
    ref = oracle.ffsrqr(A, k, 5, seed=0)
    assert np.allclose(Ss[0], ref.S, rtol=0, atol=1e-13)
    assert np.allclose(np.abs(G), np.diag(ref.S), rtol=0, atol=1e-12 * ref.S[0])
    assert np.allclose(Ss[1], ref.S, rtol=1e-12)


def test_hosvd_all_orthogonal_core():
    """Untruncated HOSVD (De Lathauwer, De Moor & Vandewalle 2000): the core is
    all-orthogonal, G_(r) G_(r)^T = diag(sigma_i(X_(r))^2), and X = G x_r U_r."""
    X = _rand((6, 5, 4), 7)
    G, Us, Ss, _ = st.hosvd(X, X.shape, svd="exact")
    assert np.allclose(st.tucker_full(G, Us), X, rtol=0, atol=1e-12)
    for r in range(3):
        s = np.linalg.svd(np.moveaxis(X, r, 0).reshape(X.shape[r], -1), compute_uv=False)
        Gr = np.moveaxis(G, r, 0).reshape(X.shape[r], -1)
        assert np.allclose(Gr @ Gr.T, np.diag(s ** 2), rtol=0, atol=1e-11)


def test_truncated_hosvd_is_a_projection_within_the_bound():
    X = _rand((9, 8, 7), 8)
    ranks = (4, 3, 5)
    G, Us, Ss, _ = st.hosvd(X, ranks, svd="exact")
    P = [U @ U.T for U in Us]
    Xh = st.tucker_full(G, Us)
    assert np.allclose(Xh, np.einsum("abc,ia,jb,kc->ijk", X, P[0], P[1], P[2]), rtol=0, atol=1e-12)
    # G = X x_r U_r^T, written out with einsum
    assert np.allclose(G, np.einsum("abc,ai,bj,ck->ijk", X, Us[0], Us[1], Us[2]), rtol=0, atol=1e-12)
    bound = 0.0
    for r in range(3):
        s = np.linalg.svd(np.moveaxis(X, r, 0).reshape(X.shape[r], -1), compute_uv=False)
        bound += np.sum(s[ranks[r]:] ** 2)
        U = np.linalg.svd(np.moveaxis(X, r, 0).reshape(X.shape[r], -1))[0][:, :ranks[r]]
        assert np.allclose(np.abs(U.T @ Us[r]), np.eye(ranks[r]), atol=1e-10)
    assert np.linalg.norm(X - Xh) ** 2 <= bound * (1 + 1e-12)


@pytest.mark.parametrize("svd", ["exact", "ffsrqr"])
def test_hosvd_exact_multilinear_rank(svd):
    dims, core = (14, 12, 11), (3, 4, 2)
    X = synth.tucker(dims, core, None, 0.0, seed=9, dtype=np.float64)
    G, Us, Ss, rep = st.hosvd(X, core, p=4, svd=svd)
    assert np.linalg.norm(X - st.tucker_full(G, Us)) <= 1e-12 * np.linalg.norm(X)
    # the same factor subspaces as the ST-HOSVD's
    _, Ut, _, _ = st.sthosvd(X, core, p=4, svd=svd)
    for r in range(3):
        assert np.allclose(Us[r] @ Us[r].T, Ut[r] @ Ut[r].T, atol=1e-10)
