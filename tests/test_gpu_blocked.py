"""GPU parity of TRQRCP with block size b < k (Alg. 2) against the FP64 oracle.

The sketch has b + p rows and the k pivots are chosen block by block: partial
QRCP on the sample updated by the earlier blocks, the block's columns
orthogonalised against the earlier blocks, one pass over A per block.  In
FP64 the device chooses the oracle's pivots and returns its singular values;
in FP32 the test matrices have well separated column norms, so the pivots
agree there too.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_1803_01982_gb300 import ffsrqr, synth  # noqa: E402

pytestmark = pytest.mark.gpu


def matrix(m, n, seed, dtype):
    rng = np.random.default_rng(seed)
    A = synth.decayed(m, n, 0.97 ** np.arange(n), 1e-4, seed=seed, dtype=np.float64)
    A = A * np.exp(0.5 * rng.standard_normal(n))[None, :]
    return np.ascontiguousarray(A.astype(dtype))


def run(A, k, b, p, mode, seed=0, g=2.0, d=0):
    plan = ffsrqr.Plan(A.shape[0], A.shape[1], k, p, mode, g=g, b=b, g2_rows=d)
    dt = torch.float64 if mode == ffsrqr.FP64 else torch.float32
    Ad = torch.as_tensor(np.ascontiguousarray(A), dtype=dt).cuda()
    U, S, V, piv = plan.run(Ad, seed=seed)
    torch.cuda.synchronize()
    return {"U": U.double().cpu().numpy(), "S": S.double().cpu().numpy(),
            "V": V.double().cpu().numpy(), "piv": piv.cpu().numpy(), "info": plan.info()}


def subspace_gap(X, Y):
    return np.linalg.norm(X @ X.T - Y @ Y.T, 2)


@pytest.mark.parametrize("b", [8, 16, 24, 40])
def test_fp64_blocked_matches_oracle(b):
    A = matrix(400, 300, 1, np.float64)
    k, p = 40, 8
    ref = oracle.ffsrqr(A, k, p, seed=2, b=b)
    got = run(A, k, b, p, ffsrqr.FP64, seed=2)
    assert got["info"]["status"] == ref.status == 0
    assert got["info"]["swaps"] == ref.swaps
    assert list(got["piv"][:k]) == list(ref.piv[:k])
    assert np.all(np.diff(got["piv"][k:]) > 0)
    np.testing.assert_allclose(got["S"], ref.S, rtol=1e-10, atol=1e-13 * ref.S[0])
    assert subspace_gap(got["U"][:, :20], ref.U[:, :20]) < 1e-8
    assert subspace_gap(got["V"][:, :20], ref.V[:, :20]) < 1e-8


def test_fp64_blocked_with_g2_estimate():
    A = matrix(300, 220, 3, np.float64)
    k, b, p = 32, 8, 6
    ref = oracle.ffsrqr(A, k, p, seed=4, b=b, g2_rows=4, g=1.2)
    got = run(A, k, b, p, ffsrqr.FP64, seed=4, g=1.2, d=4)
    assert got["info"]["swaps"] == ref.swaps
    assert got["info"]["g2_final"] == pytest.approx(ref.g2_final, rel=1e-9)
    assert list(got["piv"][:k]) == list(ref.piv[:k])
    np.testing.assert_allclose(got["S"], ref.S, rtol=1e-10, atol=1e-13 * ref.S[0])


@pytest.mark.parametrize("mode", [ffsrqr.PLAIN_FP32, ffsrqr.MIXED_TF32X3, ffsrqr.MIXED_BF16X3])
@pytest.mark.parametrize("b", [16, 32])
def test_fp32_blocked_matches_oracle(mode, b):
    A = matrix(3000, 2000, 5, np.float32)
    k, p = 64, 10
    ref = oracle.ffsrqr(A, k, p, seed=6, b=b)
    got = run(A, k, b, p, mode, seed=6)
    assert got["info"]["status"] == 0
    if mode == ffsrqr.PLAIN_FP32:
        # the FP32 sample picks the oracle's columns (well separated norms)
        assert list(got["piv"][:k]) == list(ref.piv[:k])
        np.testing.assert_allclose(got["S"], ref.S, rtol=2e-5)
    else:
        # a TF32 / BF16 sketch may pick other columns; the approximation stays
        # as good as the oracle's
        assert len(set(got["piv"][:k]) & set(ref.piv[:k])) >= k // 2
    A64 = A.astype(np.float64)
    res = np.linalg.norm(A64 - (got["U"] * got["S"]) @ got["V"].T)
    assert res <= 1.02 * oracle.residual_fro(A64, ref.U, ref.S, ref.V)
    assert np.allclose(got["U"].T @ got["U"], np.eye(k), atol=1e-4)
    assert np.allclose(got["V"].T @ got["V"], np.eye(k), atol=1e-4)


def test_one_block_equals_ffsrqr_plan():
    # b = k is the one-block pipeline: bitwise the ffsrqr_plan result
    A = matrix(1000, 800, 7, np.float32)
    got = run(A, 48, 48, 8, ffsrqr.PLAIN_FP32, seed=1)
    plan = ffsrqr.Plan(1000, 800, 48, 8, ffsrqr.PLAIN_FP32)
    U, S, V, piv = plan.run(torch.as_tensor(A).cuda(), seed=1)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(got["S"], S.double().cpu().numpy())
    np.testing.assert_array_equal(got["piv"], piv.cpu().numpy())


def test_blocked_plan_argument_checks():
    import ctypes
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    lib = ffsrqr.lib
    f = lib.ffsrqr_plan_blocked
    assert f(ctypes.byref(h), 200, 150, 40, 0, 8, 0, None, ctypes.byref(ws)) == -5
    assert f(ctypes.byref(h), 200, 150, 40, 12, 8, 0, None, ctypes.byref(ws)) == -5
    assert f(ctypes.byref(h), 200, 150, 40, 48, 8, 0, None, ctypes.byref(ws)) == -5
    assert f(ctypes.byref(h), 20, 150, 16, 16, 8, 0, None, ctypes.byref(ws)) == -6
    assert f(ctypes.byref(h), 200, 150, 40, 16, 8, 9, None, ctypes.byref(ws)) == -7
    assert f(ctypes.byref(h), 200, 150, 40, 16, 8, 0, None, None) == -9
    assert f(ctypes.byref(h), 200, 150, 40, 16, 8, 0, None, ctypes.byref(ws)) == 0
    assert lib.ffsrqr_destroy(h) == 0


@pytest.mark.parametrize("b", [8])
def test_blocked_exact_and_deficient_rank(b):
    # exactly rank k (a ragged last block of 4): the singular values are the
    # true ones; rank 5 < k = 16: the second block's sample is rounding noise,
    # its columns are orthogonalised against the first block's anyway, and
    # the approximation still holds the whole range
    import math
    B = synth.rank_k(256, 200, 12, seed=10).astype(np.float32)
    got = run(B, 12, b, 6, ffsrqr.PLAIN_FP32, seed=1)
    sv = np.linalg.svd(B.astype(np.float64), compute_uv=False)
    np.testing.assert_allclose(got["S"], sv[:12], rtol=2e-5)
    res = np.linalg.norm(B - (got["U"] * got["S"]) @ got["V"].T)
    assert res <= 1e-5 * sv[0] * math.sqrt(256 * 200)
    C = synth.rank_k(300, 240, 5, seed=12).astype(np.float32)
    got = run(C, 16, b, 6, ffsrqr.PLAIN_FP32, seed=2)
    sv = np.linalg.svd(C.astype(np.float64), compute_uv=False)
    assert got["info"]["status"] in (0, 1)
    np.testing.assert_allclose(got["S"][:5], sv[:5], rtol=2e-5)
    assert np.all(got["S"][5:] <= 2e-5 * sv[0])  # FP32 noise (measured 4.4e-6)
    res = np.linalg.norm(C - (got["U"] * got["S"]) @ got["V"].T)
    assert res <= 1e-5 * sv[0] * math.sqrt(300 * 240)
    assert np.allclose(got["U"][:, :5].T @ got["U"][:, :5], np.eye(5), atol=1e-4)
