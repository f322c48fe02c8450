"""GPU parity of randomized subspace iteration (the paper's appendix algorithm,
ffsrqr_plan_rsi, through the C ABI) against the FP64 oracle
(``oracle.rsisvd``).  Both sides orthonormalise with diag(R) > 0 (Householder
in the oracle, CholeskyQR2 on the GPU), which fixes Q, so the results agree
within the Flip-Flop SRQR tolerances of each mode."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import rsisvd as ors  # noqa: E402
from paper_1803_01982_gb300 import ffsrqr, synth  # noqa: E402

pytestmark = pytest.mark.gpu


def run(A, k, p, q, mode, seed=0):
    dt = torch.float64 if mode == ffsrqr.FP64 else torch.float32
    pl = ffsrqr.Plan(A.shape[0], A.shape[1], k, p, mode, rsi_q=q)
    Ad = torch.as_tensor(np.ascontiguousarray(A), dtype=dt).cuda()
    U, S, V, _ = pl.run(Ad, seed=seed)
    torch.cuda.synchronize()
    return pl, U.double().cpu().numpy(), S.double().cpu().numpy(), V.double().cpu().numpy()


@pytest.mark.parametrize("q", [0, 1, 2])
def test_fp64_matches_oracle(q):
    A = synth.decayed(300, 240, 0.85 ** np.arange(240), 1e-4, seed=3, dtype=np.float64)
    pl, U, S, V = run(A, 10, 5, q, ffsrqr.FP64, seed=4)
    Uo, So, Vo = ors.rsisvd(A, 10, 5, q, seed=4)
    np.testing.assert_allclose(S, So, rtol=1e-11)
    assert np.max(np.abs(U - Uo)) <= 1e-9 and np.max(np.abs(V - Vo)) <= 1e-9
    assert pl.info()["status"] == 0


@pytest.mark.parametrize("mode", [ffsrqr.PLAIN_FP32, ffsrqr.MIXED])
@pytest.mark.parametrize("shape,k,p,q", [((600, 480), 16, 5, 1), ((517, 1031), 33, 7, 2), ((2048, 640), 64, 10, 1)])
def test_fp32_matches_oracle(mode, shape, k, p, q):
    m, n = shape
    A = synth.decayed(m, n, 0.95 ** np.arange(min(m, n)), 1e-4, seed=7)
    _, U, S, V = run(A, k, p, q, mode)
    Uo, So, Vo = ors.rsisvd(A, k, p, q)
    s1 = So[0]
    assert np.all(np.abs(S - So) <= 2e-5 * s1 + 1e-5 * So)
    assert np.allclose(U.T @ U, np.eye(k), atol=2e-5) and np.allclose(V.T @ V, np.eye(k), atol=2e-5)
    A64 = A.astype(np.float64)
    # U S V^T is the rank-k truncation of Q Q^T A: A^T U = V S on the captured subspace
    assert np.allclose(A64.T @ U, V * S, atol=2e-5 * s1)


def test_second_cholqr_sweep_falls_back_to_exact_factor():
    # sigma_j = 0.9^j and k + p = 50: the QRs here are not preconditioned and
    # their first sweeps leave ||Q^T Q - I|| of order cond^2 u ~ 1e-3 or more
    # (cond(A Omega) ~ 0.9^-50), above the expansion's limit, so second sweeps
    # factor their Grams exactly; the results must still match the oracle
    m, n, k, p, q = 1000, 800, 40, 10, 1
    A = synth.decayed(m, n, 0.9 ** np.arange(min(m, n)), 1e-4, seed=9)
    pl, U, S, V = run(A, k, p, q, ffsrqr.MIXED)
    ctl = pl.item("ctl")[0].cpu().numpy()
    # QRs: A Omega, then A^T Q and A Q per iteration, then the last A^T Q
    assert ctl[15] >= 1 and ctl[14] + ctl[15] == 2 + 2 * q, ctl[13:16]
    Uo, So, Vo = ors.rsisvd(A, k, p, q)
    s1 = So[0]
    assert np.all(np.abs(S - So) <= 2e-5 * s1 + 1e-5 * So)
    assert np.allclose(U.T @ U, np.eye(k), atol=2e-5) and np.allclose(V.T @ V, np.eye(k), atol=2e-5)


def test_plan_arguments():
    import ctypes
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    f = ffsrqr.lib.ffsrqr_plan_rsi
    assert f(ctypes.byref(h), 100, 80, 0, 5, 1, 0, None, ctypes.byref(ws)) == -4
    assert f(ctypes.byref(h), 100, 80, 10, 75, 1, 0, None, ctypes.byref(ws)) == -5
    assert f(ctypes.byref(h), 100, 80, 10, 5, -1, 0, None, ctypes.byref(ws)) == -6
    assert f(ctypes.byref(h), 100, 80, 10, 5, 1, 9, None, ctypes.byref(ws)) == -7
    assert f(ctypes.byref(h), 100, 80, 10, 5, 1, 0, None, None) == -9
