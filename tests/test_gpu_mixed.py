"""GPU parity of the mixed-precision mode (FFSRQR_MIXED) against the FP64 oracle.

In this mode the sketch B = Omega A (Alg. 2) is formed on the tensor cores
from TF32 operands (about 2^-11 relative per operand), while passes 2 and 3,
the Cholesky-QR Grams and products and the output products use three TF32
products per term (head x head + head x tail + tail x head), which carries
FP32-level accuracy.

FFSRQR_MIXED_BF16X3 does the same with BF16 operands: a one-product BF16
sketch (about 2^-9 per operand) and three-product split-BF16 passes (about
2^-16 per product, random), judged by the same tolerances.

Consequences for the tests:
  * Pivots: the greedy order of Alg. 1 is compared with the oracle's on inputs
    whose column norms are graded by a factor >= 1/0.9 per step, so every
    top-2 trailing-norm gap (>= 19 % of the winner) is far above the TF32
    perturbation of the sketch.
  * After the pivots agree, the FP32 tolerances of the plain mode apply
    (singular values 2e-5 sigma_1 + 1e-5 sigma_j, 1e-5 relative in the head,
    residual 1e-4 relative, orthonormality 2e-5).
  * On inputs with a smoothly decaying spectrum the pivots may legitimately
    differ from the FP64 oracle's past the first near-tie; there the test
    checks properties any good rank-k factorisation has (head singular values
    within 1e-3 relative of the oracle's, residual within 1 % of the oracle's,
    orthonormal factors).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_1803_01982_gb300 import ffsrqr, synth  # noqa: E402

pytestmark = pytest.mark.gpu


def graded(m, n, ratio, seed):
    """Gaussian m x n with column j scaled by ratio^pi(j) for a seeded
    permutation pi: the greedy pivot order is pi^{-1}(0), pi^{-1}(1), ..."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((m, n))
    scale = ratio ** rng.permutation(n).astype(np.float64)
    return (G * scale).astype(np.float32)


def run(A, k, p, mode=ffsrqr.MIXED, seed=0):
    plan = ffsrqr.Plan(A.shape[0], A.shape[1], k, p, mode)
    Ad = torch.as_tensor(np.ascontiguousarray(A)).cuda()
    U, S, V, piv = plan.run(Ad, seed=seed)
    torch.cuda.synchronize()
    return plan, {"U": U.double().cpu().numpy(), "S": S.double().cpu().numpy(),
                  "V": V.double().cpu().numpy(), "piv": piv.cpu().numpy(), "info": plan.info(),
                  "ctl": plan.item("ctl")[0].cpu().numpy()}


def check_fp32(A, k, got, ref):
    S, So = got["S"], ref.S
    s1 = So[0]
    assert np.all(np.abs(S - So) <= 2e-5 * s1 + 1e-5 * So), np.max(np.abs(S - So) / s1)
    head = So >= 0.1 * s1
    assert np.all(np.abs(S - So)[head] <= 1e-5 * So[head])
    A64 = A.astype(np.float64)
    res = np.linalg.norm(A64 - (got["U"] * S) @ got["V"].T)
    res_o = oracle.residual_fro(A64, ref.U, ref.S, ref.V)
    assert abs(res - res_o) <= 1e-4 * res_o, (res, res_o)
    assert np.allclose(got["U"].T @ got["U"], np.eye(k), atol=2e-5)
    assert np.allclose(got["V"].T @ got["V"], np.eye(k), atol=2e-5)
    assert np.allclose(A64 @ got["V"], got["U"] * S, atol=2e-5 * s1)


@pytest.mark.parametrize("mode", [ffsrqr.MIXED_TF32X3, ffsrqr.MIXED_BF16X3])
@pytest.mark.parametrize("shape,k,p,ratio", [
    ((300, 240), 12, 6, 0.8),      # k below one MMA K block (16)
    ((1000, 800), 40, 10, 0.9),
    ((2100, 660), 64, 10, 0.9),    # ragged 128-row tiles and K blocks
    ((640, 1200), 33, 7, 0.85),    # wide
])
def test_mixed_graded_matches_oracle(shape, k, p, ratio, mode):
    m, n = shape
    A = graded(m, n, ratio, seed=m + n)
    _, got = run(A, k, p, mode)
    ref = oracle.ffsrqr(A, k, p, seed=0)
    assert got["info"]["status"] == ref.status == 0
    assert got["info"]["swaps"] == ref.swaps
    assert list(got["piv"][:k]) == list(ref.piv[:k])
    assert got["info"]["g2_first"] == pytest.approx(ref.g2_first, rel=1e-3)
    check_fp32(A, k, got, ref)
    # the three preconditioned QRs (panel, Z^T, Y_t) are well conditioned, so
    # each second Cholesky-QR sweep takes the first-order expansion
    ctl = got["ctl"]
    assert ctl[14] == 3 and ctl[15] == 0, ctl[13:16]
    # the QRCP certifies up to four pivots per grid barrier (word 38 counts them)
    assert -(-k // 4) <= ctl[38] < k, ctl[38]


@pytest.mark.parametrize("mode", [ffsrqr.MIXED_TF32X3, ffsrqr.MIXED_BF16X3])
def test_mixed_unaligned_rows_use_cuda_cores(mode):
    # a row stride that is not a multiple of 16 bytes cannot be a TMA operand;
    # the mode then runs its CUDA-core passes and must give the same results
    A = graded(500, 301, 0.85, seed=5)
    _, got = run(A, 20, 8, mode)
    ref = oracle.ffsrqr(A, 20, 8, seed=0)
    assert list(got["piv"][:20]) == list(ref.piv[:20])
    check_fp32(A, 20, got, ref)


@pytest.mark.parametrize("mode", [ffsrqr.MIXED_TF32X3, ffsrqr.MIXED_BF16X3])
@pytest.mark.parametrize("shape,k,p,decay", [
    ((2048, 1024), 64, 10, 0.97),
    ((1200, 1600), 48, 8, 0.95),
])
def test_mixed_decayed_properties(shape, k, p, decay, mode):
    m, n = shape
    A = synth.decayed(m, n, decay ** np.arange(min(m, n)), 1e-4, seed=17)
    _, got = run(A, k, p, mode)
    ref = oracle.ffsrqr(A, k, p, seed=0)
    S, So = got["S"], ref.S
    head = So >= 0.1 * So[0]
    assert np.all(np.abs(S - So)[head] <= 1e-3 * So[head])
    A64 = A.astype(np.float64)
    res = np.linalg.norm(A64 - (got["U"] * S) @ got["V"].T)
    res_o = oracle.residual_fro(A64, ref.U, ref.S, ref.V)
    assert res <= 1.01 * res_o, (res, res_o)
    assert np.allclose(got["U"].T @ got["U"], np.eye(k), atol=2e-5)
    assert np.allclose(got["V"].T @ got["V"], np.eye(k), atol=2e-5)


@pytest.mark.parametrize("mode", [ffsrqr.MIXED_TF32X3, ffsrqr.MIXED_BF16X3])
def test_mixed_deterministic(mode):
    A = graded(900, 700, 0.9, seed=3)
    _, a = run(A, 30, 10, mode)
    _, b = run(A, 30, 10, mode)
    for key in ["U", "S", "V", "piv"]:
        assert np.array_equal(a[key], b[key]), key


def test_plan_tune_keeps_results_within_tolerance():
    # the autotuner changes only launch shapes (pipeline depth, stream-K grid):
    # the tuned plan's results still match the oracle as before, and its
    # configuration is one of the candidates
    A = graded(2100, 660, 0.9, seed=2760)
    plan = ffsrqr.Plan(2100, 660, 64, 10, ffsrqr.MIXED_BF16X3)
    Ad = torch.as_tensor(A).cuda()
    cfg, ms = plan.tune(Ad)
    torch.cuda.synchronize()
    assert ms > 0 and len(cfg) == 7
    assert all(c == 0 or 2 <= c <= 8 for c in cfg[:3])
    assert cfg[3] >= 0 and all(c in (0, 1) for c in cfg[4:])
    U, S, V, piv = plan.run(Ad, seed=0)
    torch.cuda.synchronize()
    ref = oracle.ffsrqr(A, 64, 10, seed=0)
    got = {"U": U.double().cpu().numpy(), "S": S.double().cpu().numpy(), "V": V.double().cpu().numpy(),
           "piv": piv.cpu().numpy(), "info": plan.info()}
    assert list(got["piv"][:64]) == list(ref.piv[:64])
    check_fp32(A, 64, got, ref)
