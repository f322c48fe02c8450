"""GPU parity of Alg. 4's d-row random estimate of g2 against the FP64 oracle.

Both sides draw Omega_t (d x (l+1), fresh for every test t of a run) from
Philox stream 1 under the run's seed, each from its own implementation of the
generator.  In FP64 mode the device takes the same decisions as the oracle:
the same swaps, column selection, estimates (to rounding) and singular
values.  In FP32 the estimate of the first test is compared to FP32 accuracy,
and with no swap the outputs equal those of the exact-g2 run, since g2 only
decides whether swaps happen.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_1803_01982_gb300 import ffsrqr, synth  # noqa: E402

pytestmark = pytest.mark.gpu


def kahan_scaled(n, c, eps=1e-10):
    return synth.kahan(n, c) * (1.0 + eps * np.arange(n))[None, :]


def run(A, k, p, mode, g, d, seed=0, l=None):
    plan = ffsrqr.Plan(A.shape[0], A.shape[1], k, p, mode, g=g, l=l, g2_rows=d)
    dt = torch.float64 if mode == ffsrqr.FP64 else torch.float32
    Ad = torch.as_tensor(np.ascontiguousarray(A), dtype=dt).cuda()
    U, S, V, piv = plan.run(Ad, seed=seed)
    torch.cuda.synchronize()
    return {"U": U.double().cpu().numpy(), "S": S.double().cpu().numpy(),
            "V": V.double().cpu().numpy(), "piv": piv.cpu().numpy(), "info": plan.info()}


@pytest.mark.parametrize("n,c,k,p,g,d", [
    (48, 0.285, 30, 6, 1.05, 1),
    (48, 0.285, 30, 6, 1.05, 4),
    (64, 0.3, 40, 8, 1.1, 16),
    (96, 0.2, 50, 10, 1.02, 32),
])
def test_fp64_estimate_swaps_match_oracle(n, c, k, p, g, d):
    K = kahan_scaled(n, c)
    ref = oracle.ffsrqr(K, k, p, seed=0, g=g, g2_rows=d)
    got = run(K, k, p, ffsrqr.FP64, g, d)
    info = got["info"]
    assert ref.swaps > 0
    assert info["swaps"] == ref.swaps
    assert info["status"] == ref.status
    assert info["g2_first"] == pytest.approx(ref.g2_first, rel=1e-9)
    assert info["g2_final"] == pytest.approx(ref.g2_final, rel=1e-9)
    assert list(got["piv"][:k]) == list(ref.piv[:k])
    assert np.all(np.diff(got["piv"][k:]) > 0)
    np.testing.assert_allclose(got["S"], ref.S, rtol=1e-10, atol=1e-12 * ref.S[0])


def test_fp64_estimate_depth_l():
    # Omega_t has l + 1 columns at SRQR depth l
    K = kahan_scaled(64, 0.3)
    ref = oracle.ffsrqr(K, 30, 6, seed=5, g=1.1, l=36, g2_rows=4)
    got = run(K, 30, 6, ffsrqr.FP64, 1.1, 4, seed=5, l=36)
    assert got["info"]["swaps"] == ref.swaps
    assert got["info"]["g2_final"] == pytest.approx(ref.g2_final, rel=1e-9)
    np.testing.assert_allclose(got["S"], ref.S, rtol=1e-10, atol=1e-12 * ref.S[0])


@pytest.mark.parametrize("d", [1, 8, 32])
def test_fp32_estimate_first_test(d):
    m, n, k, p = 3000, 1700, 100, 10
    A = synth.decayed(m, n, (1.0 + np.arange(n)) ** -1.5, 1e-6, seed=7, dtype=np.float32)
    ref = oracle.ffsrqr(A, k, p, seed=3, g=5.0, g2_rows=d)
    got = run(A, k, p, ffsrqr.PLAIN_FP32, 5.0, d, seed=3)
    exact = run(A, k, p, ffsrqr.PLAIN_FP32, 5.0, 0, seed=3)
    assert ref.swaps == 0 and got["info"]["swaps"] == 0
    assert got["info"]["cand_first"] == ref.cand_first
    assert got["info"]["g2_first"] == pytest.approx(ref.g2_first, rel=1e-4)
    # g2 decided that no swap happens; everything else is the exact-g2 run
    for key in ("U", "S", "V", "piv"):
        np.testing.assert_array_equal(got[key], exact[key])


def test_fp32_estimate_swaps_meet_the_bound():
    K = kahan_scaled(96, 0.2).astype(np.float32)
    k, p, g = 50, 10, 1.02
    got = run(K, k, p, ffsrqr.PLAIN_FP32, g, 4)
    info = got["info"]
    assert info["swaps"] > 0
    assert info["g2_final"] <= g * (1 + 1e-5) or info["status"] == 2
    piv = got["piv"]
    assert sorted(piv.tolist()) == list(range(96))
    assert np.allclose(got["U"].T @ got["U"], np.eye(k), atol=2e-5)


def test_mixed_estimate_runs():
    A = synth.decayed(4096, 2048, (1.0 + np.arange(2048)) ** -1.5, 1e-6, seed=2, dtype=np.float32)
    got = run(A, 128, 10, ffsrqr.MIXED_BF16X3, 2.0, 8)
    assert got["info"]["status"] == 0
    assert np.allclose(got["V"].T @ got["V"], np.eye(128), atol=1e-4)


def test_set_g2_rows_errors():
    plan = ffsrqr.Plan(64, 48, 8, 4, ffsrqr.PLAIN_FP32)
    for bad in (-1, 33):
        with pytest.raises(ffsrqr.FfsrqrError, match="returned -2"):
            plan.set_g2_rows(bad)
    plan.set_g2_rows(0)
    plan.set_g2_rows(32)
    rsi = ffsrqr.Plan(64, 48, 8, 4, ffsrqr.PLAIN_FP32, rsi_q=1)
    with pytest.raises(ffsrqr.FfsrqrError, match="returned 7"):
        rsi.set_g2_rows(4)


def test_estimate_on_exact_rank():
    # alpha is rounding noise when A has rank k: the estimate's columns
    # R11^{-1}(alpha w_top - a w_k) stay finite (no division by alpha), and
    # whatever swaps the estimate asks for keep the factorisation exact
    import math
    B = synth.rank_k(256, 200, 12, seed=10).astype(np.float32)
    got = run(B, 12, 6, ffsrqr.PLAIN_FP32, 2.0, 4)
    info = got["info"]
    assert info["status"] in (0, 2)
    assert math.isfinite(info["g2_first"]) and math.isfinite(info["g2_final"])
    sv = np.linalg.svd(B.astype(np.float64), compute_uv=False)
    np.testing.assert_allclose(got["S"], sv[:12], rtol=2e-5)
    res = np.linalg.norm(B - (got["U"] * got["S"]) @ got["V"].T)
    assert res <= 1e-5 * sv[0] * math.sqrt(256 * 200)
