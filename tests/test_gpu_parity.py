"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (each derived from the arithmetic of the step it bounds):
  * Omega: the device evaluates Box-Muller in FP32 with CUDA's logf/sincospif,
    |z_gpu - z| <= 4e-6 (1 + |z|) against the FP64 definition; the raw Philox
    words are bit-identical.
  * FP32 path: singular values within 2e-5 sigma_1 + 1e-5 sigma_j (normwise
    FP32 rounding of three length-n/m reductions), relative 1e-5 where
    sigma_1/sigma_j <= 10; Frobenius residual within 1e-4 relative.
  * FP64 path: sigma and residual within 1e-11 relative.
  * Pivots: identical up to the first step whose top-2 trailing-norm gap is
    below 64 u sqrt(m) max_i ||B_i||^2 (the rounding bound of the sketch).
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
U32 = 2.0 ** -24


def run_gpu(A, k, p, mode=ffsrqr.PLAIN_FP32, seed=0, g=2.0, max_swaps=None):
    plan = ffsrqr.Plan(A.shape[0], A.shape[1], k, p, mode, g=g, max_swaps=max_swaps)
    dt = torch.float64 if mode == ffsrqr.FP64 else torch.float32
    Ad = torch.as_tensor(np.ascontiguousarray(A), dtype=dt).cuda()
    U, S, V, piv = plan.run(Ad, seed=seed)
    torch.cuda.synchronize()
    return plan, {"U": U.double().cpu().numpy(), "S": S.double().cpu().numpy(),
                  "V": V.double().cpu().numpy(), "piv": piv.cpu().numpy(), "info": plan.info()}


def well_separated_prefix(B, perm, k, m, u=U32):
    """Number of leading QRCP steps whose top-2 trailing-norm gap exceeds the
    rounding bound 64 u sqrt(m) max ||B_i||^2 (computed from the oracle's B)."""
    n = B.shape[1]
    thr = 64 * u * math.sqrt(m) * np.max(np.sum(B * B, axis=0))
    chosen = []
    for j in range(k):
        if chosen:
            Q, _ = np.linalg.qr(B[:, chosen])
            Rm = B - Q @ (Q.T @ B)
        else:
            Rm = B
        nr = np.sum(Rm * Rm, axis=0)
        nr[chosen] = -1
        top = np.sort(nr)[-2:]
        if top[1] - top[0] <= thr:
            return j
        chosen.append(int(perm[j]))
    return k


# ---------------------------------------------------------------------------
# Generator
# ---------------------------------------------------------------------------
def test_philox_raw_bit_exact():
    rng = np.random.default_rng(0)
    ck = rng.integers(0, 2 ** 32, size=(300, 6), dtype=np.uint64).astype(np.uint32)
    ck[0] = 0
    ck[1] = 0xFFFFFFFF
    dev_in = torch.from_numpy(ck.astype(np.int64)).to(torch.int32).cuda()
    out = torch.zeros(300 * 4, dtype=torch.int32, device="cuda")
    assert ffsrqr.ffsrqr_philox4x32_10(dev_in.data_ptr(), out.data_ptr(), 300, None) == 0
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.uint32).reshape(300, 4)
    for t in range(300):
        exp = oracle.philox(ck[t, :4], ck[t, 4:])
        assert list(got[t]) == list(exp), t


@pytest.mark.parametrize("mode", [ffsrqr.PLAIN_FP32, ffsrqr.FP64])
def test_omega_matches_oracle(mode):
    m, n, k, p = 1037, 300, 20, 10
    A = synth.decayed(m, n, 0.9 ** np.arange(n), 1e-3, seed=3, dtype=np.float64)
    plan, _ = run_gpu(A, k, p, mode, seed=12345)
    Om = plan.item("omega").double().cpu().numpy()
    ref = oracle.omega(12345, k + p, m)
    tol = 4e-6 if mode == ffsrqr.PLAIN_FP32 else 1e-14
    assert np.all(np.abs(Om - ref) <= tol * (1 + np.abs(ref)))


# ---------------------------------------------------------------------------
# Steps
# ---------------------------------------------------------------------------
def test_sketch_matches_oracle():
    m, n, k, p = 1200, 500, 24, 8
    A = synth.decayed(m, n, 0.9 ** np.arange(n), 1e-3, seed=4)
    plan, _ = run_gpu(A, k, p)
    Bt = plan.item("bt").double().cpu().numpy()
    Om = oracle.omega(0, k + p, m)
    B = Om @ A.astype(np.float64)
    absA = np.abs(A.astype(np.float64))
    bound = (m * U32 * (np.abs(Om) @ absA) + 4e-6 * ((1 + np.abs(Om)) @ absA))
    assert np.all(np.abs(Bt.T - B) <= bound)


@pytest.mark.parametrize("shape,k,p,decay,seed", [
    ((700, 500), 20, 10, 0.93, 1),
    ((333, 901), 17, 5, 0.9, 2),
    ((1500, 257), 40, 10, 0.97, 3),
])
def test_pivots_match_oracle(shape, k, p, decay, seed):
    m, n = shape
    A = synth.decayed(m, n, decay ** np.arange(min(m, n)), 1e-4, seed=seed)
    _, got = run_gpu(A, k, p)
    ref = oracle.ffsrqr(A, k, p, seed=0, trace=True)
    nsep = well_separated_prefix(ref.trace["B"], ref.trace["perm0"], k, m)
    assert nsep >= min(k, 5)
    if ref.swaps == 0 and got["info"]["swaps"] == 0:
        assert list(got["piv"][:nsep]) == list(ref.piv[:nsep])
    # the remaining columns are listed once each, ascending
    rest = got["piv"][k:]
    assert np.all(np.diff(rest) > 0)
    assert sorted(np.concatenate([got["piv"][:k], rest])) == list(range(n))


def _check_fp32_result(A, k, p, got, ref):
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


@pytest.mark.parametrize("shape,k,p,decay", [
    ((600, 480), 16, 8, 0.9),
    ((517, 1031), 33, 7, 0.95),
    ((2048, 640), 64, 10, 0.97),
    ((300, 300), 1, 5, 0.8),
])
def test_plain_fp32_matches_oracle(shape, k, p, decay):
    m, n = shape
    A = synth.decayed(m, n, decay ** np.arange(min(m, n)), 1e-4, seed=7)
    _, got = run_gpu(A, k, p)
    ref = oracle.ffsrqr(A, k, p, seed=0)
    assert got["info"]["status"] == ref.status == 0
    assert got["info"]["swaps"] == ref.swaps
    assert got["info"]["g2_first"] == pytest.approx(ref.g2_first, rel=1e-3)
    _check_fp32_result(A, k, p, got, ref)


def test_fp64_config1():
    A = synth.config1()
    k, p = 20, 5
    _, got = run_gpu(A, k, p, ffsrqr.FP64)
    ref = oracle.ffsrqr(A, k, p, seed=0)
    assert list(got["piv"][:k]) == list(ref.piv[:k])
    np.testing.assert_allclose(got["S"], ref.S, rtol=1e-11)
    res = np.linalg.norm(A - (got["U"] * got["S"]) @ got["V"].T)
    assert res == pytest.approx(oracle.residual_fro(A, ref.U, ref.S, ref.V), rel=1e-11)
    np.testing.assert_allclose(np.abs(got["U"].T @ ref.U), np.eye(k), atol=1e-8)


def test_k_equals_n_and_exact_rank():
    A = synth.rank_k(120, 40, 40, seed=9).astype(np.float32)
    _, got = run_gpu(A, 40, 5)
    sv = np.linalg.svd(A.astype(np.float64), compute_uv=False)
    np.testing.assert_allclose(got["S"], sv, rtol=2e-5, atol=2e-5 * sv[0])
    B = synth.rank_k(256, 200, 12, seed=10).astype(np.float32)
    _, got = run_gpu(B, 12, 6)
    sv = np.linalg.svd(B.astype(np.float64), compute_uv=False)
    np.testing.assert_allclose(got["S"], sv[:12], rtol=2e-5)
    res = np.linalg.norm(B - (got["U"] * got["S"]) @ got["V"].T)
    assert res <= 1e-5 * sv[0] * math.sqrt(256 * 200)


def test_deterministic():
    A = synth.decayed(800, 600, 0.93 ** np.arange(600), 1e-4, seed=11)
    _, a = run_gpu(A, 30, 10)
    _, b = run_gpu(A, 30, 10)
    for key in ["U", "S", "V", "piv"]:
        assert np.array_equal(a[key], b[key]), key


def test_plain_fp32_largest_k():
    """k = 224, the largest rank the FP32 plan accepts (7 x 32 columns per row
    solve; k^2 * 4 bytes <= 200 KiB of shared memory): the small SVD's QR and
    cluster Jacobi at their limits.  k = 225 is refused at plan time."""
    with pytest.raises(ffsrqr.FfsrqrError):
        ffsrqr.Plan(1400, 1100, 225, 10, ffsrqr.PLAIN_FP32)
    m, n, k, p = 1400, 1100, 224, 10
    A = synth.decayed(m, n, 0.985 ** np.arange(min(m, n)), 1e-4, seed=21)
    _, got = run_gpu(A, k, p)
    ref = oracle.ffsrqr(A, k, p, seed=0)
    assert got["info"]["status"] == ref.status == 0
    # past the first near-tie the FP32 pivots may differ from the FP64 oracle's:
    # properties any good rank-k factorisation has
    S, So = got["S"], ref.S
    head = So >= 0.1 * So[0]
    assert np.all(np.abs(S - So)[head] <= 1e-3 * So[head])
    A64 = A.astype(np.float64)
    res = np.linalg.norm(A64 - (got["U"] * S) @ got["V"].T)
    assert res <= 1.01 * oracle.residual_fro(A64, ref.U, ref.S, ref.V)
    # U = Q_t J and V = V' W with the small SVD's columns normalised (the
    # rounding drift of the rotations removed): both orthonormal to 2e-5
    eu = np.max(np.abs(got["U"].T @ got["U"] - np.eye(k)))
    ev = np.max(np.abs(got["V"].T @ got["V"] - np.eye(k)))
    assert eu <= 2e-5, eu
    assert ev <= 2e-5, ev
    assert np.allclose(A64 @ got["V"], got["U"] * S, atol=2e-5 * S[0])


def test_fp64_largest_k():
    """k = 160, the largest rank the FP64 plan accepts (k^2 * 8 bytes <= 200 KiB)."""
    m, n, k, p = 900, 700, 160, 8
    A = synth.decayed(m, n, 0.98 ** np.arange(min(m, n)), 1e-6, seed=22).astype(np.float64)
    _, got = run_gpu(A, k, p, ffsrqr.FP64)
    ref = oracle.ffsrqr(A, k, p, seed=0)
    assert got["info"]["status"] == ref.status == 0
    assert list(got["piv"][:k]) == list(ref.piv[:k])
    np.testing.assert_allclose(got["S"], ref.S, rtol=1e-10)
    res = np.linalg.norm(A - (got["U"] * got["S"]) @ got["V"].T)
    assert res == pytest.approx(oracle.residual_fro(A, ref.U, ref.S, ref.V), rel=1e-10)
    np.testing.assert_allclose(got["U"].T @ got["U"], np.eye(k), atol=1e-12)
    np.testing.assert_allclose(got["V"].T @ got["V"], np.eye(k), atol=1e-12)


@pytest.mark.parametrize("mode", [ffsrqr.PLAIN_FP32, ffsrqr.MIXED, ffsrqr.FP64])
def test_depth_l_returns_the_leading_triplets(mode):
    """ffsrqr_plan_l (Alg. 9 with SRQR depth l > k) returns exactly the leading
    k triplets and the pivots of the depth-l factorisation, and matches the
    oracle's depth-l run."""
    m, n, k, l, p = 600, 480, 16, 21, 8
    A = synth.decayed(m, n, 0.9 ** np.arange(min(m, n)), 1e-4, seed=7)
    dt = torch.float64 if mode == ffsrqr.FP64 else torch.float32
    Ad = torch.as_tensor(A, dtype=dt).cuda()
    pl = ffsrqr.Plan(m, n, k, p, mode, l=l)
    U, S, V, piv = pl.run(Ad, seed=0)
    full = ffsrqr.Plan(m, n, l, p, mode)
    Uf, Sf, Vf, pivf = full.run(Ad, seed=0)
    torch.cuda.synchronize()
    assert ffsrqr.ffsrqr_plan_depth(pl._h) == l
    assert torch.equal(S, Sf[:k]) and torch.equal(U, Uf[:, :k]) and torch.equal(V, Vf[:, :k])
    assert torch.equal(piv, pivf)
    ref = oracle.ffsrqr(A, k, p, seed=0, l=l)
    So = ref.S
    Sg = S.double().cpu().numpy()
    if mode == ffsrqr.FP64:
        np.testing.assert_allclose(Sg, So, rtol=1e-11)
    elif mode == ffsrqr.PLAIN_FP32:
        assert np.all(np.abs(Sg - So) <= 2e-5 * So[0] + 1e-5 * So)
    else:  # the TF32 sketch may pick other pivots: the smooth-input bound of the mixed mode
        head = So >= 0.1 * So[0]
        assert np.all(np.abs(Sg - So)[head] <= 1e-3 * So[head])
