"""GPU parity of the Tucker drivers (ST-HOSVD, Alg. 6, and HOSVD, Alg. 5, on
Alg. 9, through the C ABI) against the FP64 oracle (``oracle.tucker`` with
Alg. 9 for every unfolding).

Per step the GPU and the oracle factor the same unfolding up to the rounding of
the previous steps, so the per-step singular values meet the single-run FP32
bounds (|dsigma_j| <= 2e-5 sigma_1 + 1e-5 sigma_j); on graded tensors (well
separated singular values) the factors and the core agree entry by entry after
the sign rule: column j of U_r within 1e-5 sigma_1 / sigma_j (a singular vector
moves by the perturbation over its gap, and the gaps scale with sigma_j on these
spectra) and the core within 1e-4 normwise in FP32; 1e-9 in FP64.  The mixed mode's
TF32 sketch may choose other pivots, so it is held to properties: head sigma
within 1e-3 and the approximation error within 1 % of the oracle's.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import tucker as ost  # noqa: E402
from paper_1803_01982_gb300 import ffsrqr, synth  # noqa: E402

pytestmark = pytest.mark.gpu


def graded(dims, seed=11, noise=1e-5):
    decay = [0.55 + 0.05 * r for r in range(len(dims))]
    return synth.tucker(dims, dims, decay, noise, seed=seed)


def run_gpu(X, ranks, order, p, mode, seed=0, method=ffsrqr.TUCKER_STHOSVD):
    t = ffsrqr.Tucker(X.shape, ranks, order, p, mode, method)
    dt = torch.float64 if mode == ffsrqr.FP64 else torch.float32
    Xd = torch.as_tensor(np.ascontiguousarray(X), dtype=dt).cuda()
    Us, Ss, core = t.run(Xd, seed=seed)
    torch.cuda.synchronize()
    return t, ([u.double().cpu().numpy() for u in Us], [s.double().cpu().numpy() for s in Ss],
               core.double().cpu().numpy())


CASES = [
    ((40, 36, 30), (6, 5, 4), (0, 1, 2), 4),        # first unfolding read in place
    ((37, 29, 23), (5, 6, 4), (2, 0, 1), 5),        # ragged: padded unfoldings, tiled transposes
    ((12, 10, 9, 8), (3, 4, 2, 3), (3, 1, 0, 2), 3),  # order 4
    ((300, 257), (8, 8), (1, 0), 6),                # order 2: second step is k x k exact
]


@pytest.mark.parametrize("dims,ranks,order,p", CASES)
def test_plain_fp32_matches_oracle(dims, ranks, order, p):
    X = graded(dims)
    t, (Us, Ss, core) = run_gpu(X, ranks, order, p, ffsrqr.PLAIN_FP32)
    G, Uo, So, rep = ost.sthosvd(X, ranks, order, p=p)
    assert [i["status"] for i in t.infos()] == [r["status"] for r in rep] == [0] * len(dims)
    for r in range(len(dims)):
        s1 = So[r][0]
        assert np.all(np.abs(Ss[r] - So[r]) <= 2e-5 * s1 + 1e-5 * So[r]), (r, Ss[r], So[r])
        assert np.allclose(Us[r].T @ Us[r], np.eye(ranks[r]), atol=2e-5)
        # a singular vector moves by about ||dA|| / gap, and gap_j ~ sigma_j on graded spectra
        tol_u = 1e-5 * So[r][0] / So[r]
        assert np.all(np.max(np.abs(Us[r] - Uo[r]), axis=0) <= tol_u), (r, np.abs(Us[r] - Uo[r]).max(0), tol_u)
    assert np.linalg.norm(core - G) <= 1e-4 * np.linalg.norm(G)
    assert t.launch_count() > len(dims)


def test_fp64_matches_oracle():
    dims, ranks, order, p = (37, 29, 23), (5, 6, 4), (2, 0, 1), 5
    X = graded(dims).astype(np.float64)
    t, (Us, Ss, core) = run_gpu(X, ranks, order, p, ffsrqr.FP64)
    G, Uo, So, _ = ost.sthosvd(X, ranks, order, p=p)
    for r in range(3):
        np.testing.assert_allclose(Ss[r], So[r], rtol=1e-10)
        assert np.max(np.abs(Us[r] - Uo[r])) <= 1e-9
    assert np.linalg.norm(core - G) <= 1e-10 * np.linalg.norm(G)


@pytest.mark.parametrize("dims,ranks,order,p", CASES[:3])
def test_mixed_properties(dims, ranks, order, p):
    X = graded(dims)
    _, (Us, Ss, core) = run_gpu(X, ranks, order, p, ffsrqr.MIXED)
    G, Uo, So, _ = ost.sthosvd(X, ranks, order, p=p)
    X64 = X.astype(np.float64)
    err = np.linalg.norm(X64 - ost.tucker_full(core, Us))
    err_o = np.linalg.norm(X64 - ost.tucker_full(G, Uo))
    assert err <= 1.01 * err_o + 1e-6 * np.linalg.norm(X64), (err, err_o)
    for r in range(len(dims)):
        head = So[r] >= 0.1 * So[r][0]
        assert np.all(np.abs(Ss[r] - So[r])[head] <= 1e-3 * So[r][head])
        assert np.allclose(Us[r].T @ Us[r], np.eye(ranks[r]), atol=2e-5)


def test_exact_multilinear_rank_any_order():
    dims, core_dims = (33, 28, 21), (4, 3, 5)
    X = synth.tucker(dims, core_dims, None, 0.0, seed=12)
    X64 = X.astype(np.float64)
    for order in [(0, 1, 2), (2, 1, 0)]:
        _, (Us, Ss, core) = run_gpu(X, core_dims, order, 4, ffsrqr.PLAIN_FP32)
        assert np.linalg.norm(X64 - ost.tucker_full(core, Us)) <= 2e-6 * np.linalg.norm(X64)


def test_deterministic_and_seeded():
    dims, ranks, order, p = (40, 36, 30), (6, 5, 4), (1, 2, 0), 4
    X = graded(dims)
    _, a = run_gpu(X, ranks, order, p, ffsrqr.MIXED, seed=3)
    _, b = run_gpu(X, ranks, order, p, ffsrqr.MIXED, seed=3)
    assert np.array_equal(a[2], b[2]) and all(np.array_equal(x, y) for x, y in zip(a[0], b[0]))


def test_full_size_400_cubed_mixed():
    """The benchmark's tensor (400^3, multilinear rank 40 + N(0, 1e-8) noise,
    ranks 40, p = 5) in the launch configuration bench.py times: the factor
    subspaces and the approximation agree with the oracle's."""
    dims, ranks = (400, 400, 400), (40, 40, 40)
    Xd = synth.tucker_torch(dims, ranks, 1e-4, seed=5)
    t = ffsrqr.Tucker(dims, ranks, None, 5, ffsrqr.MIXED)
    Us, Ss, core = t.run(Xd, seed=0)
    torch.cuda.synchronize()
    X = Xd.double().cpu().numpy()
    del Xd
    Us = [u.double().cpu().numpy() for u in Us]
    Ss = [s.double().cpu().numpy() for s in Ss]
    core = core.double().cpu().numpy()
    G, Uo, So, _ = ost.sthosvd(X, ranks, None, p=5)
    for r in range(3):
        assert np.allclose(Us[r].T @ Us[r], np.eye(40), atol=2e-5)
        dP = np.linalg.norm(Us[r] @ Us[r].T - Uo[r] @ Uo[r].T, 2)
        assert dP <= 1e-4, (r, dP)
        assert np.all(np.abs(Ss[r] - So[r]) <= 1e-4 * So[r])
    nx = np.linalg.norm(X)
    assert np.linalg.norm(ost.tucker_full(core, Us) - ost.tucker_full(G, Uo)) <= 2e-5 * nx


@pytest.mark.parametrize("dims,ranks,p", [((40, 36, 30), (6, 5, 4), 4), ((37, 29, 23), (5, 6, 4), 5),
                                           ((12, 10, 9, 8), (3, 4, 2, 3), 3)])
@pytest.mark.parametrize("mode", [ffsrqr.PLAIN_FP32, ffsrqr.MIXED])
def test_hosvd_matches_oracle(dims, ranks, p, mode):
    """Alg. 5: every factor is Alg. 9 on an unfolding of the same input, so the
    factors meet the single-run bounds; the core G = X x_r U_r^T is one product
    per mode (three-product TF32 in the mixed mode), within 1e-4 normwise."""
    X = graded(dims)
    t, (Us, Ss, core) = run_gpu(X, ranks, None, p, mode, method=ffsrqr.TUCKER_HOSVD)
    G, Uo, So, rep = ost.hosvd(X, ranks, p=p)
    assert [i["status"] for i in t.infos()] == [0] * len(dims)
    for r in range(len(dims)):
        assert np.allclose(Us[r].T @ Us[r], np.eye(ranks[r]), atol=2e-5)
        if mode == ffsrqr.PLAIN_FP32:
            s1 = So[r][0]
            assert np.all(np.abs(Ss[r] - So[r]) <= 2e-5 * s1 + 1e-5 * So[r])
            tol_u = 1e-5 * So[r][0] / So[r]
            assert np.all(np.max(np.abs(Us[r] - Uo[r]), axis=0) <= tol_u)
        else:
            head = So[r] >= 0.1 * So[r][0]
            assert np.all(np.abs(Ss[r] - So[r])[head] <= 1e-3 * So[r][head])
    X64 = X.astype(np.float64)
    if mode == ffsrqr.PLAIN_FP32:
        assert np.linalg.norm(core - G) <= 1e-4 * np.linalg.norm(G)
    # the core is the projection of X on the GPU's own factors
    Gp = X64
    for r in range(len(dims)):
        Gp = ost.mode_product(Gp, Us[r].T, r)
    assert np.linalg.norm(core - Gp) <= 1e-5 * np.linalg.norm(Gp)
    err = np.linalg.norm(X64 - ost.tucker_full(core, Us))
    err_o = np.linalg.norm(X64 - ost.tucker_full(G, Uo))
    assert err <= 1.01 * err_o + 1e-6 * np.linalg.norm(X64), (err, err_o)


def test_hosvd_fp64():
    dims, ranks, p = (37, 29, 23), (5, 6, 4), 5
    X = graded(dims).astype(np.float64)
    _, (Us, Ss, core) = run_gpu(X, ranks, None, p, ffsrqr.FP64, method=ffsrqr.TUCKER_HOSVD)
    G, Uo, So, _ = ost.hosvd(X, ranks, p=p)
    for r in range(3):
        np.testing.assert_allclose(Ss[r], So[r], rtol=1e-10)
        assert np.max(np.abs(Us[r] - Uo[r])) <= 1e-9
    assert np.linalg.norm(core - G) <= 1e-10 * np.linalg.norm(G)


def test_invalid_arguments():
    import ctypes
    lib = ffsrqr.lib
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    dims = (ctypes.c_int64 * 3)(10, 9, 8)
    ranks = (ctypes.c_int32 * 3)(2, 2, 2)
    bad_order = (ctypes.c_int32 * 3)(0, 0, 1)
    plan = lib.ffsrqr_tucker_plan
    assert plan(ctypes.byref(h), 2, 3, dims, ranks, None, 2, 0, None, ctypes.byref(ws)) == -2
    assert plan(ctypes.byref(h), 0, 1, dims, ranks, None, 2, 0, None, ctypes.byref(ws)) == -3
    assert plan(ctypes.byref(h), 0, 3, dims, ranks, bad_order, 2, 0, None, ctypes.byref(ws)) == -6
    big = (ctypes.c_int32 * 3)(2, 10, 2)
    assert plan(ctypes.byref(h), 0, 3, dims, big, None, 2, 0, None, ctypes.byref(ws)) == -5
    # k_r + p > m_j is rejected by the step's plan
    assert plan(ctypes.byref(h), 0, 3, dims, ranks, None, 8, 0, None, ctypes.byref(ws)) == -11
    assert plan(ctypes.byref(h), 1, 3, dims, ranks, None, 8, 0, None, ctypes.byref(ws)) == -11
    t = ffsrqr.Tucker((10, 9, 8), (2, 2, 2), None, 2)
    core = torch.empty(2, 2, 2, device="cuda")
    X = torch.zeros(10, 9, 8, device="cuda")
    u_null = (ctypes.c_void_p * 3)(None, None, None)
    assert lib.ffsrqr_tucker_run(t._h, X.data_ptr(), 0, u_null, None, core.data_ptr(), t.ws_ptr, None, None) == -4
    assert lib.ffsrqr_tucker_run(t._h, None, 0, u_null, None, core.data_ptr(), t.ws_ptr, None, None) == -2
