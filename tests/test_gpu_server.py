"""Request server (ffsrqr_server_*): admission under a device-memory budget
and continuous batching over concurrent streams.  Each request's result is
the same alone and in the mix (bit for bit: the same kernels on its own
workspace slice, whatever runs beside it); requests that arrive while others
are running are admitted as memory frees up; a request whose workspace
exceeds the whole budget is refused."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1803_01982_gb300 import ffsrqr, synth  # noqa: E402

pytestmark = pytest.mark.gpu


def svt_like_requests(count, seed):
    """Rank-r plus noise (r uniform in [10, 40]), m, n log-uniform in
    [300, 1500], k = r + 10, p = 10 -- a reduced copy of the serving workload."""
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        m, n = (int(round(np.exp(rng.uniform(np.log(300), np.log(1500))))) for _ in range(2))
        n += (-n) % 4
        r = int(rng.integers(10, 41))
        XL = rng.standard_normal((m, r))
        XR = rng.standard_normal((n, r))
        A = (XL @ XR.T + 1e-3 * rng.standard_normal((m, n))).astype(np.float32)
        reqs.append((torch.as_tensor(A).cuda(), r + 10, 10))
    return reqs


def alone(A, k, p, mode):
    m, n = A.shape
    plan = ffsrqr.Plan(m, n, k, p, mode)
    out = plan.outputs()
    plan.run(A, 0, out)
    torch.cuda.synchronize()
    return [t.cpu() for t in out]


def outputs_for(A, k):
    m, n = A.shape
    return (torch.empty(m, k, device="cuda"), torch.empty(k, device="cuda"), torch.empty(n, k, device="cuda"),
            torch.empty(n, dtype=torch.int32, device="cuda"))


@pytest.mark.parametrize("mode", [ffsrqr.PLAIN_FP32, ffsrqr.MIXED])
def test_results_same_alone_and_in_the_mix(mode):
    reqs = svt_like_requests(12, seed=1)
    ref = [alone(A, k, p, mode) for A, k, p in reqs]
    # budget for about two of the larger workspaces: most requests queue
    sizes = []
    for A, k, p in reqs:
        plan = ffsrqr.Plan(A.shape[0], A.shape[1], k, p, mode)
        sizes.append(plan.workspace.numel())
    budget = int(2.2 * max(sizes))
    srv = ffsrqr.Server(budget, slots=4)
    outs = [outputs_for(A, k) for A, k, _ in reqs]
    tickets = [srv.submit(A, k, p, mode, o) for (A, k, p), o in zip(reqs[:6], outs[:6])]
    first = srv.wait(tickets[0])  # later requests arrive while earlier ones run
    tickets += [srv.submit(A, k, p, mode, o) for (A, k, p), o in zip(reqs[6:], outs[6:])]
    results = [first] + [srv.wait(t) for t in tickets[1:]]
    st = srv.stats()
    srv.close()
    assert st["completed"] == 12 and st["queued"] == 0 and st["arena_free"] == budget // 256 * 256
    lat = [r[1] for r in results]
    assert all(x > 0 for x in lat)
    for (info, _), o, r in zip(results, outs, ref):
        assert info["status"] == 0
        for got, exp in zip(o, r):
            assert torch.equal(got.cpu(), exp)


def test_request_beyond_budget_is_refused():
    A = torch.randn(2000, 2000, device="cuda")
    srv = ffsrqr.Server(1 << 20, slots=2)  # 1 MiB cannot hold the workspace
    with pytest.raises(ffsrqr.FfsrqrError, match="returned 5"):
        srv.submit(A, 50, 10, ffsrqr.PLAIN_FP32, outputs_for(A, 50))
    srv.close()


@pytest.mark.parametrize("mode", [ffsrqr.PLAIN_FP32, ffsrqr.MIXED_BF16X3])
def test_same_phase_batching_shares_small_svd_launches(mode):
    # six requests submitted while admission is held are admitted in one pass;
    # with same-phase batching their small SVDs run in one launch per
    # thread-block-cluster size (k = r + 10 in [20, 50]: 4-block clusters, one
    # launch), and every result is still bitwise the request run alone
    reqs = svt_like_requests(6, seed=8)
    ref = [alone(A, k, p, mode) for A, k, p in reqs]
    srv = ffsrqr.Server(8 << 30, slots=6)
    srv.set_phase_batch(True)
    srv.pause(True)
    outs = [outputs_for(A, k) for A, k, _ in reqs]
    tickets = [srv.submit(A, k, p, mode, o) for (A, k, p), o in zip(reqs, outs)]
    srv.pause(False)
    results = [srv.wait(t) for t in tickets]
    ph = srv.phase_stats()
    srv.close()
    assert ph["grouped_requests"] == 6, ph
    clusters = {8 if k > 64 else (4 if k > 16 else 2) for _, k, _ in reqs}
    assert ph["small_svd_launches"] == len(clusters), ph
    for (info, lat), o, r in zip(results, outs, ref):
        assert info["status"] == 0 and lat > 0
        for got, exp in zip(o, r):
            assert torch.equal(got.cpu(), exp)
