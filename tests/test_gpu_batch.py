"""Batched problems as one CUDA graph (ffsrqr_batch_*): every problem's result
equals its standalone ffsrqr_run bit for bit (the same kernels in the same
order on its own workspace slice, whichever stream the graph gives it), on
the first (captured) and later (replayed) launches and after the
autotuner; one problem is also checked against the FP64 oracle.  In the
phase-batched graph the small SVDs of all problems run in one launch per
thread-block-cluster size, again bitwise as standalone."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_1803_01982_gb300 import ffsrqr, synth  # noqa: E402

pytestmark = pytest.mark.gpu


def uneven_problems(count, seed):
    """Sizes log-uniform in [256, 2048], k uniform in [8, 40], p = 10,
    sigma_j = 0.9^j -- a reduced copy of the 256-matrix batch workload."""
    rng = np.random.default_rng(seed)
    sizes, mats = [], []
    for i in range(count):
        m, n = (int(round(np.exp(rng.uniform(np.log(256), np.log(2048))))) for _ in range(2))
        n += (-n) % 4  # 16-byte rows for the tensor-core passes
        k = int(rng.integers(8, 41))
        r = min(m, n)
        A = synth.decayed(m, n, 0.9 ** np.arange(r), 1e-4, seed=100 + i)
        sizes.append((m, n, k, 10))
        mats.append(torch.as_tensor(A).cuda())
    return sizes, mats


def standalone(sizes, mats, mode):
    res = []
    for (m, n, k, p), A in zip(sizes, mats):
        plan = ffsrqr.Plan(m, n, k, p, mode)
        out = plan.outputs()
        plan.run(A, 0, out)
        torch.cuda.synchronize()
        res.append([t.cpu() for t in out])
    return res


@pytest.mark.parametrize("mode", [ffsrqr.PLAIN_FP32, ffsrqr.MIXED])
def test_batch_equals_standalone(mode):
    sizes, mats = uneven_problems(10, seed=4)
    ref = standalone(sizes, mats, mode)
    b = ffsrqr.Batch(sizes, mode, streams=4)
    outs = b.outputs()
    for launch in range(2):  # capture, then replay
        for o in outs:
            for t in o:
                t.zero_()
        b.run(mats, outs)
        torch.cuda.synchronize()
        for i, (o, r) in enumerate(zip(outs, ref)):
            for got, exp in zip(o, r):
                assert torch.equal(got.cpu(), exp), (launch, i)
            assert b.info(i)["status"] == 0


def test_batch_autotune_and_oracle():
    sizes, mats = uneven_problems(8, seed=9)
    b = ffsrqr.Batch(sizes, ffsrqr.PLAIN_FP32, streams=1)
    outs = b.outputs()
    chosen, ms = b.tune(mats, outs)
    assert chosen in (1, 2, 4, 8) and ms > 0
    assert ffsrqr.ffsrqr_batch_streams(b._h) == chosen
    b.run(mats, outs)
    torch.cuda.synchronize()
    ref = standalone(sizes, mats, ffsrqr.PLAIN_FP32)
    for o, r in zip(outs, ref):
        for got, exp in zip(o, r):
            assert torch.equal(got.cpu(), exp)
    # problem 0 against the oracle (FP32 tolerances of the parity tests)
    m, n, k, p = sizes[0]
    A = mats[0].cpu().numpy()
    so = oracle.ffsrqr(A, k, p, seed=0)
    S = outs[0][1].double().cpu().numpy()
    assert np.all(np.abs(S - so.S) <= 2e-5 * so.S[0] + 1e-5 * so.S)


@pytest.mark.parametrize("mode", [ffsrqr.PLAIN_FP32, ffsrqr.MIXED_BF16X3])
def test_phase_batched_graph_equals_standalone(mode):
    sizes, mats = uneven_problems(9, seed=21)
    # one problem with k > 64 (an 8-block cluster) beside the k <= 40 ones
    # (2- and 4-block clusters): three cluster sizes, three batched launches
    A = synth.decayed(1500, 1204, 0.97 ** np.arange(1204), 1e-4, seed=77)
    sizes.append((1500, 1204, 80, 10))
    mats.append(torch.as_tensor(A).cuda())
    ks = [sz[2] for sz in sizes]
    clusters = {8 if k > 64 else (4 if k > 16 else 2) for k in ks}
    ref = standalone(sizes, mats, mode)
    b = ffsrqr.Batch(sizes, mode, streams=4)
    b.set_phased(True)
    assert b.phased
    outs = b.outputs()
    for launch in range(2):  # capture, then replay
        for o in outs:
            for t in o:
                t.zero_()
        b.run(mats, outs)
        torch.cuda.synchronize()
        assert b.small_svd_launches() == len(clusters)
        for i, (o, r) in enumerate(zip(outs, ref)):
            for got, exp in zip(o, r):
                assert torch.equal(got.cpu(), exp), (launch, i)
            assert b.info(i)["status"] == 0
