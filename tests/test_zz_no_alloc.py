"""ffsrqr_qrcp_static: the sketch QRCP (Alg. 1 on B) with its scratch in a
fixed device array of the library, for callers that cannot allocate device
memory at the point of the call.

Checked here through the C ABI:
  * the same sketch B^T taken from a ffsrqr_run workspace gives the same
    pivots and, within FP32 rounding of the reflectors, the same S11 as the
    planned path -- on two calls in a row, since every call must clear the
    scratch words that start at zero;
  * the call allocates nothing: the device's free memory is the same before
    and after a call (any cudaMalloc takes at least a 2 MiB page);
  * k near the 256-row limit is accepted (pivots against the FP64 oracle);
  * a sketch with fewer finite columns than k reports FFSRQR_STATUS_NONFINITE
    and leaves the skipped steps' outputs as the caller had them;
  * sizes beyond the scratch are rejected.
This file is collected last, so a run that stops at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_1803_01982_gb300 import ffsrqr, synth  # noqa: E402

pytestmark = pytest.mark.gpu


def _call(bt, n, s, lds, k, piv, s11, status):
    stream = torch.cuda.current_stream().cuda_stream
    return ffsrqr.ffsrqr_qrcp_static(ctypes.c_void_p(bt.data_ptr()), n, s, lds, k,
                                     ctypes.c_void_p(piv.data_ptr()), ctypes.c_void_p(s11.data_ptr()),
                                     ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(stream))


@pytest.mark.parametrize("shape,k,p", [((700, 900), 24, 8), ((1500, 3001), 60, 10)])
def test_static_qrcp_matches_planned_path(shape, k, p):
    m, n = shape
    A = synth.decayed(m, n, 0.93 ** np.arange(min(m, n)), 1e-4, seed=5)
    plan = ffsrqr.Plan(m, n, k, p, ffsrqr.PLAIN_FP32)
    Ad = torch.as_tensor(A).cuda()
    _, _, _, piv_run = plan.run(Ad, seed=0)
    torch.cuda.synchronize()
    assert plan.info()["status"] == 0 and plan.info()["swaps"] == 0
    bt = plan.item("bt")            # n x s view, row stride lds
    s11_ref = plan.item("s11").clone()
    lds = bt.stride(0)
    s = k + p
    piv = torch.empty(k, dtype=torch.int32, device="cuda")
    s11 = torch.empty(k, k, dtype=torch.float32, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for call in range(2):
        piv.fill_(-1)
        s11.zero_()
        status.fill_(-1)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        rc = _call(bt, n, s, lds, k, piv, s11, status)
        assert rc == 0, ffsrqr.ffsrqr_status_string(rc)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        if call == 1:  # the first call on a device may load the library's module
            assert free1 == free0, (free0, free1)
        assert int(status.item()) == 0
        assert piv.cpu().tolist() == piv_run[:k].cpu().tolist()
        scale = float(s11_ref.abs().max())
        assert torch.allclose(s11, s11_ref, atol=2e-6 * scale, rtol=0)


def test_static_qrcp_k_near_row_limit():
    # s = lds = 256 rows (the scratch's limit), k = 240 pivots.  The k pivot
    # columns are orthogonal directions Q e_i scaled by 0.97^i, the others
    # are shorter than the last of them: projecting out a chosen direction
    # leaves the other pivot columns' norms unchanged and only shrinks the
    # rest, so the greedy order is exactly by scale, 3 % apart at every step.
    n, s, k = 1200, 256, 240
    rng = np.random.default_rng(11)
    Q, _ = np.linalg.qr(rng.standard_normal((s, s)))
    d = 0.97 ** np.arange(k)
    pos = rng.permutation(n)
    B = np.zeros((s, n))
    B[:, pos[:k]] = Q[:, :k] * d
    rest = rng.standard_normal((s, n - k))
    B[:, pos[k:]] = rest * (0.3 * d[-1] / np.linalg.norm(rest, axis=0))
    B = B.astype(np.float32)
    bt = torch.as_tensor(np.ascontiguousarray(B.T)).cuda()
    piv = torch.full((k,), -1, dtype=torch.int32, device="cuda")
    s11 = torch.zeros(k, k, dtype=torch.float32, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    assert _call(bt, n, s, s, k, piv, s11, status) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    perm, _, st = oracle.qrcp(B.astype(np.float64), k)
    assert st == 0
    assert piv.cpu().tolist() == list(perm[:k]) == pos[:k].tolist()


def test_static_qrcp_reports_nonfinite_sketch():
    # only 5 of 300 columns are finite and k = 8: steps 0..4 pick the finite
    # columns, steps 5..7 find no finite candidate and are skipped
    n, s, k, nf = 300, 16, 8, 5
    rng = np.random.default_rng(2)
    B = np.full((s, n), np.nan, dtype=np.float32)
    good = np.sort(rng.choice(n, nf, replace=False))
    B[:, good] = rng.standard_normal((s, nf)) * (0.5 ** np.arange(nf))[None, :]
    bt = torch.as_tensor(np.ascontiguousarray(B.T)).cuda()
    piv = torch.full((k,), -7, dtype=torch.int32, device="cuda")
    s11 = torch.full((k, k), 3.0, dtype=torch.float32, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    assert _call(bt, n, s, s, k, piv, s11, status) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 4
    got = piv.cpu().numpy()
    assert sorted(got[:nf].tolist()) == good.tolist()
    assert np.all(got[nf:] == -7)
    S = s11.cpu().numpy()
    assert np.all(np.isfinite(S[:nf, :nf]))
    # the skipped columns keep the caller's values (up to the row signs that
    # the non-negative-diagonal normalisation flips)
    assert np.all(np.abs(S[:, nf:]) == 3.0)


def test_static_qrcp_rejects_sizes_beyond_its_scratch():
    null = ctypes.c_void_p(0)
    dummy = torch.empty(4, device="cuda")
    ptr = ctypes.c_void_p(dummy.data_ptr())
    # n above 65536 columns and lds above 256 exceed the static scratch
    assert ffsrqr.ffsrqr_qrcp_static(ptr, 70000, 8, 8, 4, ptr, ptr, null, null) == 7
    assert ffsrqr.ffsrqr_qrcp_static(ptr, 100, 8, 260, 4, ptr, ptr, null, null) == 7
    assert ffsrqr.ffsrqr_qrcp_static(ptr, 100, 8, 4, 4, ptr, ptr, null, null) == -4
