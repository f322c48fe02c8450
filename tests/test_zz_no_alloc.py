"""ffsrqr_qrcp_static (QRCP of a sketch with library-owned static scratch, no
allocation) against the planned path: the same sketch B^T taken from a
ffsrqr_run workspace gives the same pivots and, within FP32 rounding of the
reflectors, the same S11 -- on two calls in a row, since every call must
clear the scratch words that start at zero."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1803_01982_gb300 import ffsrqr, synth  # noqa: E402

pytestmark = pytest.mark.gpu


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
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        piv.fill_(-1)
        s11.zero_()
        rc = ffsrqr.ffsrqr_qrcp_static(ctypes.c_void_p(bt.data_ptr()), n, s, lds, k,
                                       ctypes.c_void_p(piv.data_ptr()), ctypes.c_void_p(s11.data_ptr()),
                                       ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(stream))
        assert rc == 0, ffsrqr.ffsrqr_status_string(rc)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert piv.cpu().tolist() == piv_run[:k].cpu().tolist()
        scale = float(s11_ref.abs().max())
        assert torch.allclose(s11, s11_ref, atol=2e-6 * scale, rtol=0)


def test_static_qrcp_rejects_sizes_beyond_its_scratch():
    null = ctypes.c_void_p(0)
    dummy = torch.empty(4, device="cuda")
    ptr = ctypes.c_void_p(dummy.data_ptr())
    # n above 65536 columns and lds above 256 exceed the static scratch
    assert ffsrqr.ffsrqr_qrcp_static(ptr, 70000, 8, 8, 4, ptr, ptr, null, null) == 7
    assert ffsrqr.ffsrqr_qrcp_static(ptr, 100, 8, 260, 4, ptr, ptr, null, null) == 7
    assert ffsrqr.ffsrqr_qrcp_static(ptr, 100, 8, 4, 4, ptr, ptr, null, null) == -4
