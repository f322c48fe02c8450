"""The host-buffer pipeline (ffsrqr_pipe_*): problems whose A and outputs live
in host memory, the copy of each problem's A overlapping the previous one's
computation.  Every output must be bitwise the device path's (ffsrqr_run on a
device copy of the same A), which the other GPU tests compare with the oracle."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1803_01982_gb300 import ffsrqr, synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", [ffsrqr.PLAIN_FP32, ffsrqr.MIXED])
def test_pipe_equals_device_runs(mode):
    m, n, k, p = 1500, 1200, 40, 10
    plan = ffsrqr.Plan(m, n, k, p, mode)
    pipe = ffsrqr.Pipe(plan)
    As, outs, seeds = [], [], []
    for i in range(5):
        A = synth.decayed(m, n, 0.95 ** np.arange(n), 1e-4, seed=30 + i)
        if i == 3:  # a padded host row stride
            Ap = np.zeros((m, n + 5), dtype=np.float32)
            Ap[:, :n] = A
            At = torch.from_numpy(Ap).pin_memory()[:, :n]
        else:
            At = torch.from_numpy(A).pin_memory()
        As.append(At)
        outs.append(pipe.host_outputs())
        seeds.append(7 * i)
    infos = pipe.run(As, outs, seeds)
    torch.cuda.synchronize()
    for i in range(5):
        U, S, V, piv = plan.run(As[i].cuda().contiguous(), seed=seeds[i])
        torch.cuda.synchronize()
        hU, hS, hV, hpiv = outs[i]
        assert torch.equal(hU, U.cpu()), i
        assert torch.equal(hS, S.cpu()), i
        assert torch.equal(hV, V.cpu()), i
        assert torch.equal(hpiv, piv.cpu()), i
        rep = ffsrqr.Info.from_buffer_copy(bytes(infos[i * ctypes.sizeof(ffsrqr.Info):
                                                        (i + 1) * ctypes.sizeof(ffsrqr.Info)].numpy()))
        assert rep.status == 0


def test_pipe_empty_and_invalid():
    plan = ffsrqr.Plan(300, 200, 10, 5, ffsrqr.PLAIN_FP32)
    pipe = ffsrqr.Pipe(plan)
    pipe.run([], [])  # nothing to do
    torch.cuda.synchronize()
    A = torch.zeros(300, 200).pin_memory()
    U, S, V, piv = pipe.host_outputs()
    bad = ffsrqr.HostProblem(A.data_ptr(), 100, 0, U.data_ptr(), U.stride(0), S.data_ptr(), V.data_ptr(),
                             V.stride(0), piv.data_ptr())  # lda < n
    arr = (ffsrqr.HostProblem * 1)(bad)
    rc = ffsrqr.lib.ffsrqr_pipe_run(pipe._h, arr, 1, pipe.device_mem.data_ptr() + pipe._off, plan.ws_ptr,
                                    None, None)
    assert rc == -2
    assert ffsrqr.lib.ffsrqr_pipe_run(None, arr, 1, None, None, None, None) == -1
