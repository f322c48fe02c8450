"""Failure detection on the device without a GPU fault: every wait in this
library's kernels is bounded, and a wait that expires turns into
FFSRQR_STATUS_TIMEOUT in the run's report while the context stays usable.

The wait is made to run out on purpose with FFSRQR_FLAG_TEST_STALL: the grid
barrier of the sketch QRCP's last step then waits for one block more than
the cooperative grid holds -- an arrival that never comes.  Every block gives
up after its spin limit (about a second) and returns; the rest of the
pipeline runs to its own bounds on the unfinished factor; the status word
keeps the largest code, and TIMEOUT (3) is above every code the garbage
outputs can raise (rank deficiency 1, swap cap 2).  A normal run on the same
context afterwards must give bitwise the results it gave before."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1803_01982_gb300 import ffsrqr, synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", [ffsrqr.PLAIN_FP32, ffsrqr.MIXED])
def test_stalled_wait_reports_timeout_and_context_survives(mode):
    m, n, k, p = 900, 700, 24, 8
    A = synth.decayed(m, n, 0.9 ** np.arange(min(m, n)), 1e-4, seed=3)
    Ad = torch.as_tensor(A).cuda()
    good = ffsrqr.Plan(m, n, k, p, mode)
    ref = [t.clone() for t in good.run(Ad, seed=0)]
    torch.cuda.synchronize()
    assert good.info()["status"] == 0

    stall = ffsrqr.Plan(m, n, k, p, mode, flags=ffsrqr.FLAG_TEST_STALL)
    stall.workspace.zero_()
    t0 = time.time()
    stall.run(Ad, seed=0)
    torch.cuda.synchronize()
    elapsed = time.time() - t0
    assert stall.info()["status"] == 3, stall.info()
    assert elapsed < 30.0, elapsed  # bounded: about one spin limit, not a hang

    again = good.run(Ad, seed=0)
    torch.cuda.synchronize()
    assert good.info()["status"] == 0
    for a, b in zip(ref, again):
        assert torch.equal(a, b)
