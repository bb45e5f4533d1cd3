"""GPU: device-side failure detection without a fault.

The tensor-core transform kernel's waits on its mbarriers are bounded (0.5 s
of %globaltimer); when one gives up, the kernel sets a device flag, drains
and returns, and the host reports SG_ETIMEOUT.  Here a wait runs out on a
barrier phase that nothing completes (sg_selftest_wait_timeout: count 1, no
arrival, no copy in flight): the test checks the status, the flag, that the
kernel returned after about the limit, and that the context is still usable
afterwards (a matvec against the oracle).
"""
import numpy as np
import pytest

from oracle import sg
from paper_2209_14740_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def test_bounded_wait_gives_up_and_context_survives():
    from paper_2209_14740_gb300 import binding as B
    status, timed_out, seconds = B.selftest_wait_timeout()
    assert status == B.SG_ETIMEOUT, B.STATUS_NAMES[status]
    assert timed_out == 1
    assert 0.4 <= seconds <= 5.0, seconds
    # the context still runs kernels and gives the oracle's answer
    pr = inputs.random_problem(5, dim=2, g=14, s=2, r=2)
    ref = sg.assemble_problem(pr)
    op = B.SG(pr)
    x = np.random.default_rng(5).standard_normal(op.N) + 1j * np.random.default_rng(6).standard_normal(op.N)
    X = torch.from_numpy(x).to(DEV)
    Y = torch.empty_like(X)
    op.matvec(X, Y, B.FP64)
    y = Y.cpu().numpy()
    scale = abs(ref.A) @ np.abs(x)
    assert np.all(np.abs(y - ref.A @ x) <= 1e-13 * scale)
    op.close()
    # and a second self-test behaves the same (the flag is per call)
    status2, timed_out2, _ = B.selftest_wait_timeout()
    assert status2 == B.SG_ETIMEOUT and timed_out2 == 1
