"""Failure path of the kernels' bounded device waits, without a GPU fault.

The banded stage waits on other blocks' completion counters and the TMA-staged tiles wait
on an mbarrier; each wait gives up after a bounded number of polls and reports
WCNS_ERR_TIMEOUT through the sticky error word.  wcns_selftest_waits runs the same two
waits on a counter that nothing increments and an mbarrier that no copy fills: both must
give up within seconds, the status must say so, and the context must keep working.
"""
import time

import pytest

from paper_2306_09760_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    import torch
    assert torch.cuda.is_available()
    from paper_2306_09760_gb300 import build as wbuild
    wbuild.build()
    from paper_2306_09760_gb300 import wcns
    return wcns


def test_bounded_waits_give_up_and_the_context_stays_usable(W):
    import torch
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        S = W.Solver(inputs.riemann2d(256, seed=0), "f32", stream=stream)
        t0 = time.perf_counter()
        gave_up = W.wcns_selftest_waits(S.ctx)
        elapsed = time.perf_counter() - t0
        st, _ = S.status()
        S.step(0.0, 3)
        st2, _ = S.status()
        u = S.numpy()
        S.close()
    print(f"\nbounded waits gave up after {elapsed:.2f} s in all: {gave_up}")
    assert gave_up == [1, 1]
    assert st == W.WCNS_ERR_TIMEOUT, W.wcns_status_string(st)
    assert elapsed < 30.0
    assert st2 == W.WCNS_OK, W.wcns_status_string(st2)
    assert (u[0] > 0).all()
