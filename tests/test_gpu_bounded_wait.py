"""Failure detection without a GPU fault: the bounded mbarrier wait of the TMA-fed
kernels gives up on a barrier that nothing completes, reports it through its error
word, and the context stays usable."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_reports():
    import paper_1007_4895_gb300 as lb
    t0 = time.time()
    assert lb.lb_selftest_bounded_wait(polls=200000)
    assert time.time() - t0 < 30.0
    # the device is still usable afterwards
    from lbinputs import couette
    lat = lb.Lattice.from_workload(couette(nx=8, ny=16, rows=3), store="f32_dev")
    lat.step(10)
    assert np.isfinite(lat.moments()["ux"]).all()
    assert lat.reductions()["nonfinite"] == 0
