"""Failure detection without a GPU fault: an injected workspace-allocation
failure, and device waits that nothing ends (the bounded-wait exits of the TMA
mbarrier wait and of the persistent seeding kernel's counter wait).  Each must
come back as a status code with the context still usable."""
import numpy as np
import pytest

import oracle
from paper_2307_00071_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gira():
    from paper_2307_00071_gb300 import gira as g
    return g


def test_injected_allocation_failure_is_reported_and_cleared(gira):
    cl = synth.gmm_cloud(5_000, 4, seed=1)
    gira.gira_release_workspace()
    gira.gira_test_fail_next_allocations(1)
    with pytest.raises(gira.GiraError) as e:
        gira.gira_gmm_fit(cl.points, 4, iters=3, tol=0.0)
    assert e.value.status == gira.ERR_OOM
    assert "injected" in str(e.value)
    r = gira.gira_gmm_fit(cl.points, 4, iters=3, tol=0.0)   # the next call allocates normally
    ref = oracle.gmm_fit(cl.points, 4, iters=3, tol=0.0, reg=1e-6, seed=0, lloyd_iters=10)
    assert np.max(np.abs(r["trace"] - ref["trace"])) < 1e-5


def test_mbarrier_wait_times_out(gira):
    import time
    t0 = time.perf_counter()
    assert gira.gira_test_bounded_wait(0, 50_000_000) == gira.ERR_TIMEOUT   # 50 ms of wall time
    assert time.perf_counter() - t0 < 30.0


def test_counter_wait_times_out_and_context_survives(gira):
    assert gira.gira_test_bounded_wait(1, 100_000) == gira.ERR_TIMEOUT
    cl = synth.gmm_cloud(3_000, 3, seed=2)
    r = gira.gira_gmm_fit(cl.points, 3, iters=2, tol=0.0)
    assert r["iters_done"] == 2 and np.all(np.isfinite(r["trace"]))
