"""The bounded device-wide barrier of the step and filter kernels: with one
arrival missing it gives up after its time limit, records the timeout and
returns, and the device stays usable (no fault, no hang)."""
import time

import numpy as np
import pytest

from paper_1702_00216_gb300 import tcm
from paper_1702_00216_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def test_barrier_completes():
    rc, err = tcm.tcm_barrier_selftest(0, skew=0, timeout_s=0.05)
    assert (rc, err) == (tcm.TCM_OK, 0)


def test_barrier_times_out_and_device_stays_usable():
    t = time.perf_counter()
    rc, err = tcm.tcm_barrier_selftest(0, skew=1, timeout_s=0.05)
    dt = time.perf_counter() - t
    assert rc == tcm.TCM_ETIMEOUT and err & 2
    assert dt < 5.0
    # the context still works: a barrier that completes, then a simulation
    assert tcm.tcm_barrier_selftest(0, skew=0, timeout_s=0.05) == (tcm.TCM_OK, 0)
    wl = W.small(n=32, steps=20)
    s = tcm.Sim.from_workload(wl)
    s.step(20)
    assert np.isfinite(s.read_field(0)).all() and s.active_count()[0] > 0
    s.close()
