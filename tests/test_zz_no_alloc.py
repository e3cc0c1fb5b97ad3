"""tcm_energy_noalloc: the energy entry point that allocates nothing.

Callers that cannot call cudaMalloc/cudaFree mid-run (device memory owned by
another fixed-budget allocator, or a latency-critical path that must not
synchronise the device) use it instead of tcm_energy.  This checks, through
the C ABI, that two calls in a row give tcm_energy's value within the energy
tolerance used elsewhere in the tests (relative 1e-12) for every field
storage and inside a batch that changed since its last step, and that an
active list longer than the static scratch is rejected.  The file name makes pytest
collect it last.
"""
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


def _workload():
    shape = (24, 40, 33)
    media = W.random_dense_media(shape, 21, 1.0, 1.7)
    dt = 0.5 / media.c_max()
    return W.Workload("noalloc", shape, media, 1.0, dt, [(11, 20, 12, W.ricker(1 / 6, dt)),
                                                        (30, 3, 20, W.ricker(1 / 9, dt))], 0)


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
def test_energy_noalloc_matches_energy_twice(storage):
    """Two calls in a row (different states) for every field storage: the
    16-bit storages rebuild phi^{n-1} from phi^n and v^n in the energy."""
    import torch
    wl = _workload()
    sim = tcm.Sim.from_workload(wl, storage=storage)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    seen = []
    for steps, slot in ((25, 0), (60, 1)):          # two calls in a row, different states
        sim.step(steps)
        tcm.tcm_energy_noalloc(sim.handle, out[slot].data_ptr())
        torch.cuda.synchronize()
        ref = sim.energy()
        got = float(out[slot].item())
        assert ref != 0.0
        assert got == pytest.approx(ref, rel=1e-12)
        seen.append((sim.active_count()[0], got))
    assert seen[0][0] != seen[1][0] and seen[0][1] != seen[1][1]
    sim.close()


def test_energy_noalloc_in_a_batch_after_a_removal():
    """Two simulations in one batch: every entry of the shared active list
    that belongs to the other simulation contributes nothing; after the other
    simulation is removed (the batch changed since the last step) the call
    still works and equals tcm_energy."""
    import torch
    wl_a = _workload()
    wl_b = W.Workload("other", (32, 32, 32), W.homogeneous(1.0), 1.0, 0.5,
                      [(9, 20, 14, W.ricker(1 / 8, 0.5))], 0)
    b = tcm.Batch(pool_bytes=512 * tcm.tcm_slot_bytes(), max_bricks=8192, max_sims=4)
    sa, sb = b.add(wl_a), b.add(wl_b)
    b.step(30)
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    for i, s in enumerate((sa, sb)):
        tcm.tcm_energy_noalloc(s.handle, out[i].data_ptr())
        torch.cuda.synchronize()
        ref = s.energy()
        assert ref != 0.0
        assert float(out[i].item()) == pytest.approx(ref, rel=1e-12)
    b.remove(sb)
    tcm.tcm_energy_noalloc(sa.handle, out[2].data_ptr())
    torch.cuda.synchronize()
    assert float(out[2].item()) == pytest.approx(sa.energy(), rel=1e-12)
    b.step(5)
    tcm.tcm_energy_noalloc(sa.handle, out[3].data_ptr())
    torch.cuda.synchronize()
    assert float(out[3].item()) == pytest.approx(sa.energy(), rel=1e-12)
    assert float(out[3].item()) != float(out[2].item())
    b.close()


def test_energy_noalloc_rejects_active_sets_beyond_scratch():
    import torch
    # nz, ny, nx = 264, 512, 256: 33 * 64 * 32 = 67584 bricks, all active (dense) > 65536
    wl = W.Workload("big", (264, 512, 256), W.homogeneous(1.0), 1.0, 0.5, [], 0)
    sim = tcm.Sim.from_workload(wl, dense=True)
    sim.step(1)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(tcm.TCMError) as e:
        tcm.tcm_energy_noalloc(sim.handle, out.data_ptr())
    assert e.value.status == tcm.TCM_EINVAL
    sim.close()


def test_energy_noalloc_needs_a_started_sim():
    import torch
    wl = W.Workload("fresh", (16, 16, 16), W.homogeneous(1.0), 1.0, 0.5, [], 0)
    sim = tcm.Sim.from_workload(wl)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(tcm.TCMError) as e:
        tcm.tcm_energy_noalloc(sim.handle, out.data_ptr())
    assert e.value.status == tcm.TCM_ESTATE
    sim.close()
