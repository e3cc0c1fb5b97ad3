"""Serving: requests admitted into one running batch (FP32 and BF16 requests
in one batch of mixed storage, one launch per step for all) as they arrive
and as boxes free up, paused and resumed when the pool gets tight, give each
the oracle's result for the same simulation (bit for bit: FP32 in binary32,
BF16 in the oracle's storage form) and the result of the same simulation
run alone.  The bound on claimable boxes that admission relies on holds."""
import numpy as np
import pytest

import oracle
from paper_1702_00216_gb300 import serve, tcm
from paper_1702_00216_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def small_stream(n=10, seed=216, **kw):
    """Like the serving stream but with small grids and short runs."""
    kw.setdefault("rate_hz", 1.0)
    reqs = W.serving_stream(n_requests=n, seed=seed, edge_lo=20, edge_hi=56, steps_lo=30, steps_hi=90, **kw)
    for r in reqs:
        r.workload.thr_mode, r.workload.tau = 1, 1e-6
        r.workload.decay_alpha, r.workload.decay_steps = 0.8, 5
    return reqs


def oracle_run(wl, storage="f32"):
    o = oracle.OracleTCM(wl.shape, wl.media, wl.dx, wl.dt, brick=wl.brick, thr_mode=wl.thr_mode, tau=wl.tau,
                         decay_alpha=wl.decay_alpha, decay_steps=wl.decay_steps, storage=storage)
    for x, y, z, w in wl.sources:
        o.add_source(x, y, z, np.asarray(w, np.float32))
    o.step(wl.steps)
    r = (o.read_field(0), o.updates, o.active_count()[0])
    o.close()
    return r


def solo_run(wl, storage="f32"):
    s = tcm.Sim.from_workload(wl, storage=storage)
    s.step(wl.steps)
    r = (s.read_field(0), s.updates)
    s.close()
    return r


def test_served_results_equal_the_oracle_and_solo_runs():
    reqs = small_stream(n=12, seed=77)
    assert {r.storage for r in reqs} == {"f32", "bf16"}
    # a pool far smaller than the requests' grids: admission by footprint,
    # with peak footprints deliberately underestimated so that the running
    # waves outgrow the free boxes and get paused and resumed
    total = sum(serve.Server.bricks_of(q.workload) for q in reqs)
    srv = serve.Server(pool_bytes=700 * tcm.tcm_slot_bytes(), max_bricks=1 << 16, max_sims=8, steps_per_tick=7,
                       keep_fields=True, storages=("f32", "bf16"), peak_margin=0.1)
    res = srv.run(reqs, time_scale=1.0, virtual=True)
    srv.close()
    assert len(res) == len(reqs)
    # more grid bricks running at once than the pool has boxes: admission by
    # whole grids could not have run them together
    assert srv.stats["max_grid_bricks_running"] > srv.n_slots, srv.stats
    assert srv.stats["pauses"] > 0, srv.stats
    overlapped = sum(any(q.rid != r.rid and q.admitted < r.done and r.admitted < q.done for q in res) for r in res)
    assert overlapped >= len(res) // 2, "requests should share the GPU"
    assert total > 700
    for r in res:
        q = reqs[r.rid]
        assert r.storage == q.storage
        f, u, _ = oracle_run(q.workload, q.storage)
        assert np.array_equal(r.field, f), (q.rid, q.storage)
        assert r.cell_updates == u
        assert np.array_equal(r.plane, f[q.workload.shape[0] // 2])
        g, gu = solo_run(q.workload, q.storage)
        assert np.array_equal(r.field, g) and gu == u


def test_pause_and_resume_leave_results_unchanged():
    wls = [r.workload for r in small_stream(n=3, seed=5)]
    b = tcm.Batch(pool_bytes=3000 * tcm.tcm_slot_bytes(), max_bricks=1 << 16, max_sims=4)
    sims = [b.add(wl, n_steps=wl.steps) for wl in wls]
    b.step(10)
    b.pause(sims[1])
    b.step(17)
    b.pause(sims[2])
    b.resume(sims[1])
    b.step(11)
    b.resume(sims[2])
    for _ in range(40):
        b.step(5)
        if all(s.done() for s in sims):
            break
    assert all(s.done() for s in sims)
    for s, wl in zip(sims, wls):
        f, u, _ = oracle_run(wl)
        assert s.step_index == wl.steps
        assert np.array_equal(s.read_field(0), f) and s.updates == u
    b.close()


@pytest.mark.parametrize("T", [1, 9, 20])
def test_headroom_bounds_the_boxes_claimed(T):
    """At threshold 0 nothing is released, so the growth of the boxed sets
    over T steps is exactly the boxes claimed; it never exceeds the bound the
    library gave before the steps, and the bound never exceeds the unboxed
    cells.  The 26-neighbour schedule (Eq. 5 interval) is covered too."""
    reqs = small_stream(n=6, seed=31)
    for i, r in enumerate(reqs):
        r.workload.thr_mode, r.workload.tau, r.workload.decay_steps = 0, 0.0, 0
        if i % 2:
            r.workload.interval, r.workload.neighbours = 0, 26
    b = tcm.Batch(pool_bytes=20000 * tcm.tcm_slot_bytes(), max_bricks=1 << 16, max_sims=8)
    sims = [b.add(r.workload, n_steps=r.workload.steps) for r in reqs]
    grown = 0
    for _ in range(100 // T + 1):
        bound = b.headroom(T)
        before = sum(s.active_count()[0] for s in sims)
        unboxed = sum(serve.Server.bricks_of(r.workload) for r in reqs) - before
        assert 0 <= bound <= unboxed
        free_before = b.info()[1]
        b.step(T)
        after = sum(s.active_count()[0] for s in sims)
        assert after - before == free_before - b.info()[1]
        assert after - before <= bound, (after - before, bound)
        grown += after - before
    assert grown > 0
    b.close()


def test_mixed_storage_batch_steps_all_storages_in_one_launch():
    """FP32, BF16 and FP16 simulations in one batch of mixed storage: every
    step is one launch for all of them, and each equals the oracle in its
    storage form and its solo run."""
    wls = [r.workload for r in small_stream(n=3, seed=13)]
    storages = ["f32", "bf16", "f16"]
    b = tcm.Batch(pool_bytes=4000 * tcm.tcm_slot_bytes(), max_bricks=1 << 16, max_sims=4, storage="mixed")
    sims = [b.add(wl, n_steps=wl.steps, storage=st) for wl, st in zip(wls, storages)]
    steps = max(wl.steps for wl in wls)
    b.step(steps)
    assert sims[0].launches == steps
    for s, wl, st in zip(sims, wls, storages):
        f, u, n = oracle_run(wl, st)
        assert np.array_equal(s.read_field(0), f), st
        assert s.updates == u and s.active_count()[0] == n
        g, gu = solo_run(wl, st)
        assert np.array_equal(s.read_field(0), g) and gu == u
    with pytest.raises(tcm.TCMError) as e:
        tcm.tcm_set_storage(sims[0].handle, "bf16")    # after the first step
    assert e.value.status == tcm.TCM_ESTATE
    b.close()


def test_summary_percentiles():
    reqs = small_stream(n=6, seed=5)
    srv = serve.Server(pool_bytes=2000 * tcm.tcm_slot_bytes(), max_bricks=8000, max_sims=8,
                       steps_per_tick=16)
    import time
    t = time.perf_counter()
    res = srv.run(reqs, time_scale=0.0)          # all arrive at once
    wall = time.perf_counter() - t
    srv.close()
    s = serve.summarize(res, wall)
    assert s["requests"] == 6 and 0 < s["p50_s"] <= s["p99_s"] <= wall + 1e-6
    assert s["cell_updates"] > 0
