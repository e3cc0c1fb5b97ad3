"""Serving: requests admitted into one running batch as they arrive and room
frees up give, each, bit for bit the result of the same simulation run alone
(FP32 storage: the tolerance is zero)."""
import numpy as np
import pytest

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


def small_stream(n=10, seed=216):
    """Like the serving stream but with small grids and short runs."""
    reqs = W.serving_stream(n_requests=n, seed=seed, edge_lo=20, edge_hi=56, steps_lo=30,
                            steps_hi=90, rate_hz=1.0)
    for r in reqs:
        r.workload.thr_mode, r.workload.tau = 1, 1e-6
        r.workload.decay_alpha, r.workload.decay_steps = 0.8, 5
    return reqs


def solo_field(wl):
    s = tcm.Sim.from_workload(wl)
    s.step(wl.steps)
    f = s.read_field(0)
    u = s.updates
    s.close()
    return f, u


def test_each_result_equals_solo_run():
    reqs = small_stream()
    # a pool that fits only a few requests at once, so admission has to wait
    srv = serve.Server(pool_bytes=600 * tcm.tcm_slot_bytes(), max_bricks=4000, max_sims=4,
                       steps_per_tick=7, keep_fields=True)
    res = srv.run(reqs, time_scale=1.0, virtual=True)
    srv.close()
    assert len(res) == len(reqs)
    by_id = {r.rid: r for r in res}
    overlapped = 0
    for r in res:
        others = [q for q in res if q.rid != r.rid and q.admitted < r.done and r.admitted < q.done]
        overlapped += bool(others)
    assert overlapped >= len(res) // 2, "requests should share the GPU"
    for q in reqs:
        f, u = solo_field(q.workload)
        got = by_id[q.rid]
        assert np.array_equal(got.field, f), q.rid
        assert got.cell_updates == u
        assert np.array_equal(got.plane, f[q.workload.shape[0] // 2])


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


def test_mixed_storage_lanes_equal_solo_runs():
    """FP32 and BF16 requests served side by side, one lane (batch) per
    storage: each result equals its solo run in the same storage, bit for bit."""
    reqs = small_stream(n=8, seed=77)
    assert {r.storage for r in reqs} == {"f32", "bf16"}
    srv = serve.Server(pool_bytes=900 * tcm.tcm_slot_bytes(), max_bricks=8000, max_sims=6,
                       steps_per_tick=9, keep_fields=True, storages=("f32", "bf16"))
    res = srv.run(reqs, time_scale=1.0, virtual=True)
    srv.close()
    assert len(res) == len(reqs)
    for r in res:
        q = reqs[r.rid]
        assert r.storage == q.storage
        s = tcm.Sim.from_workload(q.workload, storage=q.storage)
        s.step(q.workload.steps)
        assert np.array_equal(r.field, s.read_field(0)), q.rid
        assert r.cell_updates == s.updates
        s.close()
