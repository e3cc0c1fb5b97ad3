"""Host logic of the serving loop (admission, reservations, completion) with
a fake batch in place of the GPU library."""
import numpy as np

from paper_1702_00216_gb300 import serve
from paper_1702_00216_gb300 import workloads as W


class FakeSim:
    def __init__(self, wl):
        self.wl = wl
        self.step_index = 0
        self.updates = 0

    def done(self):
        return self.step_index >= self.wl.steps

    def read_field(self, which=0, origin=(0, 0, 0), size=None):
        if size is None:
            size = (self.wl.nx, self.wl.ny, self.wl.nz)
        return np.zeros((size[2], size[1], size[0]), np.float32)

    def active_count(self):
        return (1, 512)


class FakeBatch:
    made = []

    def __init__(self, pool_bytes, max_bricks, max_sims, device=0, storage="f32"):
        self.slots = pool_bytes // (4096 if storage == "f32" else 2048)
        self.storage = storage
        self.max_sims = max_sims
        FakeBatch.made.append(self)
        self.sims = []
        self.peak = 0
        self.events = []

    def info(self):
        return (self.slots, self.slots, len(self.sims))

    def add(self, wl, n_steps=0, dense=False):
        s = FakeSim(wl)
        self.sims.append(s)
        self.peak = max(self.peak, len(self.sims))
        self.events.append(("add", wl.name))
        return s

    def step(self, n):
        for s in self.sims:
            if not s.done():
                k = min(n, s.wl.steps - s.step_index)
                s.step_index += k
                s.updates += k * 512

    def step_async(self, n):
        self.step(n)

    def sync(self):
        pass

    def remove(self, sim):
        self.sims.remove(sim)
        self.events.append(("remove", sim.wl.name))

    def close(self):
        pass


def test_admission_respects_capacity_and_finishes_everything(monkeypatch):
    monkeypatch.setattr(serve.tcm, "Batch", FakeBatch)
    reqs = W.serving_stream(n_requests=40, seed=3, edge_lo=16, edge_hi=64, steps_lo=10,
                            steps_hi=60, rate_hz=2.0)
    # 64^3 grid = 512 bricks; capacity of 1200 boxes holds two large requests at most
    srv = serve.Server(pool_bytes=1200 * 4096, max_bricks=4096, max_sims=5, steps_per_tick=5)
    res = srv.run(reqs, time_scale=1.0, virtual=True)
    assert sorted(r.rid for r in res) == [r.rid for r in reqs]
    assert srv.batch.peak <= 5
    assert srv.reserved_boxes == 0 and srv.reserved_bricks == 0 and not srv.running
    for r in res:
        q = reqs[r.rid]
        assert r.steps == q.workload.steps and r.cell_updates == q.workload.steps * 512
        assert r.admitted >= 0 and r.done >= r.admitted
    # admission order is arrival order
    adds = [e[1] for e in srv.batch.events if e[0] == "add"]
    assert adds == [q.workload.name for q in sorted(reqs, key=lambda q: q.arrival)]


def test_summarize():
    rs = [serve.Result(i, 0.0, 0.0, float(i + 1), 10, 100, 1) for i in range(100)]
    s = serve.summarize(rs, 10.0)
    assert s["requests"] == 100 and abs(s["p50_s"] - 50.5) < 1e-9 and s["p99_s"] > 99
    assert s["cell_updates_per_s"] == 1000.0


def test_lanes_route_by_storage():
    FakeBatch.made = []
    import pytest
    mp = pytest.MonkeyPatch()
    mp.setattr(serve.tcm, "Batch", FakeBatch)
    try:
        reqs = W.serving_stream(n_requests=30, seed=8, edge_lo=16, edge_hi=48, steps_lo=10,
                                steps_hi=40, rate_hz=3.0)
        assert {r.storage for r in reqs} == {"f32", "bf16"}
        srv = serve.Server(pool_bytes=2000 * 4096, max_bricks=8192, max_sims=6, steps_per_tick=4,
                           storages=("f32", "bf16"), pool_shares=(0.5, 0.5))
        res = srv.run(reqs, virtual=True)
        assert sorted(r.rid for r in res) == [r.rid for r in reqs]
        lanes = {b.storage: b for b in FakeBatch.made}
        assert set(lanes) == {"f32", "bf16"}
        # the BF16 lane holds twice the boxes of the FP32 one for the same bytes
        assert lanes["bf16"].slots == 2 * lanes["f32"].slots
        for r in res:
            assert r.storage == reqs[r.rid].storage
        for st, b in lanes.items():
            adds = [e[1] for e in b.events if e[0] == "add"]
            want = [q.workload.name for q in sorted(reqs, key=lambda q: q.arrival) if q.storage == st]
            assert adds == want and b.peak <= 3
        s = serve.summarize(res, 1.0)
        assert sum(s["by_storage"].values()) == 30
    finally:
        mp.undo()


def test_request_that_never_fits_is_refused(monkeypatch):
    monkeypatch.setattr(serve.tcm, "Batch", FakeBatch)
    reqs = W.serving_stream(n_requests=3, seed=1, edge_lo=64, edge_hi=65, steps_lo=5, steps_hi=6)
    srv = serve.Server(pool_bytes=100 * 4096, max_bricks=4096, max_sims=2)
    import pytest
    with pytest.raises(RuntimeError):
        srv.run(reqs, virtual=True)
