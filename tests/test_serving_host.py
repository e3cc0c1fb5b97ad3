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
    def __init__(self, pool_bytes, max_bricks, max_sims, device=0):
        self.slots = pool_bytes // 4096
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
