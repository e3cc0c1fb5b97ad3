"""Host logic of the serving loop (admission by footprint or by grid,
pausing, resuming, eviction, completion) with a fake batch in place of the
GPU library.  The fake boxes cells the way a pulse does -- the source cell at
the start, then the cells the loop's own estimate at the default margin
predicts for each step -- and fails loudly if the pool would run out, so a
correct loop never trips it."""
import numpy as np
import pytest

from paper_1702_00216_gb300 import serve
from paper_1702_00216_gb300 import workloads as W



def grown(wl, steps):
    """Cells a fake simulation has boxed after `steps` steps."""
    return int(serve.Server.footprint_at(wl, [steps])[0])


class FakeSim:
    def __init__(self, wl, batch):
        self.wl = wl
        self.batch = batch
        self.step_index = 0
        self.updates = 0
        self.nb = serve.Server.bricks_of(wl)
        self.boxed = 0
        self.started = False
        self.paused = False
        self.storage = None

    def done(self):
        return self.step_index >= self.wl.steps

    def read_field(self, which=0, origin=(0, 0, 0), size=None):
        if size is None:
            size = (self.wl.nx, self.wl.ny, self.wl.nz)
        return np.zeros((size[2], size[1], size[0]), np.float32)

    def active_count(self):
        return (self.boxed, self.boxed * 512)

    def live(self):
        return not self.paused and not self.done()


class FakeBatch:
    made = []

    def __init__(self, pool_bytes, max_bricks, max_sims, device=0, storage="f32"):
        self.slots = pool_bytes // (2048 * 3 // 2 if storage in ("bf16", "f16") else 4096)
        self.storage = storage
        self.max_sims = max_sims
        FakeBatch.made.append(self)
        self.sims = []
        self.peak = 0
        self.events = []

    def used(self):
        return sum(s.boxed for s in self.sims)

    def _start(self):
        for s in self.sims:
            if not s.started:
                s.started = True
                s.boxed = min(s.nb, len(s.wl.sources))
                assert self.used() <= self.slots, "pool exhausted at admission"

    def info(self):
        return (self.slots, self.slots - self.used(), len(self.sims))

    def headroom(self, steps):
        self._start()
        return sum(max(0, grown(s.wl, s.step_index + steps) - s.boxed) for s in self.sims if s.live())

    def add(self, wl, n_steps=0, dense=False, storage=None):
        s = FakeSim(wl, self)
        s.storage = storage
        self.sims.append(s)
        self.peak = max(self.peak, len(self.sims))
        self.events.append(("add", wl.name))
        return s

    def pause(self, sim):
        sim.paused = True
        self.events.append(("pause", sim.wl.name))

    def resume(self, sim):
        sim.paused = False
        self.events.append(("resume", sim.wl.name))

    def step(self, n):
        self._start()
        for _ in range(n):
            for s in self.sims:
                if s.live():
                    s.step_index += 1
                    s.updates += s.boxed * 512
                    s.boxed = max(s.boxed, grown(s.wl, s.step_index))
            if self.used() > self.slots:
                raise RuntimeError("pool exhausted in the middle of a step")

    def step_async(self, n):
        self.step(n)

    def sync(self):
        pass

    def remove(self, sim):
        self.sims.remove(sim)
        self.events.append(("remove", sim.wl.name))

    def close(self):
        pass


@pytest.fixture
def fake(monkeypatch):
    FakeBatch.made = []
    monkeypatch.setattr(serve.tcm, "Batch", FakeBatch)


def stream(n, seed, **kw):
    kw.setdefault("edge_lo", 16)
    kw.setdefault("edge_hi", 64)
    kw.setdefault("steps_lo", 10)
    kw.setdefault("steps_hi", 60)
    kw.setdefault("rate_hz", 2.0)
    return W.serving_stream(n_requests=n, seed=seed, **kw)


def check_done(srv, res, reqs):
    assert sorted(r.rid for r in res) == sorted(r.rid for r in reqs)
    assert not srv.running and srv.bricks_used == 0
    for r in res:
        q = next(x for x in reqs if x.rid == r.rid)
        assert r.steps == q.workload.steps and r.admitted >= 0 and r.done >= r.admitted


def test_footprint_admission_finishes_everything_and_never_exhausts(fake):
    reqs = stream(40, 3)
    # 64^3 grid = 512 cells: admitted by grid, 1200 boxes hold two such requests
    srv = serve.Server(pool_bytes=1200 * 4096, max_bricks=1 << 16, max_sims=16, steps_per_tick=5)
    res = srv.run(reqs, time_scale=1.0, virtual=True)
    check_done(srv, res, reqs)
    b = FakeBatch.made[-1]
    assert b.peak <= 16
    # admission follows arrival order (no request overtakes an earlier one)
    adds = [e[1] for e in b.events if e[0] == "add"]
    first = {}
    for i, name in enumerate(adds):
        first.setdefault(name, i)
    order = sorted(first, key=first.get)
    assert order == [q.workload.name for q in sorted(reqs, key=lambda q: q.arrival)]


def test_footprint_holds_more_simulations_than_dense_admission(fake):
    # short runs in large grids: the waves stay far smaller than the grids
    reqs = stream(30, 5, rate_hz=50.0, edge_lo=48, edge_hi=64, steps_lo=12, steps_hi=20)
    peaks = {}
    for adm in ("dense", "footprint"):
        srv = serve.Server(pool_bytes=1500 * 4096, max_bricks=1 << 16, max_sims=32, steps_per_tick=4,
                           admission=adm)
        res = srv.run(reqs, time_scale=1.0, virtual=True)
        check_done(srv, res, reqs)
        peaks[adm] = srv.stats["max_concurrent"]
    assert peaks["dense"] <= 1500 // 216 + 1          # 48^3 = 216 cells at least each
    assert peaks["footprint"] >= 2 * peaks["dense"], peaks


def test_pauses_and_resumes_when_growth_outruns_the_pool(fake):
    # few boxes, many long requests arriving together, and peak footprints
    # estimated far too small: running simulations outgrow the free boxes and
    # must be paused, then resumed
    reqs = stream(12, 9, rate_hz=1000.0, edge_lo=40, edge_hi=48, steps_lo=60, steps_hi=90)
    srv = serve.Server(pool_bytes=400 * 4096, max_bricks=1 << 16, max_sims=12, steps_per_tick=6,
                       peak_margin=0.02)
    res = srv.run(reqs, time_scale=1.0, virtual=True)
    check_done(srv, res, reqs)
    assert srv.stats["pauses"] > 0 and srv.stats["resumes"] > 0, srv.stats


def test_eviction_when_paused_simulations_hold_the_pool(fake):
    # each request alone fits (216-343 cells <= 360 boxes), but two grown ones
    # do not: the loop must evict and restart rather than stall
    reqs = stream(6, 11, rate_hz=1000.0, edge_lo=48, edge_hi=56, steps_lo=80, steps_hi=90)
    srv = serve.Server(pool_bytes=360 * 4096, max_bricks=1 << 16, max_sims=6, steps_per_tick=6,
                       peak_margin=0.02)
    res = srv.run(reqs, time_scale=1.0, virtual=True)
    check_done(srv, res, reqs)
    assert srv.stats["evictions"] > 0 and any(r.restarts for r in res), srv.stats


def test_dense_admission_reserves_whole_grids(fake):
    reqs = stream(20, 4)
    srv = serve.Server(pool_bytes=1200 * 4096, max_bricks=4096, max_sims=5, steps_per_tick=5,
                       admission="dense")
    res = srv.run(reqs, time_scale=1.0, virtual=True)
    check_done(srv, res, reqs)
    assert srv.reserved_boxes == 0 and srv.stats["pauses"] == 0
    assert FakeBatch.made[-1].peak <= 5


def test_mixed_storages_share_one_batch(fake):
    reqs = stream(30, 8, edge_hi=48, steps_hi=40, rate_hz=3.0)
    assert {r.storage for r in reqs} == {"f32", "bf16"}
    srv = serve.Server(pool_bytes=2000 * 4096, max_bricks=8192, max_sims=6, steps_per_tick=4,
                       storages=("f32", "bf16"))
    res = srv.run(reqs, virtual=True)
    check_done(srv, res, reqs)
    assert len(FakeBatch.made) == 1 and FakeBatch.made[0].storage == "mixed"
    for r in res:
        assert r.storage == reqs[r.rid].storage
    s = serve.summarize(res, 1.0)
    assert sum(s["by_storage"].values()) == 30


def test_summarize():
    rs = [serve.Result(i, 0.0, 0.0, float(i + 1), 10, 100, 1) for i in range(100)]
    s = serve.summarize(rs, 10.0)
    assert s["requests"] == 100 and abs(s["p50_s"] - 50.5) < 1e-9 and s["p99_s"] > 99
    assert s["cell_updates_per_s"] == 1000.0


def test_request_that_never_fits_is_refused(fake):
    reqs = W.serving_stream(n_requests=3, seed=1, edge_lo=64, edge_hi=65, steps_lo=5, steps_hi=6)
    srv = serve.Server(pool_bytes=100 * 4096, max_bricks=4096, max_sims=2)
    with pytest.raises(RuntimeError):
        srv.run(reqs, virtual=True)


def test_new_request_bound_covers_its_first_tick():
    """The bound the loop charges a new request: its source cell and all cells
    within the tick's reach, clipped to the grid."""
    wl = W.Workload("r", (40, 48, 56), W.homogeneous(1.0), 1.0, 0.5, [(3, 20, 39, W.ricker(0.1, 0.5))], 10)
    srv = serve.Server.__new__(serve.Server)
    srv.steps_per_tick = 16
    r = srv.reach_cells()
    assert r == 3
    # cell (0, 2, 4) of a 7 x 6 x 5 grid: x 0..3, y 0..5, z 1..4 -> 4 * 6 * 4
    assert srv.new_request_bound(wl) == 4 * 6 * 4


def test_peak_footprint_estimate():
    """The cells a wave can reach over a run at 1.25 x the Courant speed,
    clipped to the grid: 20 steps at Courant 0.5 reach 13.5 -> 14 nodes."""
    wl = W.Workload("p", (64, 64, 64), W.homogeneous(1.0), 1.0, 0.5, [(30, 5, 60, W.ricker(0.1, 0.5))], 20)
    # x 16..44 -> cells 2..5 (4), y 0..19 -> 0..2 (3), z 46..63 -> 5..7 (3)
    assert serve.Server.peak_footprint(wl) == 4 * 3 * 3
    long_run = W.Workload("q", (64, 64, 64), W.homogeneous(1.0), 1.0, 0.5, [(30, 5, 60, W.ricker(0.1, 0.5))], 900)
    assert serve.Server.peak_footprint(long_run) == 512


def test_peak_estimates_keep_the_loop_from_thrashing(fake):
    """With the default estimate of each request's peak footprint, a burst of
    long requests is admitted only as far as their peaks fit: no pauses or
    evictions are needed."""
    reqs = stream(12, 9, rate_hz=1000.0, edge_lo=40, edge_hi=48, steps_lo=60, steps_hi=90)
    srv = serve.Server(pool_bytes=400 * 4096, max_bricks=1 << 16, max_sims=12, steps_per_tick=6)
    res = srv.run(reqs, time_scale=1.0, virtual=True)
    check_done(srv, res, reqs)
    assert srv.stats["pauses"] == 0 and srv.stats["evictions"] == 0, srv.stats


def test_long_requests_are_staggered_beyond_dense_admission(fake):
    """A burst of identical requests whose waves end up filling their grids
    (216 cells each) in a pool of 600 boxes: dense admission runs two at a
    time; admission by predicted footprint starts a third while the first two
    are still running, because it stays small until they end (and the 125
    cells within its first tick's reach are free)."""
    def req(i):
        wl = W.Workload(f"long{i}", (48, 48, 48), W.homogeneous(1.0), 1.0, 0.5, [(24, 24, 24, W.ricker(1 / 8, 0.5))],
                        120)
        return W.Request(i, 0.0, wl, "f32")
    assert serve.Server.peak_footprint(req(0).workload) == 216
    peaks = {}
    for adm in ("dense", "footprint"):
        srv = serve.Server(pool_bytes=600 * 4096, max_bricks=1 << 16, max_sims=16, steps_per_tick=6,
                           admission=adm)
        reqs = [req(i) for i in range(8)]
        res = srv.run(reqs, time_scale=1.0, virtual=True)
        check_done(srv, res, reqs)
        peaks[adm] = srv.stats["max_concurrent"]
        if adm == "footprint":
            assert srv.stats["pauses"] == 0 and srv.stats["evictions"] == 0, srv.stats
    assert peaks["dense"] == 2
    assert peaks["footprint"] >= 3, peaks
