"""Continuous-batching request loop over one running batch of simulations.

Requests (workloads.Request: a simulation, its arrival time and its field
storage) are admitted into a running batch as soon as they have arrived and
the pool can take them.  Admission is by active footprint, not by grid size:
a simulation only holds boxes for the cells its wave occupies, and that
footprint grows with the simulation's step count while the requests admitted
earlier run towards their end and free their boxes.  The loop estimates each
request's footprint after s steps -- the cells within a little more than
the distance the wave travels in s steps (the Courant number times s, times
a margin) of a source, clipped to its grid: an estimate, not a bound -- and,
since every running simulation advances the same steps per tick, the
footprint of every running request at every future tick until it ends.  A
request is admitted when, added to those, its own predicted footprint fits
the pool at every future tick, and when the free boxes cover the upper bound
the library gives on the boxes the running simulations can claim during the
next tick (tcm_batch_headroom) plus the request's own (its source cells and
their neighbourhood within one tick's reach).  Before every tick the bound is
checked again; if the running simulations could claim more boxes than are
free, the most recently admitted ones are paused (tcm_batch_pause: they keep
their boxes and state and later continue unchanged) until it fits, and
paused ones are resumed, oldest first, as boxes free up.  If nothing can run,
the newest paused request is evicted (removed, its boxes freed) and queued
again from the start.  So the pool never runs out in the middle of a step.
``admission="dense"`` instead reserves a box for every brick of a request's
grid (the comparison).

FP32 and BF16 requests share one batch of mixed storage (each simulation its
own storage), so one persistent launch per step, replayed from captured CUDA
graphs, steps all of them.  Each tick steps the batch by `steps_per_tick`
launches; a simulation stops stepping when it has done its steps, its result
is read and it is removed, which frees its boxes, brick range and table slot.
Everything runs through the C ABI (tcm_batch_*).

Result of a request: the final phi^n on the plane z = nz // 2 (the whole
field with keep_fields), its active (boxed) brick count and node updates;
time to result = completion time - arrival time.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np

from . import tcm


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    done: float
    steps: int
    cell_updates: int
    active_bricks: int
    plane: Optional[np.ndarray] = None
    field: Optional[np.ndarray] = None
    storage: str = "f32"
    restarts: int = 0

    @property
    def time_to_result(self) -> float:
        return self.done - self.arrival


@dataclasses.dataclass
class _Running:
    req: object
    sim: object
    admitted: float
    bricks: int
    paused: bool = False
    reserve: int = 0


class Server:
    def __init__(self, pool_bytes: int, max_bricks: int, max_sims: int = 256, steps_per_tick: int = 8,
                 device: int = 0, keep_fields: bool = False, clock: Optional[Callable[[], float]] = None,
                 storage: str = "f32", storages: Optional[Sequence[str]] = None, admission: str = "footprint",
                 peak_margin: float = 1.25):
        """storage: the field storage of every request; storages: serve these
        storages side by side in one batch of mixed storage (requests carry
        their own).  admission: "footprint" (default) or "dense".  peak_margin:
        factor over the Courant speed in the estimate of a request's footprint
        (smaller admits more at once and pauses more)."""
        names = list(dict.fromkeys(storages)) if storages else [storage]
        self.mixed = len(names) > 1
        self.storages = names
        assert admission in ("footprint", "dense")
        self.admission = admission
        self.peak_margin = float(peak_margin)
        self.batch = tcm.Batch(pool_bytes=pool_bytes, max_bricks=max_bricks, max_sims=max_sims, device=device,
                               storage="mixed" if self.mixed else names[0])
        self.n_slots = self.batch.info()[0]
        self.max_bricks = max_bricks
        self.max_sims = max_sims
        self.steps_per_tick = int(steps_per_tick)
        self.keep_fields = keep_fields
        self._clock = clock or time.perf_counter
        self._t0 = None
        self.results: List[Result] = []
        self.updates = 0
        self.ticks = 0
        self._virtual = False
        self._scale = 1.0
        self.running: Dict[int, _Running] = {}      # in admission order
        self.queue: collections.deque = collections.deque()
        self.bricks_used = 0          # brick-table space of the running requests
        self.reserved_boxes = 0       # boxes reserved for whole grids (dense admission)
        self.restarts = collections.Counter()
        self.stats = {"max_concurrent": 0, "max_grid_bricks_running": 0, "pauses": 0, "resumes": 0,
                      "evictions": 0, "headroom_calls": 0}

    # ---- geometry -------------------------------------------------------
    @staticmethod
    def bricks_of(wl) -> int:
        nz, ny, nx = wl.shape
        bx, by, bz = wl.brick
        return -(-nx // bx) * -(-ny // by) * -(-nz // bz)

    def reach_cells(self, brick=(8, 8, 8)) -> int:
        """Cells within which a simulation can box new cells in one tick
        (the radius tcm_batch_headroom uses)."""
        return math.ceil(self.steps_per_tick / min(brick)) + 1

    def new_request_bound(self, wl) -> int:
        """Boxes a request can hold by the end of its first tick: its source
        cells and every cell within the tick's reach of them."""
        nz, ny, nx = wl.shape
        bx, by, bz = wl.brick
        m = (-(-nx // bx), -(-ny // by), -(-nz // bz))
        r = self.reach_cells(wl.brick)
        cells = set()
        for x, y, z, _ in wl.sources:
            c = (x // bx, y // by, z // bz)
            span = [range(max(0, c[d] - r), min(m[d], c[d] + r + 1)) for d in range(3)]
            for k in span[2]:
                for j in span[1]:
                    for i in span[0]:
                        cells.add((i, j, k))
        return min(len(cells), self.bricks_of(wl))

    @staticmethod
    def footprint_at(wl, steps_done, margin: float = 1.25) -> np.ndarray:
        """Estimated boxed cells of a request after each of `steps_done` steps:
        the cells within margin x (c_max dt / dx) x steps nodes of a source
        (values above the level travel at the wave speed; the margin covers
        the dispersion of Eq. 3 near the front), counted over the bounding box
        of that ball and clipped to the grid."""
        nz, ny, nx = wl.shape
        bx, by, bz = wl.brick
        courant = wl.media.c_max() * wl.dt / wl.dx
        R = np.ceil(margin * courant * np.asarray(steps_done, np.float64)).astype(np.int64) + 1
        total = np.zeros_like(R)
        for x, y, z, _ in wl.sources:
            n = np.ones_like(R)
            for c, size, b in ((x, nx, bx), (y, ny, by), (z, nz, bz)):
                n = n * (np.minimum(size - 1, c + R) // b - np.maximum(0, c - R) // b + 1)
            total = total + n
        return np.minimum(total, Server.bricks_of(wl))

    @staticmethod
    def peak_footprint(wl, margin: float = 1.25) -> int:
        """The estimate after the request's last step."""
        return int(Server.footprint_at(wl, [wl.steps], margin)[0])

    def trajectory(self, wl, step_now: int) -> np.ndarray:
        """Estimated boxed cells of a request at the end of each coming tick
        (index 0: the next tick) until the tick in which it ends."""
        rem = wl.steps - int(step_now)
        n = -(-rem // self.steps_per_tick) if rem > 0 else 0
        ends = np.minimum(int(step_now) + self.steps_per_tick * np.arange(1, n + 1), wl.steps)
        return self.footprint_at(wl, ends, self.peak_margin)

    def predicted_load(self) -> np.ndarray:
        """Sum over the running requests of their trajectories."""
        trajs = [self.trajectory(r.req.workload, r.sim.step_index) for r in self.running.values()]
        out = np.zeros(max([len(t) for t in trajs] + [0]), np.int64)
        for t in trajs:
            out[:len(t)] += t
        return out

    # ---- state ----------------------------------------------------------
    def now(self) -> float:
        """Seconds since the start of run(), or ticks in virtual mode."""
        if self._virtual:
            return float(self.ticks)
        return self._clock() - self._t0

    def free_boxes(self) -> int:
        return self.batch.info()[1]

    def headroom(self) -> int:
        self.stats["headroom_calls"] += 1
        return self.batch.headroom(self.steps_per_tick)

    def fits_empty(self, wl) -> bool:
        nb = self.bricks_of(wl)
        return nb <= self.n_slots and (nb + 31) // 32 * 32 <= self.max_bricks

    def _table_room(self, wl) -> bool:
        nb = self.bricks_of(wl)
        return len(self.running) < self.max_sims and self.bricks_used + (nb + 31) // 32 * 32 <= self.max_bricks

    # ---- admission ------------------------------------------------------
    def admit(self, req) -> None:
        wl = req.workload
        storage = getattr(req, "storage", self.storages[0]) if self.mixed else None
        sim = self.batch.add(wl, n_steps=wl.steps, storage=storage)
        nb = self.bricks_of(wl)
        self.bricks_used += (nb + 31) // 32 * 32
        reserve = nb if self.admission == "dense" else 0
        self.reserved_boxes += reserve
        self.running[req.rid] = _Running(req, sim, self.now(), nb, reserve=reserve)
        self.stats["max_concurrent"] = max(self.stats["max_concurrent"], len(self.running))
        # boxes that admission by whole grids would have had to reserve
        self.stats["max_grid_bricks_running"] = max(self.stats["max_grid_bricks_running"],
                                                    sum(r.bricks for r in self.running.values()))

    def _admit_arrived(self, time_scale: float) -> None:
        need = None
        free = None
        load = None
        while self.queue and self.queue[0].arrival * time_scale <= self.now() and self._table_room(self.queue[0].workload):
            wl = self.queue[0].workload
            if self.admission == "dense":
                if self.reserved_boxes + self.bricks_of(wl) > self.n_slots:
                    break
            else:
                if any(r.paused for r in self.running.values()):
                    break
                if load is None:
                    load = self.predicted_load()
                traj = self.trajectory(wl, 0)
                both = np.zeros(max(len(load), len(traj)), np.int64)
                both[:len(load)] += load
                both[:len(traj)] += traj
                if self.running and len(both) and int(both.max()) > self.n_slots:
                    break
                if need is None:
                    need, free = self.headroom(), self.free_boxes()
                est = self.new_request_bound(wl)
                if free - need < est:
                    break
                need += est
                load = both
            self.admit(self.queue.popleft())

    def _fit(self) -> None:
        """Pause the newest running simulations until the boxes they can claim
        in the next tick fit the free boxes; resume paused ones, oldest first,
        while they still fit; evict the newest paused one if nothing runs."""
        if self.admission == "dense" or not self.running:
            return
        while True:
            free = self.free_boxes()
            need = self.headroom()
            live = [rid for rid, r in self.running.items() if not r.paused]
            while need > free and len(live) > 0:
                rid = live.pop()
                self.batch.pause(self.running[rid].sim)
                self.running[rid].paused = True
                self.stats["pauses"] += 1
                need = self.headroom()
            for rid, r in self.running.items():
                if not r.paused:
                    continue
                self.batch.resume(r.sim)
                n2 = self.headroom()
                if n2 > free:
                    self.batch.pause(r.sim)
                    break
                r.paused = False
                self.stats["resumes"] += 1
                need = n2
            if any(not r.paused for r in self.running.values()):
                return
            # nothing can step: give the newest paused request's boxes back and
            # queue it again from the start
            rid = next(reversed(self.running))
            r = self.running.pop(rid)
            self.batch.remove(r.sim)
            self.bricks_used -= (r.bricks + 31) // 32 * 32
            self.reserved_boxes -= r.reserve
            self.queue.appendleft(r.req)
            self.restarts[rid] += 1
            self.stats["evictions"] += 1

    def collect(self) -> None:
        for rid in list(self.running):
            r = self.running[rid]
            if not r.sim.done():
                continue
            wl = r.req.workload
            nz, ny, nx = wl.shape
            plane = r.sim.read_field(0, origin=(0, 0, nz // 2), size=(nx, ny, 1))[0]
            field = r.sim.read_field(0) if self.keep_fields else None
            upd = r.sim.updates
            active = r.sim.active_count()[0]
            self.batch.remove(r.sim)
            self.bricks_used -= (r.bricks + 31) // 32 * 32
            self.reserved_boxes -= r.reserve
            self.updates += upd
            storage = getattr(r.req, "storage", self.storages[0]) if self.mixed else self.storages[0]
            self.results.append(Result(rid, r.req.arrival * self._scale, r.admitted, self.now(), wl.steps, upd,
                                       active, plane, field, storage, self.restarts[rid]))
            del self.running[rid]

    def run(self, requests, time_scale: float = 1.0, virtual: bool = False) -> List[Result]:
        """Serve requests (sorted by arrival, seconds x time_scale).  virtual=True
        admits by tick count instead of wall-clock time (arrival = tick index)."""
        for r in sorted(requests, key=lambda r: r.arrival):
            if not self.fits_empty(r.workload):
                raise RuntimeError(f"request {r.rid} can never fit this server")
            if self.mixed and getattr(r, "storage", "f32") not in self.storages:
                raise ValueError(f"request {r.rid}: storage {r.storage!r} not served")
            self.queue.append(r)
        self._t0 = self._clock()
        self._virtual = bool(virtual)
        self._scale = float(time_scale)
        while self.queue or self.running:
            self._admit_arrived(time_scale)
            self._fit()
            if self.running:
                self.batch.step_async(self.steps_per_tick)
                self.batch.sync()
                self.ticks += 1
                self.collect()
            else:
                nxt = self.queue[0].arrival * time_scale
                if virtual:
                    self.ticks = max(self.ticks + 1, int(np.ceil(nxt)))
                else:
                    wait = nxt - self.now()
                    if wait > 0:
                        time.sleep(min(wait, 0.05))
        return self.results

    def close(self):
        self.batch.close()


def summarize(results: List[Result], wall_s: float) -> dict:
    ttr = np.array([r.time_to_result for r in results]) if results else np.zeros(1)
    upd = sum(r.cell_updates for r in results)
    out = {"requests": len(results), "p50_s": float(np.percentile(ttr, 50)),
           "p99_s": float(np.percentile(ttr, 99)), "cell_updates": int(upd),
           "cell_updates_per_s": upd / wall_s if wall_s > 0 else 0.0, "wall_s": wall_s}
    by = collections.Counter(r.storage for r in results)
    if len(by) > 1:
        out["by_storage"] = dict(by)
    return out
