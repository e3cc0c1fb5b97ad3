"""Continuous-batching request loop over running batches of simulations.

Requests (workloads.Request: a simulation, its arrival time and its field
storage) are admitted into a running batch as soon as they have arrived and
the batch has room -- free boxes in the pool for the request's whole brick
count (so the pool can never run out mid-run), brick-table space and a
simulation slot.  A server runs one batch per field storage it serves
("lanes", e.g. FP32 and BF16, each with its own share of the pool); a request
goes to the lane of its storage and waits only behind earlier requests of
that lane.  Each tick steps every lane with running simulations by
`steps_per_tick` launches; a simulation stops stepping when it has done its
steps, its result is read and it is removed, which frees its boxes and brick
range for waiting requests.  Everything runs through the C ABI (tcm_batch_*).

Result of a request: the final phi^n on the plane z = nz // 2, its active
(boxed) brick count and node updates; time to result = completion time -
arrival time.
"""
from __future__ import annotations

import collections
import dataclasses
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

    @property
    def time_to_result(self) -> float:
        return self.done - self.arrival


class Lane:
    """One running batch with one field storage and its capacity accounting."""

    def __init__(self, storage: str, pool_bytes: int, max_bricks: int, max_sims: int, device: int):
        self.storage = storage
        self.batch = tcm.Batch(pool_bytes=pool_bytes, max_bricks=max_bricks, max_sims=max_sims,
                               device=device, storage=storage)
        self.n_slots = self.batch.info()[0]
        self.max_bricks = max_bricks
        self.max_sims = max_sims
        self.reserved_boxes = 0
        self.reserved_bricks = 0
        self.running: Dict[int, tuple] = {}
        self.queue: collections.deque = collections.deque()

    def fits_empty(self, wl) -> bool:
        nb = Server.bricks_of(wl)
        return nb <= self.n_slots and (nb + 31) // 32 * 32 <= self.max_bricks

    def fits(self, wl) -> bool:
        nb = Server.bricks_of(wl)
        return (len(self.running) < self.max_sims and self.reserved_boxes + nb <= self.n_slots
                and self.reserved_bricks + (nb + 31) // 32 * 32 <= self.max_bricks)


class Server:
    def __init__(self, pool_bytes: int, max_bricks: int, max_sims: int = 256,
                 steps_per_tick: int = 8, device: int = 0, keep_fields: bool = False,
                 clock: Optional[Callable[[], float]] = None, storage: str = "f32",
                 storages: Optional[Sequence[str]] = None,
                 pool_shares: Optional[Sequence[float]] = None):
        """storage: the single lane's field storage (every request goes there).
        storages: serve several storages, one lane each, requests routed by
        their own storage; pool_shares splits pool_bytes, max_bricks and
        max_sims between them (equal shares by default)."""
        names = list(storages) if storages else [storage]
        shares = list(pool_shares) if pool_shares else [1.0 / len(names)] * len(names)
        assert len(shares) == len(names) and abs(sum(shares) - 1.0) < 1e-9
        self.lanes = {n: Lane(n, int(pool_bytes * f), max(32, int(max_bricks * f)),
                              max(1, int(round(max_sims * f))), device)
                      for n, f in zip(names, shares)}
        self.routed = storages is not None and len(names) > 1
        self.steps_per_tick = int(steps_per_tick)
        self.keep_fields = keep_fields
        self._clock = clock or time.perf_counter
        self._t0 = None
        self.results: List[Result] = []
        self.updates = 0
        self.ticks = 0
        self._virtual = False
        self._scale = 1.0

    # single-lane views kept for callers that use one storage
    @property
    def batch(self):
        return next(iter(self.lanes.values())).batch

    @property
    def n_slots(self):
        return sum(l.n_slots for l in self.lanes.values())

    @property
    def reserved_boxes(self):
        return sum(l.reserved_boxes for l in self.lanes.values())

    @property
    def reserved_bricks(self):
        return sum(l.reserved_bricks for l in self.lanes.values())

    @property
    def running(self):
        out = {}
        for l in self.lanes.values():
            out.update(l.running)
        return out

    def now(self) -> float:
        """Seconds since the start of run(), or ticks in virtual mode."""
        if self._virtual:
            return float(self.ticks)
        return self._clock() - self._t0

    @staticmethod
    def bricks_of(wl) -> int:
        nz, ny, nx = wl.shape
        bx, by, bz = wl.brick
        return -(-nx // bx) * -(-ny // by) * -(-nz // bz)

    def lane_of(self, req) -> Lane:
        if not self.routed:
            return next(iter(self.lanes.values()))
        st = getattr(req, "storage", "f32")
        if st not in self.lanes:
            raise ValueError(f"request {req.rid}: no lane serves storage {st!r}")
        return self.lanes[st]

    def fits(self, wl, lane: Optional[Lane] = None) -> bool:
        return (lane or next(iter(self.lanes.values()))).fits(wl)

    def admit(self, req, lane: Lane) -> None:
        wl = req.workload
        sim = lane.batch.add(wl, n_steps=wl.steps)
        nb = self.bricks_of(wl)
        lane.reserved_boxes += nb
        lane.reserved_bricks += (nb + 31) // 32 * 32
        lane.running[req.rid] = (req, sim, self.now(), nb)

    def collect(self, lane: Lane) -> None:
        for rid in list(lane.running):
            req, sim, t_adm, nb = lane.running[rid]
            if not sim.done():
                continue
            wl = req.workload
            nz, ny, nx = wl.shape
            plane = sim.read_field(0, origin=(0, 0, nz // 2), size=(nx, ny, 1))[0]
            field = sim.read_field(0) if self.keep_fields else None
            upd = sim.updates
            active = sim.active_count()[0]
            lane.batch.remove(sim)
            lane.reserved_boxes -= nb
            lane.reserved_bricks -= (nb + 31) // 32 * 32
            self.updates += upd
            self.results.append(Result(rid, req.arrival * self._scale, t_adm, self.now(), wl.steps, upd,
                                       active, plane, field, lane.storage))
            del lane.running[rid]

    def run(self, requests, time_scale: float = 1.0, virtual: bool = False) -> List[Result]:
        """Serve requests (sorted by arrival, seconds x time_scale).  virtual=True
        admits by tick count instead of wall-clock time (arrival = tick index)."""
        for r in sorted(requests, key=lambda r: r.arrival):
            lane = self.lane_of(r)
            if not lane.fits_empty(r.workload):
                raise RuntimeError(f"request {r.rid} can never fit this server")
            lane.queue.append(r)
        self._t0 = self._clock()
        self._virtual = bool(virtual)
        self._scale = float(time_scale)
        lanes = list(self.lanes.values())
        while any(l.queue or l.running for l in lanes):
            t = self.now()
            # admit everything that has arrived and fits, in arrival order per lane
            for l in lanes:
                while l.queue and l.queue[0].arrival * time_scale <= t and l.fits(l.queue[0].workload):
                    self.admit(l.queue.popleft(), l)
            busy = [l for l in lanes if l.running]
            if busy:
                for l in busy:
                    l.batch.step_async(self.steps_per_tick)
                for l in busy:
                    l.batch.sync()
                self.ticks += 1
                for l in busy:
                    self.collect(l)
            else:
                nxt = min(l.queue[0].arrival for l in lanes if l.queue) * time_scale
                if virtual:
                    self.ticks = max(self.ticks + 1, int(np.ceil(nxt)))
                else:
                    wait = nxt - self.now()
                    if wait > 0:
                        time.sleep(min(wait, 0.05))
        return self.results

    def close(self):
        for l in self.lanes.values():
            l.batch.close()


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
