"""Continuous-batching request loop over one batch of simulations.

Requests (workloads.Request: a simulation and its arrival time) are admitted
into one running batch as soon as they have arrived and the batch has room
-- free boxes in the pool for the request's whole brick count (so the pool
can never run out mid-run), brick-table space and a simulation slot.  The
batch steps every admitted simulation together, a tick of `steps_per_tick`
launches at a time; a simulation stops stepping when it has done its steps,
its result is read and it is removed, which frees its boxes and brick range
for waiting requests.  Everything runs through the C ABI (tcm_batch_*).

Result of a request: the final phi^n on the plane z = nz // 2, its active
(boxed) brick count and node updates; time to result = completion time -
arrival time.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Callable, Dict, List, Optional

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

    @property
    def time_to_result(self) -> float:
        return self.done - self.arrival


class Server:
    def __init__(self, pool_bytes: int, max_bricks: int, max_sims: int = 256,
                 steps_per_tick: int = 8, device: int = 0, keep_fields: bool = False,
                 clock: Optional[Callable[[], float]] = None):
        self.batch = tcm.Batch(pool_bytes=pool_bytes, max_bricks=max_bricks, max_sims=max_sims,
                               device=device)
        self.steps_per_tick = int(steps_per_tick)
        self.keep_fields = keep_fields
        self.max_sims = max_sims
        self.max_bricks = max_bricks
        self.n_slots = self.batch.info()[0]
        self._clock = clock or time.perf_counter
        self._t0 = None
        self.reserved_boxes = 0
        self.reserved_bricks = 0
        self.running: Dict[int, tuple] = {}
        self.results: List[Result] = []
        self.updates = 0
        self.ticks = 0
        self._virtual = False
        self._scale = 1.0

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

    def fits(self, wl) -> bool:
        nb = self.bricks_of(wl)
        return (len(self.running) < self.max_sims and self.reserved_boxes + nb <= self.n_slots
                and self.reserved_bricks + (nb + 31) // 32 * 32 <= self.max_bricks)

    def admit(self, req) -> None:
        wl = req.workload
        sim = self.batch.add(wl, n_steps=wl.steps)
        nb = self.bricks_of(wl)
        self.reserved_boxes += nb
        self.reserved_bricks += (nb + 31) // 32 * 32
        self.running[req.rid] = (req, sim, self.now(), nb)

    def collect(self) -> None:
        for rid in list(self.running):
            req, sim, t_adm, nb = self.running[rid]
            if not sim.done():
                continue
            wl = req.workload
            nz, ny, nx = wl.shape
            plane = sim.read_field(0, origin=(0, 0, nz // 2), size=(nx, ny, 1))[0]
            field = sim.read_field(0) if self.keep_fields else None
            upd = sim.updates
            active = sim.active_count()[0]
            self.batch.remove(sim)
            self.reserved_boxes -= nb
            self.reserved_bricks -= (nb + 31) // 32 * 32
            self.updates += upd
            self.results.append(Result(rid, req.arrival * self._scale, t_adm, self.now(), wl.steps, upd,
                                       active, plane, field))
            del self.running[rid]

    def run(self, requests, time_scale: float = 1.0, virtual: bool = False) -> List[Result]:
        """Serve requests (sorted by arrival, seconds x time_scale).  virtual=True
        admits by tick count instead of wall-clock time (arrival = tick index)."""
        queue = collections.deque(sorted(requests, key=lambda r: r.arrival))
        self._t0 = self._clock()
        self._virtual = bool(virtual)
        self._scale = float(time_scale)
        while queue or self.running:
            t = self.now()
            # admit everything that has arrived and fits, in arrival order
            while queue and queue[0].arrival * time_scale <= t and self.fits(queue[0].workload):
                self.admit(queue.popleft())
            if self.running:
                self.batch.step(self.steps_per_tick)
                self.ticks += 1
                self.collect()
            elif queue:
                if virtual:
                    self.ticks = max(self.ticks + 1, int(np.ceil(queue[0].arrival * time_scale)))
                else:
                    wait = queue[0].arrival * time_scale - self.now()
                    if wait > 0:
                        time.sleep(min(wait, 0.05))
                    if not self.fits(queue[0].workload):
                        raise RuntimeError(f"request {queue[0].rid} can never fit this server")
        return self.results

    def close(self):
        self.batch.close()


def summarize(results: List[Result], wall_s: float) -> dict:
    ttr = np.array([r.time_to_result for r in results]) if results else np.zeros(1)
    upd = sum(r.cell_updates for r in results)
    return {"requests": len(results), "p50_s": float(np.percentile(ttr, 50)),
            "p99_s": float(np.percentile(ttr, 99)), "cell_updates": int(upd),
            "cell_updates_per_s": upd / wall_s if wall_s > 0 else 0.0, "wall_s": wall_s}
