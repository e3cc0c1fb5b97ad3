"""Autotuner: choose the brick shape (and, if allowed, the update schedule)
for a workload by timing it.

Each candidate runs the workload through the C ABI: the steps before the
probe window untimed, then the window timed with CUDA events on the
library's stream.  The choice minimises the device time of the window (the
time to solution of those steps; node-update counts differ between shapes
because the cells differ).  Candidates:

  brick shapes     4x4x4, 8x8x8, 16x8x8 (one build of the library each)
  schedules        update every step with face neighbours (always); with
                   allow_schedule, also the Eq. 5 interval with the 26
                   neighbour set (at threshold 0 both equal the dense grid;
                   above it the active sets differ slightly)
  L2 prefetch      on (always); with allow_prefetch, the fastest of the
                   above is timed once more with it off (same results)

Results are cached per (workload name, shape, window, candidates) in the
process, and the chosen configuration can be applied with `apply`.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Sequence, Tuple

from . import tcm

BRICKS: Tuple[Tuple[int, int, int], ...] = ((4, 4, 4), (8, 8, 8), (16, 8, 8))
_CACHE: Dict[tuple, dict] = {}


@dataclasses.dataclass
class Candidate:
    brick: Tuple[int, int, int]
    interval: int = 1
    neighbours: int = 6
    prefetch: bool = True

    def label(self) -> str:
        b = "x".join(map(str, self.brick))
        b = b if (self.interval, self.neighbours) == (1, 6) else f"{b}/eq5-26"
        return b if self.prefetch else f"{b}/no-prefetch"


def candidates(allow_schedule: bool = False, bricks: Sequence = BRICKS) -> List[Candidate]:
    out = [Candidate(tuple(b)) for b in bricks]
    if allow_schedule:
        out += [Candidate(tuple(b), 0, 26) for b in bricks]
    return out


def apply(wl, c: Candidate):
    """The workload with the candidate's brick shape, schedule and prefetch."""
    return dataclasses.replace(wl, brick=tuple(c.brick), interval=c.interval, neighbours=c.neighbours,
                               prefetch=c.prefetch)


def _pool_bytes(wl, brick) -> Optional[int]:
    if wl.pool_bytes is None:
        return None
    # the same memory budget, whatever the box size
    return wl.pool_bytes


def measure(wl, c: Candidate, start: int, count: int, device: int = 0, storage="f32") -> dict:
    import torch
    w = apply(wl, c)
    # direct launches: a graph captured inside the timed window would add its
    # host-side capture time to the window
    s = tcm.Sim.from_workload(w, device=device, pool_bytes=_pool_bytes(w, c.brick), storage=storage,
                              graphs=False)
    try:
        s.step(start)
        u0 = s.updates
        torch.cuda.synchronize(device)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        s.step_async(count)
        e1.record()
        s.sync()
        ms = e0.elapsed_time(e1)
        upd = s.updates - u0
    finally:
        s.close()
    return {"config": c.label(), "brick": list(c.brick), "schedule": [c.interval, c.neighbours],
            "prefetch": c.prefetch, "window_ms": ms, "cell_updates": upd, "updates_per_s": upd / (ms / 1e3) if ms > 0 else 0.0}


def autotune(wl, start: Optional[int] = None, count: Optional[int] = None, allow_schedule: bool = False,
             device: int = 0, storage="f32", bricks: Sequence = BRICKS, allow_prefetch: bool = False) -> dict:
    """Time every candidate on steps [start, start+count) of the workload and
    return {"best": Candidate, "table": [...]} (fastest window first)."""
    steps = max(int(wl.steps), 1)
    if count is None:
        count = max(1, min(200, steps // 5))
    if start is None:
        start = max(0, min(steps - count, (steps * 2) // 5))
    key = (wl.name, tuple(wl.shape), start, count, allow_schedule, storage, tuple(map(tuple, bricks)),
           allow_prefetch)
    if key in _CACHE:
        return _CACHE[key]
    table = []
    for c in candidates(allow_schedule, bricks):
        r = measure(wl, c, start, count, device, storage)
        r["candidate"] = c
        table.append(r)
    table.sort(key=lambda r: r["window_ms"])
    if allow_prefetch:
        c = dataclasses.replace(table[0]["candidate"], prefetch=False)
        r = measure(wl, c, start, count, device, storage)
        r["candidate"] = c
        table.append(r)
        table.sort(key=lambda r: r["window_ms"])
    out = {"best": table[0]["candidate"], "window": [start, start + count],
           "table": [{k: v for k, v in r.items() if k != "candidate"} for r in table]}
    _CACHE[key] = out
    return out
