"""Benchmark of the Triggered Cells Method hot path on one GB300.

A step is one time step of the whole hot path (Eq. 3 on the active bricks,
source insertion, Eq. 6 decay, maxima, trigger/retire/box, active-list
compaction) = one launch of the persistent step kernel, on the 512^3 layered,
perturbed medium (relative threshold 1e-6, 20-step decay, 1500 steps).
By default the timed region is the whole run after W warm-up steps (steps
W..1500); with a smaller K the simulation is first advanced untimed so that
the K timed steps end at step 1500.  Inputs stay resident in HBM (they are
far larger than L2).

Metric: active-cell updates per second (plus HBM GB/s against the measured
copy roofline, TCM vs dense time to solution, per-step p50/p99).
`--impl reference` times the CPU oracle on the host cores instead.

Run: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

TOTAL_STEPS = 1500
BYTES_PER_UPDATE = 16          # read phi^n, phi^{n-1}, k; write phi^{n+1} (FP32, per-node k)
BYTES_PER_UPDATE_16 = 12       # 16-bit velocity form: read phi^n, v^n (2 B), k (4 B); write phi, v
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "k_step_layered512_traffic.txt")


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


class ClockSampler:
    """SM clock and clock-event reasons during the timed region.

    NVML queries (read-only) from a thread every ~1 ms, so even a region of a
    few milliseconds gets samples; nvidia-smi every 50 ms when NVML cannot be
    loaded.  The region starts once the first sample is in."""

    # clock-event reason bits of NVML (nvml.h)
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, pci=None):
        self.index = index
        self.pci = pci
        self.proc = None
        self.samples = []          # (sm_mhz, sm_max_mhz, reasons set)
        self.first = 0
        self.interval_ms = 1.0
        self._stop = threading.Event()
        self._nvml = None

    def _nvml_open(self):
        import ctypes as C
        lib = None
        for name in ("libnvidia-ml.so.1", "libnvidia-ml.so"):
            try:
                lib = C.CDLL(name)
                break
            except OSError:
                continue
        if lib is None or lib.nvmlInit_v2() != 0:
            return None
        h = C.c_void_p()
        ok = False
        if self.pci:
            ok = lib.nvmlDeviceGetHandleByPciBusId_v2(self.pci.encode(), C.byref(h)) == 0
        if not ok:
            ok = lib.nvmlDeviceGetHandleByIndex_v2(C.c_uint(self.index), C.byref(h)) == 0
        if not ok:
            return None
        smax = C.c_uint(0)
        lib.nvmlDeviceGetMaxClockInfo(h, 1, C.byref(smax))
        reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        return lib, h, float(smax.value), reasons_fn

    def _poll_nvml(self):
        import ctypes as C
        lib, h, smax, reasons_fn = self._nvml
        clk, rs = C.c_uint(0), C.c_ulonglong(0)
        while not self._stop.is_set():
            if lib.nvmlDeviceGetClockInfo(h, 1, C.byref(clk)) == 0 and reasons_fn(h, C.byref(rs)) == 0:
                self.samples.append((float(clk.value), smax,
                                     {n for b, n in self.REASONS.items() if rs.value & b}))
            time.sleep(self.interval_ms / 1e3)

    def _read_smi(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.strip().split(",")]
            if len(parts) < 8:
                continue
            try:
                sm, smax = float(parts[0]), float(parts[1])
            except ValueError:
                continue
            self.samples.append((sm, smax, {n for n, v in zip(names, parts[4:8]) if v.lower() == "active"}))

    def __enter__(self):
        try:
            self._nvml = self._nvml_open()
        except Exception:
            self._nvml = None
        try:
            if self._nvml is not None:
                self.t = threading.Thread(target=self._poll_nvml, daemon=True)
            else:
                self.interval_ms = 50.0
                self.proc = subprocess.Popen(
                    ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                     "--format=csv,noheader,nounits", "-lms", "50"],
                    stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
                self.t = threading.Thread(target=self._read_smi, daemon=True)
            self.t.start()
            t0 = time.perf_counter()
            while not self.samples and time.perf_counter() - t0 < 3.0:
                time.sleep(0.001)
            self.first = len(self.samples)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.last = len(self.samples)
        self._stop.set()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        """Samples taken during the region (the one just before it when the
        region was too short for any)."""
        during = self.samples[self.first:getattr(self, "last", len(self.samples))]
        rows = during if during else self.samples[self.first - 1:self.first]
        sm = [r[0] for r in rows]
        reasons = set()
        for r in rows:
            reasons |= r[2]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": rows[-1][1] if rows else None,
                "reasons": sorted(reasons), "samples": len(sm), "interval_ms": self.interval_ms,
                "source": "nvml" if self._nvml is not None else "nvidia-smi",
                "during_region": bool(during)}


def kernel_source_hash() -> str:
    """Hash of the kernel sources' code: comments and blank space are left
    out, so a change of wording does not mark the recorded counters stale."""
    import re
    h = hashlib.sha256()
    for f in ("tcm_kernels.cu", "tcm_internal.cuh"):
        src = open(os.path.join(ROOT, "paper_1702_00216_gb300", "csrc", f)).read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(updates_per_launch: float):
    """DRAM bytes per launch from the committed ncu summary, scaled by units, or None
    when the kernel changed since the counters were taken."""
    try:
        d = dict(ln.split(":", 1) for ln in open(PROFILE_TRAFFIC)
                 if ":" in ln and not ln.startswith("#"))
        d = {k.strip(): v.strip() for k, v in d.items()}
    except Exception:
        return None
    if d.get("kernel_hash") != kernel_source_hash():
        return None
    return float(d["dram_bytes_per_update"]) * updates_per_launch


def job_totals(torch, total_ms: float, updates: int, world: int, dev):
    """Whole-job figures over the replicas: the slowest rank's time (max) and
    the node updates of all ranks (sum); the identity on one rank."""
    if world <= 1:
        return total_ms, float(updates)
    tt = torch.tensor([total_ms], device=dev, dtype=torch.float64)
    torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
    uu = torch.tensor([float(updates)], device=dev, dtype=torch.float64)
    torch.distributed.all_reduce(uu)
    return float(tt.item()), float(uu.item())


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


# ---------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import torch
    import __graft_entry__ as ge
    from paper_1702_00216_gb300 import tcm, workloads as W

    torch.cuda.set_device(local_rank)
    if rank == 0 or not os.path.exists(os.path.join(ROOT, "paper_1702_00216_gb300", "libtcm.so")):
        ge.build()
    if world > 1:
        torch.distributed.barrier()
        ge.build()
    dev = torch.device("cuda", local_rank)
    K, Wm = args.steps, args.warmup
    wl = W.layered(n=args.grid, steps=TOTAL_STEPS)
    if args.lpf:
        # the Eq. 7 shut-down instead of the Eq. 6 decay (pass, stop of Nyquist)
        import dataclasses
        wl = dataclasses.replace(wl, lpf=tuple(float(v) for v in args.lpf.split(",")))
    # enough boxes for every brick of the grid (the layered wave reaches most of it)
    storage = tcm.STORAGES[args.storage]
    bpu = BYTES_PER_UPDATE if args.storage == "f32" else BYTES_PER_UPDATE_16
    pool_bytes = (args.grid // 8) ** 3 * tcm.tcm_slot_bytes(wl.brick, storage)
    pool = torch.empty(pool_bytes, dtype=torch.uint8, device=dev)
    if args.save_state:
        # profiling aid: the run's state at a late step, to resume it with few
        # launches before the ones a profiler captures
        sim = tcm.Sim.from_workload(wl, pool_tensor=pool, device=local_rank, storage=storage,
                                    graphs=not args.no_graphs)
        sim.step(args.state_step)
        np.savez(args.save_state, now=sim.read_field(0), prev=sim.read_field(1), step=args.state_step)
        print(json.dumps({"saved_state": args.save_state, "step": args.state_step,
                          "active_bricks": sim.active_count()[0]}), flush=True)
        sim.close()
        return
    if args.load_state:
        # resume from a saved state (its sources have ended): phi^n, phi^{n-1}
        # become the initial fields; K timed steps after W warm-up steps
        import dataclasses
        st = np.load(args.load_state)
        wl = dataclasses.replace(wl, sources=[], name=f"{wl.name} from step {int(st['step'])}")
        sim = tcm.Sim.from_workload(wl, pool_tensor=pool, device=local_rank, storage=storage,
                                    graphs=not args.no_graphs)
        sim.set_field(st["now"], st["prev"])
        del st
        t0 = 0
    else:
        sim = tcm.Sim.from_workload(wl, pool_tensor=pool, device=local_rank, storage=storage,
                                    graphs=not args.no_graphs)
        t0 = max(0, TOTAL_STEPS - K - Wm)
    if args.trace:
        # one step at a time, recording the node updates of every launch
        with open(args.trace, "w") as f:
            last = 0
            for n in range(t0 + Wm):
                sim.step(1)
                u = sim.updates
                f.write(json.dumps({"launch": n, "step": n, "cell_updates": u - last}) + "\n")
                last = u
    else:
        sim.step(t0)
        sim.step(Wm)
    torch.cuda.synchronize()
    u0 = sim.updates
    l0 = sim.launches
    ph0 = sim.phase_ns()
    # The timed region: the K steps in one call of the public API (one
    # launch per step, replayed from a CUDA graph captured inside the call).
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    props = torch.cuda.get_device_properties(local_rank)
    pci = f"{props.pci_domain_id:08x}:{props.pci_bus_id:02x}:{props.pci_device_id:02x}.0"
    with ClockSampler(local_rank, pci) as clk:
        ev[0].record()
        sim.step_async(K)
        ev[1].record()
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    sim.sync()
    total_ms = ev[0].elapsed_time(ev[1])
    updates = sim.updates - u0
    launches = sim.launches - l0
    ph = [b - a for a, b in zip(ph0, sim.phase_ns())]
    active_end = sim.active_count()

    t_max, upd_all = job_totals(torch, total_ms, updates, world, dev)
    value = upd_all / (t_max / 1e3)

    peaks, peak_kind = measured_peaks()
    achieved = updates * bpu / (total_ms / 1e3) / 1e9
    # the committed counters are those of the binary32 kernel
    traffic = profiled_traffic(updates / max(launches, 1)) if args.storage == "f32" else None
    sim.close()
    marginal, step_ms = None, None
    if not args.quick and world == 1 and not args.load_state:
        # over the whole run (steps 5..1500), whatever the timed window: the
        # fit needs steps of very different active-set sizes
        marginal, step_ms = per_cell_fit(torch, tcm, W, wl, pool, local_rank, 5, TOTAL_STEPS - 5,
                                         peaks["hbm_gbs"], storage, bpu)
    del pool
    torch.cuda.empty_cache()

    extra = {}
    if rank == 0 and not args.quick:
        extra = time_to_solution(torch, tcm, W, wl, dev, local_rank)
    e2e = end_to_end(torch, tcm, W, wl, local_rank) if not args.quick else None
    if e2e is not None and world > 1:
        # whole job over the replicas: every rank ran the same end-to-end call
        t_e, u_e = job_totals(torch, e2e["seconds"] * 1e3, e2e["cell_updates"], world, dev)
        e2e.update({"value": u_e / (t_e / 1e3), "seconds": t_e / 1e3, "cell_updates": u_e,
                    "h2d_bytes_per_step": e2e["h2d_bytes_per_step"] * world,
                    "d2h_bytes_per_step": e2e["d2h_bytes_per_step"] * world, "replicas": world})
    cpu, o512 = cpu_baseline(W, args, wl=wl) if (rank == 0 and world == 1 and not args.quick) else (None, None)
    otimes = None
    if cpu is not None and args.oracle_timings:
        otimes = oracle_timings(torch, tcm, W, args, local_rank, cpu, o512,
                                extra.get("time_to_solution") if extra else None)
    if o512 is not None:
        o512.close()
        del o512
    serving = serving_leg(torch, W, args, local_rank) if (rank == 0 and not args.quick and args.serving > 0) else None
    precision = precision_leg(torch, tcm, W, dev, local_rank) if (rank == 0 and not args.quick) else None
    virtual = virtual_leg(torch, tcm, W, local_rank) if (rank == 0 and not args.quick and args.virtual) else None
    tuning = tuning_leg(torch, tcm, W, wl, dev, local_rank) if (rank == 0 and not args.quick) else None

    if rank != 0:
        return
    line = {
        "metric": "active-cell updates/s",
        "value": value,
        "unit": "cell-updates/s",
        "n_gpus": world,
        "steps": K,
        "warmup": Wm,
        "ms_per_step": t_max / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": wl.name, "grid": list(wl.shape[::-1]), "brick": list(wl.brick),
                   "threshold": "relative 1e-6", "decay": "alpha 0.8, 20 steps",
                   "storage": args.storage,
                   "shutdown": f"Eq. 7 LPF {args.lpf}" if args.lpf else "Eq. 6 decay",
                   "timed_steps": [TOTAL_STEPS - K, TOTAL_STEPS],
                   "l2": "inputs larger than L2 (fields + per-node k > 1.5 GB)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                     "peak_source": peak_kind, "frac_of_nominal_8tbs": achieved / 8000.0,
                     "algorithmic_bytes_per_update": bpu,
                     "kernel": "k_step (persistent, one launch per step)"},
        "step_ms": None if step_ms is None else {
            "p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
            "min": float(min(step_ms)), "max": float(max(step_ms)),
            "how": "untimed replay of steps 5..1500, one call and one event per step"},
        "per_active_cell": marginal,
        "phase_ms": {"time_stepping": ph[0] / 1e6, "update_active": ph[1] / 1e6,
                     "compaction": ph[2] / 1e6},
        "active_bricks_end": active_end[0],
        "active_cells_end": active_end[1],
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    line.update(extra)
    if serving is not None:
        line["serving"] = serving
    if precision is not None:
        line["precision"] = precision
    if virtual is not None:
        line["virtual_4096"] = virtual
    if tuning is not None:
        line["autotune"] = tuning
    if otimes is not None:
        line["oracle_time_to_solution"] = otimes
    print(json.dumps(line), flush=True)


def per_cell_fit(torch, tcm, W, wl, pool, local_rank, first, K, hbm_peak, storage=0, bpu=16):
    """Split the time of steps first..first+K into a fixed cost per step and a
    cost per active cell.  Two untimed replays of the same (deterministic)
    run: one call and one CUDA event per step (the step times; each includes
    its call's launch gap, so the fixed cost is an upper bound), and one
    synchronous step at a time (the node updates of every step).  Then
    t_step = fixed + updates / rate by least squares, and the whole-step rate
    of the last 200 steps (the largest active sets).  Returns the fit and the
    per-step times in ms."""
    s = tcm.Sim.from_workload(wl, pool_tensor=pool, device=local_rank, storage=storage)
    s.step(first)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    ev[0].record()
    for i in range(K):
        s.step_async(1)
        ev[i + 1].record()
    torch.cuda.synchronize()
    s.sync()
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(K)]
    s.close()
    s = tcm.Sim.from_workload(wl, pool_tensor=pool, device=local_rank, storage=storage)
    s.step(first)
    upd = []
    last = s.updates
    for _ in range(K):
        s.step(1)
        u = s.updates
        upd.append(u - last)
        last = u
    s.close()
    u = np.asarray(upd, dtype=np.float64)
    t = np.asarray(step_ms, dtype=np.float64) / 1e3
    A = np.vstack([np.ones_like(u), u]).T
    (fixed, per_update), *_ = np.linalg.lstsq(A, t, rcond=None)
    rate = bpu / per_update / 1e9
    late = slice(max(0, len(t) - 200), len(t))
    late_gbs = u[late].sum() * bpu / t[late].sum() / 1e9
    return {"fixed_us_per_step": fixed * 1e6, "marginal_gbs": rate, "marginal_frac": rate / hbm_peak,
            "fixed_share_of_run": fixed * len(t) / t.sum(),
            "last_200_steps_gbs": late_gbs, "last_200_steps_frac": late_gbs / hbm_peak,
            "last_200_steps_mean_active_cells": float(u[late].mean()),
            "how": "least squares t_step = fixed + updates/rate over an untimed replay of the timed "
                   "steps (one call and event per step); updates per step from a second replay"}, step_ms


def virtual_leg(torch, tcm, W, local_rank):
    """The virtual 4096^3 domain (a dense grid would need 4096^3 x 3 x 4 B =
    824 GB): sphere inclusion, 3-cycle Ricker burst, relative threshold 1e-6,
    20-step decay, pool capped at 120 GiB, 2500 steps from create to the last
    step, device time; the steps once more with the L2 prefetch off."""
    import dataclasses
    wl = W.virtual()
    torch.cuda.synchronize()
    t = time.perf_counter()
    s = tcm.Sim.from_workload(wl, device=local_rank)
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    s.step_async(wl.steps)
    e1.record()
    s.sync()
    ms = e0.elapsed_time(e1)
    boxes, free = s.pool_info()
    out = {"workload": f"{wl.name}, {wl.steps} steps", "create_s": t_create, "steps_s": ms / 1e3,
           "cell_updates": s.updates, "updates_per_s": s.updates / (ms / 1e3),
           "active_bricks_end": s.active_count()[0], "pool_boxes": boxes, "pool_boxes_free_end": free,
           "dense_bytes_needed": 4096 ** 3 * 12, "pool_bytes": wl.pool_bytes}
    s.close()
    s = tcm.Sim.from_workload(dataclasses.replace(wl, prefetch=False), device=local_rank)
    e0.record()
    s.step_async(wl.steps)
    e1.record()
    s.sync()
    ms = e0.elapsed_time(e1)
    out["no_prefetch"] = {"steps_s": ms / 1e3, "updates_per_s": s.updates / (ms / 1e3)}
    s.close()
    torch.cuda.empty_cache()
    return out


def tuning_leg(torch, tcm, W, wl, dev, local_rank):
    """The autotuner on the benchmark workload (brick shapes, CTA blocking of
    the 8x8x8 build, update schedules, then the fastest with the L2 prefetch
    off; steps 600..800 timed; each candidate's field at step 800 compared
    with the dense grid's, the choice the fastest within 1e-5 max|phi|), then
    the full create-to-result run with its choice, compared with the dense
    result."""
    from paper_1702_00216_gb300 import autotune
    r = autotune.autotune(wl, start=600, count=200, allow_schedule=True, device=local_rank, allow_prefetch=True,
                          allow_blocking=True, accuracy=True, tolerance=1e-5)
    best = autotune.apply(wl, r["best"])
    out = {"window": r["window"], "table": r["table"], "best": r["best"].label(), "choice": r["choice"]}
    runs = {}
    for name, w, dense in (("dense", wl, True), ("tuned", best, False)):
        torch.cuda.synchronize()
        t = time.perf_counter()
        s = tcm.Sim.from_workload(w, dense=dense, device=local_rank)
        s.step(TOTAL_STEPS)
        buf = torch.empty(w.shape, dtype=torch.float32, device=dev)
        tcm.tcm_read_field_device(s.handle, 0, (0, 0, 0), w.shape[::-1], buf.data_ptr())
        torch.cuda.synchronize()
        runs[name] = (time.perf_counter() - t, s.updates, buf)
        s.close()
    out["tuned_s"] = runs["tuned"][0]
    out["tuned_cell_updates"] = runs["tuned"][1]
    out["dense_s"] = runs["dense"][0]
    out["speedup_vs_dense"] = runs["dense"][0] / runs["tuned"][0]
    out["max_abs_diff_vs_dense"] = float((runs["tuned"][2] - runs["dense"][2]).abs().max().item())
    del runs
    torch.cuda.empty_cache()
    return out


def time_to_solution(torch, tcm, W, wl, dev, local_rank):
    """Full 1500-step runs from create to the final field on the device: TCM
    (update procedure every step, face neighbours, Eq. 6 decay), TCM on the
    Eq. 5 schedule (update every 8 steps, 26 neighbours), TCM with the Eq. 7
    shut-down (LPF pass 0.25, stop 0.5 of Nyquist), and the same kernel over
    every brick (dense, no update procedure); each run twice, the faster
    reported."""
    import dataclasses
    runs = [("dense", wl, True), ("tcm", wl, False),
            ("tcm_eq5_26", dataclasses.replace(wl, interval=0, neighbours=26), False),
            ("tcm_lpf", dataclasses.replace(wl, lpf=(0.25, 0.5)), False)]
    out = {}
    ref = None
    for name, w, dense in runs:
        dts = []
        for rep in range(2):   # best of two (the first pays one-off allocation costs)
            if rep:
                del buf
                s.close()
            torch.cuda.synchronize()
            t = time.perf_counter()
            s = tcm.Sim.from_workload(w, dense=dense, device=local_rank, pool_bytes=None)
            s.step(TOTAL_STEPS)
            buf = torch.empty(w.shape, dtype=torch.float32, device=dev)
            tcm.tcm_read_field_device(s.handle, 0, (0, 0, 0), w.shape[::-1], buf.data_ptr())
            torch.cuda.synchronize()
            dts.append(time.perf_counter() - t)
        dt = min(dts)
        r = {"seconds": dt, "seconds_each": dts, "cell_updates": s.updates, "schedule": list(s.schedule())}
        if w.lpf is not None:
            # the Eq. 7 filter's roofline: binary32 multiply-adds of the
            # separable operator per filtered brick over the filter kernel's
            # device time, against the CUDA-core FP32 rate derived from unit
            # counts and clocks (152 SMs x 128 FMA lanes x 2 flops x 2.07 GHz)
            ns, nbr, fma = tcm.tcm_lpf_info(s.handle)
            flops = 2.0 * fma * nbr
            peak = 152 * 128 * 2 * 2.07e9 / 1e12
            r["k_lpf"] = {"ms": ns / 1e6, "bricks_filtered": nbr, "fp32_fma_per_brick": fma,
                          "fp32_tflops": flops / (ns * 1e-9) / 1e12 if ns else None,
                          "peak_tflops": peak, "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                          "frac": (flops / (ns * 1e-9) / 1e12) / peak if ns else None,
                          "share_of_run": (ns / 1e9) / dt}
        if ref is None:
            ref = buf
            r["max_abs_field"] = float(buf.abs().max().item())
        else:
            r["max_abs_diff_vs_dense"] = float((buf - ref).abs().max().item())
            del buf
        out[name] = r
        s.close()
    del ref
    torch.cuda.empty_cache()
    return {"time_to_solution": {
        "workload": f"{wl.name}, {TOTAL_STEPS} steps, create + steps + device readback",
        "tcm_s": out["tcm"]["seconds"], "dense_s": out["dense"]["seconds"],
        "speedup": out["dense"]["seconds"] / out["tcm"]["seconds"],
        "tcm_cell_updates": out["tcm"]["cell_updates"],
        "dense_cell_updates": out["dense"]["cell_updates"],
        "max_abs_diff_tcm_vs_dense": out["tcm"]["max_abs_diff_vs_dense"],
        "max_abs_field": out["dense"]["max_abs_field"],
        "eq5_interval_26_neighbours": out["tcm_eq5_26"],
        "eq7_lpf_shutdown": out["tcm_lpf"]}}


def precision_leg(torch, tcm, W, dev, local_rank):
    """Field storage FP32 / BF16 / FP16 on the 256^3 homogeneous medium with
    the 64^3 configuration's source (relative threshold 1e-6, 20-step decay),
    800 steps each: device time of the steps, node updates/s, HBM GB/s at the
    storage's algorithmic bytes per update, max and RMS error of phi^800
    against the FP32 run, and the drift of the leapfrog energy from step
    len(wavelet)+50 to step 800 (FP64 reduction on the device)."""
    from paper_1702_00216_gb300 import autotune
    wl = W.precision(256, 800)
    # brick shape and CTA blocking from the autotuner (steps 300..400, binary32)
    tuned = autotune.autotune(wl, start=300, count=100, device=local_rank, allow_blocking=True)
    wl = autotune.apply(wl, tuned["best"])
    n_src = len(wl.sources[0][3])
    out = {"workload": f"{wl.name}, 800 steps, relative threshold 1e-6, 20-step decay",
           "tuned": {"best": tuned["best"].label(), "window": tuned["window"],
                     "table": [{k: t[k] for k in ("config", "window_ms", "updates_per_s")} for t in tuned["table"]]}}
    ref = None
    for st in ("f32", "bf16", "f16"):
        s = tcm.Sim.from_workload(wl, device=local_rank, storage=st)
        s.step(1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        u0 = s.updates
        e0.record()
        s.step_async(n_src + 49)
        e1.record()
        s.sync()
        ms = e0.elapsed_time(e1)
        en_a = s.energy()
        u1 = s.updates
        e0.record()
        s.step_async(800 - n_src - 50)
        e1.record()
        s.sync()
        ms += e0.elapsed_time(e1)
        en_b = s.energy()
        upd = s.updates - u0
        buf = torch.empty(wl.shape, dtype=torch.float32, device=dev)
        tcm.tcm_read_field_device(s.handle, 0, (0, 0, 0), wl.shape[::-1], buf.data_ptr())
        torch.cuda.synchronize()
        # every brick has a scalar k (homogeneous medium): binary32 reads phi^n
        # and phi^{n-1} and writes phi^{n+1}; 16-bit reads phi and v (2 B
        # each) and writes both
        bpu = 12 if st == "f32" else 8
        r = {"updates_per_s": upd / (ms / 1e3), "ms": ms, "bytes_per_update": bpu,
             "hbm_gbs": upd * bpu / (ms / 1e3) / 1e9,
             "energy_drift": abs(en_b - en_a) / abs(en_a) if en_a else None}
        if ref is None:
            ref = buf
            gmax = float(ref.abs().max().item())
            grms = float(ref.double().pow(2).mean().sqrt().item())
        else:
            d = (buf - ref).double()
            r["max_rel_err_vs_f32"] = float(d.abs().max().item()) / gmax
            r["rms_rel_err_vs_f32"] = float(d.pow(2).mean().sqrt().item()) / grms
            del buf
        out[st] = r
        s.close()
    del ref
    torch.cuda.empty_cache()
    out["layered_512"] = storage_throughput(torch, tcm, W, local_rank)
    return out


def storage_throughput(torch, tcm, W, local_rank):
    """Each storage on the 512^3 layered workload as the headline measures it:
    steps 5..1500 in one call (CUDA events around it), node updates/s and HBM
    GB/s at the storage's algorithmic bytes per update, as a fraction of the
    measured copy bandwidth."""
    wl = W.layered(steps=TOTAL_STEPS)
    peaks, _ = measured_peaks()
    n_bricks = (wl.shape[0] // 8) * (wl.shape[1] // 8) * (wl.shape[2] // 8)
    out = {"workload": f"{wl.name}, steps 5..{TOTAL_STEPS} in one call"}
    for st in ("f32", "bf16", "f16"):
        code = tcm.STORAGES[st]
        s = tcm.Sim.from_workload(wl, device=local_rank, storage=st,
                                  pool_bytes=n_bricks * tcm.tcm_slot_bytes(wl.brick, code))
        s.step(5)
        torch.cuda.synchronize()
        u0 = s.updates
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        s.step_async(TOTAL_STEPS - 5)
        e1.record()
        s.sync()
        ms = e0.elapsed_time(e1)
        upd = s.updates - u0
        s.close()
        bpu = 16 if st == "f32" else 12
        gbs = upd * bpu / (ms / 1e3) / 1e9
        out[st] = {"updates_per_s": upd / (ms / 1e3), "ms": ms, "bytes_per_update": bpu, "hbm_gbs": gbs,
                   "frac_of_measured": gbs / peaks["hbm_gbs"]}
    torch.cuda.empty_cache()
    return out


def serving_leg(torch, W, args, local_rank):
    """Continuous batching on the serving stream (grid edge log-uniform
    64..512, 2-6 layers, Ricker at a random node, 200..3000 steps, relative
    threshold 1e-6, 20-step decay; FP32 and BF16 requests in one batch of
    mixed storage, admitted by active footprint into a 2 GiB pool).  First the
    capacity is calibrated: a burst of requests all arriving at once, served
    to completion (requests per second).  Then the next requests of the
    stream arrive as a Poisson process at 75 % of that capacity: p50/p99 time
    to result (arrival -> result read back) and aggregate node updates per
    second.  The burst is also served with admission by whole grids, for the
    concurrency that admission reaches in the same pool."""
    from paper_1702_00216_gb300 import serve
    n_cal, n_run = args.serving_calibrate, args.serving
    pool = 2 * 1024 ** 3

    def stream(rate):
        reqs = W.serving_stream(n_requests=n_cal + n_run, seed=216, rate_hz=rate)
        for r in reqs:
            r.workload.thr_mode, r.workload.tau = 1, 1e-6
            r.workload.decay_alpha, r.workload.decay_steps = 0.8, 20
        return reqs

    def serve_once(reqs, time_scale, admission, pool_bytes=pool):
        srv = serve.Server(pool_bytes=pool_bytes, max_bricks=24 * 1024 ** 2, max_sims=512, steps_per_tick=16,
                           device=local_rank, storages=("f32", "bf16"), admission=admission)
        torch.cuda.synchronize()
        t = time.perf_counter()
        res = srv.run(reqs, time_scale=time_scale)
        wall = time.perf_counter() - t
        stats = dict(srv.stats, ticks=srv.ticks, pool_boxes=srv.n_slots)
        srv.close()
        return res, wall, stats

    burst = stream(1.0)[:n_cal]
    res, wall, stats = serve_once(burst, 0.0, "footprint")
    capacity = len(res) / wall
    cal = dict(serve.summarize(res, wall), capacity_requests_per_s=capacity, **stats)
    _, wall_d, stats_d = serve_once(burst, 0.0, "dense")
    dense = {"wall_s": wall_d, "max_concurrent": stats_d["max_concurrent"],
             "max_grid_bricks_running": stats_d["max_grid_bricks_running"]}
    # the same burst in a 1 GiB pool (the smallest that holds a whole 512^3
    # grid), where the pool rather than the GPU limits how many run at once
    small = {}
    for adm in ("footprint", "dense"):
        _, wall_s, st_s = serve_once(burst, 0.0, adm, pool_bytes=1024 ** 3)
        small[adm] = {"wall_s": wall_s, "max_concurrent": st_s["max_concurrent"],
                      "max_grid_bricks_running": st_s["max_grid_bricks_running"], "pauses": st_s["pauses"],
                      "evictions": st_s["evictions"], "pool_boxes": st_s["pool_boxes"]}
    rate = 0.75 * capacity
    reqs = stream(rate)[n_cal:]
    t0 = reqs[0].arrival
    for r in reqs:
        r.arrival -= t0
    res, wall, stats = serve_once(reqs, 1.0, "footprint")
    out = serve.summarize(res, wall)
    out.update(stats)
    out.update({"stream": f"requests {n_cal}..{n_cal + n_run} of the serving stream (seed 216), Poisson "
                          f"arrivals at 75 % of the calibrated capacity ({rate:.2f}/s), FP32/BF16 mix in one "
                          f"batch of mixed storage, admission by active footprint, 2 GiB pool",
                "rate_hz": rate, "steps_per_tick": 16, "calibration": cal,
                "dense_admission_burst": dense, "burst_in_1gib_pool": small})
    torch.cuda.empty_cache()
    return out


def end_to_end(torch, tcm, W, wl, local_rank):
    """The same metric through the public API with host buffers: velocity model
    and wavelet from pinned host memory, 1500 steps, final field back to host.
    Run three times, the fastest reported (the first pays one-off costs)."""
    nz, ny, nx = wl.shape
    c_host = torch.empty(wl.shape, dtype=torch.float32, pin_memory=True)
    c_host.numpy()[...] = wl.media.c
    out_host = torch.empty(wl.shape, dtype=torch.float32, pin_memory=True)
    media = W.dense_media(c_host.numpy())
    dts = []
    for _ in range(3):
        torch.cuda.synchronize()
        t = time.perf_counter()
        s = tcm.Sim(wl.shape, media, wl.dx, wl.dt, threshold=wl.tau, brick=wl.brick,
                    thr_mode=wl.thr_mode, decay_alpha=wl.decay_alpha, decay_steps=wl.decay_steps,
                    pool_bytes=None, device=local_rank)
        for x, y, z, w in wl.sources:
            s.add_source(x, y, z, np.asarray(w, np.float32))
        s.step(TOTAL_STEPS)
        rc = tcm.lib().tcm_read_field(s.handle, 0, 0, 0, 0, nx, ny, nz,
                                      tcm.C.c_void_p(out_host.data_ptr()))
        if rc != 0:
            raise tcm.TCMError(rc, "tcm_read_field")
        dts.append(time.perf_counter() - t)
        upd = s.updates
        s.close()
    dt = min(dts)
    h2d = c_host.numel() * 4 + sum(len(w) * 4 for *_, w in wl.sources)
    d2h = out_host.numel() * 4
    return {"value": upd / dt, "unit": "cell-updates/s",
            "h2d_bytes_per_step": h2d / TOTAL_STEPS, "d2h_bytes_per_step": d2h / TOTAL_STEPS,
            "seconds": dt, "seconds_each": dts, "steps": TOTAL_STEPS, "cell_updates": upd,
            "what": "tcm_create from host velocity + tcm_add_source + tcm_step(1500) + "
                    "tcm_read_field of the whole grid to pinned host memory (best of three)"}


def cpu_baseline(W, args, budget_s: float = 45.0, wl=None):
    """The oracle (plain C, as it stands) on all host cores: the layered 512^3
    workload from step 0 to the end of the run (its time to solution), unless
    the time budget runs out first; then two more steps on one core and two
    on all cores from the final state (the largest active sets), whose rates
    give the single-core estimate.  Returns the line's cpu_baseline and the
    final oracle (for the dense-grid windows of the timing leg)."""
    import oracle
    threads = os.cpu_count() or 1
    used = oracle.set_threads(threads)
    if wl is None:
        wl = W.layered(steps=TOTAL_STEPS)
    t = time.perf_counter()
    o = oracle.OracleTCM(wl.shape, wl.media, wl.dx, wl.dt, brick=wl.brick, thr_mode=wl.thr_mode,
                         tau=wl.tau, decay_alpha=wl.decay_alpha, decay_steps=wl.decay_steps)
    for x, y, z, w in wl.sources:
        o.add_source(x, y, z, np.asarray(w, np.float32))
    t_create = time.perf_counter() - t
    t = time.perf_counter()
    steps = 0
    while time.perf_counter() - t < budget_s and steps < TOTAL_STEPS:
        o.step(10)
        steps += 10
    dt = time.perf_counter() - t
    upd = o.updates
    t1 = time.perf_counter()
    o.read_field(0)
    t_read = time.perf_counter() - t1
    rates = {}
    for name, th in (("all_cores", threads), ("one_core", 1)):
        oracle.set_threads(th)
        u0 = o.updates
        t2 = time.perf_counter()
        o.step(2)
        rates[name] = (o.updates - u0) / (time.perf_counter() - t2)
    oracle.set_threads(threads)
    out = {"value": upd / dt, "unit": "cell-updates/s", "cores": used, "kind": "oracle",
           "sample": f"{wl.name}: steps 0..{steps} of {TOTAL_STEPS} ({upd} cell updates, {dt:.1f} s, "
                     f"all cores)",
           "time_to_solution_s": t_create + dt + t_read if steps >= TOTAL_STEPS else None,
           "single_thread": {"value": rates["one_core"], "cores": 1,
                             "all_cores_same_window": rates["all_cores"],
                             "sample": f"steps {steps}..{steps + 2} on all cores, then "
                                       f"{steps + 2}..{steps + 4} on one"}}
    return out, o


def oracle_timings(torch, tcm, W, args, local_rank, cpu, o512, tts):
    """Time to solution of the oracle as it stands (create + steps + reading
    the final field) on one host core and on all of them, beside the GPU's
    (create + steps + device readback), for each workload: the 64^3 pulse
    (100 steps), the 512^3 layered run (1500 steps), the first 300 steps of
    the virtual 4096^3 domain and the 256^3 precision workload (800 steps).
    Runs that would take minutes on the host are estimated from the rate of a
    short window times the run's node updates, and say so."""
    import oracle
    threads = os.cpu_count() or 1

    def gpu_run(wl, steps, dense=False):
        best = None
        for _ in range(2):
            torch.cuda.synchronize()
            t = time.perf_counter()
            s = tcm.Sim.from_workload(wl, dense=dense, device=local_rank)
            s.step(steps)
            buf = torch.empty(wl.shape if wl.shape[0] * wl.shape[1] * wl.shape[2] <= 1 << 28 else (1,),
                              dtype=torch.float32, device=f"cuda:{local_rank}")
            if buf.numel() > 1:
                tcm.tcm_read_field_device(s.handle, 0, (0, 0, 0), wl.shape[::-1], buf.data_ptr())
            torch.cuda.synchronize()
            dt = time.perf_counter() - t
            upd = s.updates
            s.close()
            del buf
            best = dt if best is None else min(best, dt)
        return best, upd

    def tcm_oracle(wl, steps, th):
        oracle.set_threads(th)
        t = time.perf_counter()
        o = oracle.OracleTCM(wl.shape, wl.media, wl.dx, wl.dt, brick=wl.brick, thr_mode=wl.thr_mode,
                             tau=wl.tau, decay_alpha=wl.decay_alpha, decay_steps=wl.decay_steps)
        for x, y, z, w in wl.sources:
            o.add_source(x, y, z, np.asarray(w, np.float32))
        o.step(steps)
        if wl.shape[0] * wl.shape[1] * wl.shape[2] <= 1 << 28:
            o.read_field(0)
        dt = time.perf_counter() - t
        upd = o.updates
        o.close()
        oracle.set_threads(threads)
        return dt, upd

    def dense_window(wl, now, prev, steps, th, dtype=np.float32):
        oracle.set_threads(th)
        k = oracle.k_from_c(wl.media.c if wl.media.kind == "dense" else oracle.rules_c(wl.shape, wl.media),
                            wl.dt, wl.dx, dtype)
        t = time.perf_counter()
        oracle.dense_run(k, now.astype(dtype), prev.astype(dtype), steps)
        dt = time.perf_counter() - t
        oracle.set_threads(threads)
        return int(np.prod(wl.shape)) * steps / dt

    out = {"cores": threads}
    # 64^3 pulse, threshold 0: full runs
    wl = W.small()
    r = {"steps": wl.steps}
    for name, th in (("one_core", 1), ("all_cores", threads)):
        dt, upd = tcm_oracle(wl, wl.steps, th)
        r[f"oracle_tcm_{name}_s"] = dt
        oracle.set_threads(th)
        k = oracle.k_from_c(np.ones(wl.shape, np.float32), wl.dt, wl.dx, np.float32)
        z = np.zeros(wl.shape, np.float32)
        t = time.perf_counter()
        oracle.dense_run(k, z, z, wl.steps, [(x, y, zz, np.asarray(w, np.float32)) for x, y, zz, w in wl.sources])
        r[f"oracle_dense_{name}_s"] = time.perf_counter() - t
        oracle.set_threads(threads)
    r["gpu_tcm_s"], r["cell_updates"] = gpu_run(wl, wl.steps)
    r["gpu_dense_s"], _ = gpu_run(wl, wl.steps, dense=True)
    out["small_64"] = r
    # 512^3 layered run: the TCM oracle's full run on all cores is the
    # cpu_baseline; one core and the dense grid from windows
    upd = tts.get("tcm_cell_updates") if tts else None
    r = {"steps": TOTAL_STEPS, "oracle_tcm_all_cores_s": cpu.get("time_to_solution_s"),
         "gpu_tcm_s": tts.get("tcm_s") if tts else None, "gpu_dense_s": tts.get("dense_s") if tts else None}
    if upd:
        r["oracle_tcm_one_core_s_estimated"] = upd / cpu["single_thread"]["value"]
    if o512 is not None:
        wl = W.layered(steps=TOTAL_STEPS)
        a, b = o512.read_field(0), o512.read_field(1)
        dense_upd = int(np.prod(wl.shape)) * TOTAL_STEPS
        for name, th in (("all_cores", threads), ("one_core", 1)):
            rate = dense_window(wl, a, b, 1, th)
            r[f"oracle_dense_{name}_s_estimated"] = dense_upd / rate
        del a, b
    r["estimated_from"] = "rate of 2 TCM steps (1500..1502) / 1 dense step from the final state x the run's updates"
    out["layered_512"] = r
    # virtual 4096^3, first 300 steps: full runs
    wl = W.virtual(steps=300, pool_bytes=4 * 1024 ** 3)
    r = {"steps": 300}
    for name, th in (("one_core", 1), ("all_cores", threads)):
        r[f"oracle_tcm_{name}_s"], r["cell_updates"] = tcm_oracle(wl, 300, th)
    r["gpu_tcm_s"], _ = gpu_run(wl, 300)
    r["dense"] = "infeasible (4096^3 x 3 x 4 B = 824 GB)"
    out["virtual_4096_first_300"] = r
    # 256^3 precision workload: TCM on all cores in full; one core and the
    # FP64 dense grid (the reference of the error table) from windows
    wl = W.precision(256, 800)
    r = {"steps": 800}
    r["oracle_tcm_all_cores_s"], upd = tcm_oracle(wl, 800, threads)
    r["cell_updates"] = upd
    r["gpu_tcm_s"], _ = gpu_run(wl, 800)
    r["gpu_dense_s"], _ = gpu_run(wl, 800, dense=True)
    o = oracle.OracleTCM(wl.shape, wl.media, wl.dx, wl.dt, brick=wl.brick, thr_mode=wl.thr_mode, tau=wl.tau,
                         decay_alpha=wl.decay_alpha, decay_steps=wl.decay_steps)
    for x, y, z, w in wl.sources:
        o.add_source(x, y, z, np.asarray(w, np.float32))
    o.step(780)
    rates = {}
    for name, th in (("all_cores", threads), ("one_core", 1)):
        oracle.set_threads(th)
        u0 = o.updates
        t = time.perf_counter()
        o.step(4)
        rates[name] = (o.updates - u0) / (time.perf_counter() - t)
    oracle.set_threads(threads)
    r["oracle_tcm_one_core_s_estimated"] = upd / rates["one_core"]
    a, b = o.read_field(0), o.read_field(1)
    o.close()
    for name, th in (("all_cores", threads), ("one_core", 1)):
        rate = dense_window(wl, a, b, 2, th, np.float64)
        r[f"oracle_dense_f64_{name}_s_estimated"] = int(np.prod(wl.shape)) * 800 / rate
    r["estimated_from"] = "rates of 4 TCM steps (780..784) and 2 FP64 dense steps x the run's updates"
    out["precision_256"] = r
    torch.cuda.empty_cache()
    return out


def run_reference(args, rank, world):
    """The CPU oracle as the reference arm: the same K timed steps of the same
    workload as the GPU arm (ending at step 1500, reached untimed, after W
    untimed warm-up steps), on all host cores."""
    if rank != 0:
        return
    import oracle
    from paper_1702_00216_gb300 import workloads as W
    oracle.lib()
    threads = os.cpu_count() or 1
    used = oracle.set_threads(threads)
    wl = W.layered(n=args.grid, steps=TOTAL_STEPS)
    o = oracle.OracleTCM(wl.shape, wl.media, wl.dx, wl.dt, brick=wl.brick, thr_mode=wl.thr_mode,
                         tau=wl.tau, decay_alpha=wl.decay_alpha, decay_steps=wl.decay_steps)
    for x, y, z, w in wl.sources:
        o.add_source(x, y, z, np.asarray(w, np.float32))
    # the same window as the GPU arm: steps TOTAL_STEPS - K .. TOTAL_STEPS,
    # reached untimed, after W untimed warm-up steps
    t0 = max(0, TOTAL_STEPS - args.steps - args.warmup)
    o.step(t0)
    o.step(args.warmup)
    first = o.step_index
    u0 = o.updates
    t = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t
    upd = o.updates - u0
    v = upd / dt
    line = {"metric": "active-cell updates/s", "value": v, "unit": "cell-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3 / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": wl.name, "grid": list(wl.shape[::-1]), "brick": list(wl.brick),
                       "threshold": "relative 1e-6", "decay": "alpha 0.8, 20 steps", "storage": "f32",
                       "timed_steps": [first, first + args.steps]},
            "cpu_baseline": {"value": v, "unit": "cell-updates/s", "cores": used, "kind": "oracle",
                             "sample": f"steps {first}..{first + args.steps} of {wl.name} "
                                       f"({upd} cell updates, {dt:.1f} s; steps 0..{first} untimed)"},
            "e2e": {"value": v, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    o.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=TOTAL_STEPS - 5)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--grid", type=int, default=512, help="edge of the layered workload")
    ap.add_argument("--storage", choices=["f32", "bf16", "f16"], default="f32",
                    help="field storage of the timed run (the arithmetic is binary32 in all)")
    ap.add_argument("--lpf", default=None, metavar="PASS,STOP",
                    help="time the run with the Eq. 7 shut-down (fractions of Nyquist), e.g. 0.25,0.5")
    ap.add_argument("--trace", default=None,
                    help="write per-launch node updates of the untimed steps (JSON lines)")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-graphs", action="store_true",
                    help="issue every step launch directly instead of replaying CUDA graphs")
    ap.add_argument("--save-state", default=None, metavar="FILE.npz",
                    help="advance the run to --state-step, save phi^n and phi^{n-1}, exit")
    ap.add_argument("--state-step", type=int, default=TOTAL_STEPS - 20)
    ap.add_argument("--load-state", default=None, metavar="FILE.npz",
                    help="start the timed run from a saved state (profiling: few launches before it)")
    ap.add_argument("--oracle-timings", type=int, default=1,
                    help="time the oracle's time to solution per workload (0: skip)")
    ap.add_argument("--quick", action="store_true",
                    help="skip time-to-solution, e2e, CPU baseline and serving")
    ap.add_argument("--serving", type=int, default=100, help="requests in the serving stream (0: skip)")
    ap.add_argument("--serving-calibrate", type=int, default=48,
                    help="requests of the burst that calibrates the serving capacity")
    ap.add_argument("--virtual", type=int, default=1, help="run the virtual 4096^3 leg (0: skip)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = env_int("RANK", 0)
    world = env_int("WORLD_SIZE", 1)
    local_rank = env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
