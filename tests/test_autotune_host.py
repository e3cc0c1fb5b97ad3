"""Autotuner host logic with the timing replaced: candidate sets, the
choice of the fastest window, caching and applying a choice."""
import pytest

from paper_1702_00216_gb300 import autotune as A
from paper_1702_00216_gb300 import workloads as W


def test_candidates():
    assert [c.label() for c in A.candidates()] == ["4x4x4", "8x8x8", "16x8x8"]
    labels = [c.label() for c in A.candidates(allow_schedule=True)]
    assert labels[3:] == ["4x4x4/eq5-26", "8x8x8/eq5-26", "16x8x8/eq5-26"]


def test_picks_fastest_window_and_caches(monkeypatch):
    calls = []

    def fake(wl, c, start, count, device=0, storage="f32", ref=None):
        calls.append((c.label(), start, count))
        ms = {"4x4x4": 3.0, "8x8x8": 1.0, "16x8x8": 2.0}[c.label()]
        return {"config": c.label(), "brick": list(c.brick), "schedule": [c.interval, c.neighbours],
                "window_ms": ms, "cell_updates": 1, "updates_per_s": 1.0}

    monkeypatch.setattr(A, "measure", fake)
    A._CACHE.clear()
    wl = W.small(n=32, steps=100)
    r = A.autotune(wl)
    assert r["best"].brick == (8, 8, 8) and r["window"] == [40, 60]
    assert [t["config"] for t in r["table"]] == ["8x8x8", "16x8x8", "4x4x4"]
    n = len(calls)
    assert A.autotune(wl) is r and len(calls) == n        # cached
    w2 = A.apply(wl, A.Candidate((16, 8, 8), 0, 26))
    assert w2.brick == (16, 8, 8) and (w2.interval, w2.neighbours) == (0, 26) and wl.brick == (8, 8, 8)


def test_prefetch_refinement(monkeypatch):
    """With allow_prefetch the fastest configuration is timed once more with
    the L2 prefetch off, and the faster of the two is chosen."""
    calls = []

    def fake(wl, c, start, count, device=0, storage="f32", ref=None):
        calls.append(c.label())
        ms = {"4x4x4": 3.0, "8x8x8": 1.0, "16x8x8": 2.0, "8x8x8/no-prefetch": 0.5}[c.label()]
        return {"config": c.label(), "brick": list(c.brick), "schedule": [c.interval, c.neighbours],
                "prefetch": c.prefetch, "window_ms": ms, "cell_updates": 1, "updates_per_s": 1.0}

    monkeypatch.setattr(A, "measure", fake)
    A._CACHE.clear()
    wl = W.small(n=32, steps=100)
    r = A.autotune(wl, allow_prefetch=True)
    assert calls == ["4x4x4", "8x8x8", "16x8x8", "8x8x8/no-prefetch"]
    assert r["best"].brick == (8, 8, 8) and r["best"].prefetch is False
    assert A.apply(wl, r["best"]).prefetch is False and wl.prefetch is True


def test_blocking_axis_and_labels():
    labels = [c.label() for c in A.candidates(allow_blocking=True)]
    assert labels == ["4x4x4", "8x8x8", "16x8x8", "8x8x8/w4", "8x8x8/w12"]
    # 16-bit storage: the library's default for 8x8x8 is 12 warps, so the
    # axis adds 8 instead
    labels = [c.label() for c in A.candidates(allow_blocking=True, storage="bf16")]
    assert labels == ["4x4x4", "8x8x8", "16x8x8", "8x8x8/w4", "8x8x8/w8"]
    assert A.default_warps((8, 8, 8), "f16") == 12 and A.default_warps((16, 8, 8), "bf16") == 8
    c = A.Candidate((8, 8, 8), cta_warps=12, prefetch=False)
    assert c.same_results_as() == A.Candidate((8, 8, 8))
    wl = W.small(n=32, steps=100)
    assert A.apply(wl, c).cta_warps == 12 and wl.cta_warps == 0


def test_choice_respects_the_accuracy_tolerance(monkeypatch):
    """Schedules and shapes that change results are chosen only if they stay
    within the tolerance of the dense grid; the fastest within it wins."""
    def fake(wl, c, start, count, device=0, storage="f32", ref=None):
        ms = {"4x4x4": 3.0, "8x8x8": 2.0, "16x8x8": 2.5, "8x8x8/w4": 2.2, "8x8x8/w12": 2.1,
              "4x4x4/eq5-26": 0.5, "8x8x8/eq5-26": 1.5, "16x8x8/eq5-26": 1.8}[c.label()]
        rel = {"4x4x4/eq5-26": 3e-5}.get(c.label(), 2e-6)
        return {"config": c.label(), "window_ms": ms, "cell_updates": 1, "updates_per_s": 1.0,
                "max_abs_diff_vs_dense": rel, "rel_diff_vs_dense": rel}

    monkeypatch.setattr(A, "measure", fake)
    monkeypatch.setattr(A, "dense_reference", lambda wl, steps, device=0: object())
    A._CACHE.clear()
    wl = W.small(n=32, steps=100)
    r = A.autotune(wl, allow_schedule=True, allow_blocking=True, accuracy=True, tolerance=1e-5)
    assert r["table"][0]["config"] == "4x4x4/eq5-26"        # fastest, but outside the tolerance
    assert r["best"].label() == "8x8x8/eq5-26"
    assert "within" in r["choice"]
