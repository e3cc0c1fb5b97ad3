"""Batching: several simulations stepped by one launch per step give, bit for
bit, the results each gives alone (and the oracle's), including simulations
admitted while others are running, frozen after their step count, and
removed with their boxes returned to the pool."""
import numpy as np
import pytest

import oracle
from paper_1702_00216_gb300 import tcm
from paper_1702_00216_gb300 import workloads as W

pytestmark = pytest.mark.gpu
F32 = np.float32


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def workloads():
    rng = np.random.default_rng(5)
    out = []
    # ragged heterogeneous, threshold 0
    m = W.random_dense_media((21, 30, 37), 3, 1.0, 2.0)
    dt = 0.5 / m.c_max()
    out.append(W.Workload("a", (21, 30, 37), m, 1.0, dt, [(5, 6, 7, W.ricker(1 / 8, dt))], 0))
    # layered rules, relative threshold with decay
    m = W.Media(kind="rules", c_background=1.0, layers=[(20.0, 1.6)])
    dt = 0.5 / m.c_max()
    out.append(W.Workload("b", (40, 32, 48), m, 1.0, dt, [(20, 16, 10, W.ricker(1 / 8, dt))], 0,
                          thr_mode=1, tau=1e-4, decay_alpha=0.7, decay_steps=4))
    # homogeneous, absolute threshold, two sources
    out.append(W.Workload("c", (32, 32, 32), W.homogeneous(1.0), 1.0, 0.5,
                          [(8, 9, 10, W.ricker(1 / 6, 0.5)), (25, 20, 22, W.ricker(1 / 10, 0.5))], 0,
                          thr_mode=0, tau=2e-3))
    # sphere inclusion, decay without threshold release
    m = W.Media(kind="rules", c_background=1.0, spheres=[(20.5, 18.0, 16.0, 7.0, 1.7)])
    dt = 0.5 / m.c_max()
    out.append(W.Workload("d", (33, 35, 41), m, 1.0, dt,
                          [(int(rng.integers(41)), int(rng.integers(35)), int(rng.integers(33)),
                            W.ricker(1 / 7, dt))], 0, thr_mode=1, tau=1e-6, decay_alpha=0.8,
                          decay_steps=20))
    return out


def solo(wl, steps):
    s = tcm.Sim.from_workload(wl)
    s.step(steps)
    r = (s.read_field(0), s.read_field(1), s.active_bricks(), s.updates)
    s.close()
    return r


def test_batch_equals_solo_and_oracle():
    wls = workloads()
    steps = 70
    b = tcm.Batch(pool_bytes=20000 * tcm.tcm_slot_bytes(), max_bricks=40000, max_sims=8)
    sims = [b.add(wl) for wl in wls]
    b.step(steps)
    for wl, s in zip(wls, sims):
        a0, a1, ids, upd = solo(wl, steps)
        assert np.array_equal(s.read_field(0), a0), wl.name
        assert np.array_equal(s.read_field(1), a1), wl.name
        assert np.array_equal(s.active_bricks(), ids), wl.name
        assert s.updates == upd
        o = oracle.OracleTCM(wl.shape, wl.media, wl.dx, wl.dt, thr_mode=wl.thr_mode, tau=wl.tau,
                             decay_alpha=wl.decay_alpha, decay_steps=wl.decay_steps)
        for x, y, z, w in wl.sources:
            o.add_source(x, y, z, np.asarray(w, F32))
        o.step(steps)
        assert np.array_equal(o.read_field(0), a0), wl.name
    b.close()


def test_staggered_admission_freeze_and_remove():
    wls = workloads()
    b = tcm.Batch(pool_bytes=20000 * tcm.tcm_slot_bytes(), max_bricks=40000, max_sims=8)
    slots, free0, _ = b.info()
    first = b.add(wls[0], n_steps=50)
    b.step(20)
    second = b.add(wls[1], n_steps=40)            # admitted while the first runs
    b.step(25)
    third = b.add(wls[2], n_steps=30)
    b.step(60)                                   # first and second finish and freeze
    assert first.done() and second.done() and third.done()
    assert first.step_index == 50 and second.step_index == 40 and third.step_index == 30
    for wl, s, n in zip(wls[:3], (first, second, third), (50, 40, 30)):
        a0, a1, ids, upd = solo(wl, n)
        assert np.array_equal(s.read_field(0), a0), wl.name
        assert np.array_equal(s.read_field(1), a1), wl.name
        assert s.updates == upd
    assert b.info()[1] < free0
    for s in (first, second, third):
        b.remove(s)
    assert b.info() == (slots, free0, 0)
    # the freed brick space and boxes are reused by a new simulation
    again = b.add(wls[3], n_steps=35)
    b.step(35)
    a0, _, ids, _ = solo(wls[3], 35)
    assert np.array_equal(again.read_field(0), a0)
    assert np.array_equal(again.active_bricks(), ids)
    b.close()


def test_batch_rejects_when_full():
    b = tcm.Batch(pool_bytes=64 * tcm.tcm_slot_bytes(), max_bricks=600, max_sims=2)
    wl = W.small(n=64, steps=10)                  # 512 bricks
    b.add(wl)
    with pytest.raises(tcm.TCMError) as e:
        b.add(wl)                                 # brick space exhausted
    assert e.value.status == tcm.TCM_ENOMEM
    b.close()
