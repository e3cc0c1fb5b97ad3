"""Update-procedure schedule on the GPU (Eq. 5 interval, 26-neighbour
activation of Fig. 3, and the run of the procedure on the initial state):
bit-exact against the oracle, and equal to the dense grid at threshold 0
whenever the interval does not exceed the brick edge."""
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


def het(interval, neighbours, thr_mode=0, tau=0.0, alpha=1.0, decay=0, shape=(37, 30, 45), steps=90):
    m = W.random_dense_media(shape, 21, 1.0, 2.0)
    dt = 0.5 / m.c_max()
    w = W.ricker(1 / 8, dt)
    nz, ny, nx = shape
    return W.Workload("sched", shape, m, 1.0, dt, [(3, ny - 3, 5, w), (nx - 4, 4, nz - 6, w[:30] * 2.0)], steps,
                      thr_mode=thr_mode, tau=tau, decay_alpha=alpha, decay_steps=decay,
                      interval=interval, neighbours=neighbours)


def oracle_of(wl, dense=False):
    o = oracle.OracleTCM(wl.shape, wl.media, wl.dx, wl.dt, thr_mode=wl.thr_mode, tau=wl.tau,
                         decay_alpha=wl.decay_alpha, decay_steps=wl.decay_steps, dense=dense,
                         interval=wl.interval, neighbours=wl.neighbours)
    for x, y, z, w in wl.sources:
        o.add_source(x, y, z, np.asarray(w, F32))
    return o


def compare(s, o, chunks):
    for c in chunks:
        s.step(c)
        o.step(c)
        assert np.array_equal(s.read_field(0), o.read_field(0))
        assert np.array_equal(s.read_field(1), o.read_field(1))
        assert np.array_equal(s.active_bricks(), o.active_bricks())
    assert s.updates == o.updates


@pytest.mark.parametrize("interval", [2, 5, 8])
def test_interval26_threshold0_equals_oracle_and_dense(interval):
    wl = het(interval, 26)
    s = tcm.Sim.from_workload(wl)
    assert s.schedule() == (interval, 26)
    o = oracle_of(wl)
    compare(s, o, [7, 13, 30, 40])          # checkpoints inside intervals too
    d = tcm.Sim.from_workload(het(1, 6), dense=True)
    d.step(90)
    assert np.array_equal(s.read_field(0), d.read_field(0))
    assert s.updates < d.updates
    s.close()
    d.close()


@pytest.mark.parametrize("interval,neighbours,mode,tau,alpha,decay", [
    (3, 26, 1, 1e-3, 0.7, 7),
    (4, 6, 0, 2e-3, 0.8, 5),
    (1, 26, 1, 3e-3, 0.9, 3),
    (6, 26, 0, 1e-3, 1.0, 0),
])
def test_schedules_with_thresholds_equal_oracle(interval, neighbours, mode, tau, alpha, decay):
    wl = het(interval, neighbours, mode, tau, alpha, decay, steps=120)
    s = tcm.Sim.from_workload(wl)
    o = oracle_of(wl)
    compare(s, o, [11, 29, 40, 40])
    s.close()


def test_eq5_interval():
    m = W.homogeneous(1.0)
    s = tcm.Sim((16, 16, 16), m, 1.0, 0.5)
    s.set_schedule(0, 26)                   # Eq. 5: 1 * 8 / (2 * 1 * 0.5) = 8
    assert s.schedule() == (8, 26)
    s.close()
    s = tcm.Sim((16, 16, 16), W.Media(kind="rules", c_background=1.0, layers=[(8.0, 2.0)]), 1.0, 0.25)
    s.set_schedule(0, 6)                    # 8 / (2 * 2 * 0.25) = 8; c_max = 2
    assert s.schedule() == (8, 6)
    s.close()
    s = tcm.Sim((16, 16, 16), m, 1.0, 0.3)
    s.set_schedule(0, 26)                   # floor(8 / 0.6) = 13
    assert s.schedule() == (13, 26)
    with pytest.raises(tcm.TCMError):
        s.set_schedule(2, 18)
    s.step(1)
    with pytest.raises(tcm.TCMError):
        s.set_schedule(2, 26)               # after the first step
    s.close()


@pytest.mark.parametrize("interval,neighbours", [(1, 6), (4, 26)])
def test_initial_field_on_cell_faces(interval, neighbours):
    shape = (24, 24, 24)
    m = W.homogeneous(1.0)
    now = np.zeros(shape, F32)
    prev = np.zeros(shape, F32)
    now[8, 8:16, 8:16] = 1.0
    now[8:16, 15, 15] = -0.5
    prev[15, 15, 15] = 0.25
    s = tcm.Sim(shape, m, 1.0, 0.5)
    s.set_schedule(interval, neighbours)
    s.set_field(now, prev)
    o = oracle.OracleTCM(shape, m, 1.0, 0.5, interval=interval, neighbours=neighbours)
    o.set_field(now, prev)
    compare(s, o, [1, 5, 6])
    k = oracle.k_from_c(np.ones(shape, F32), 0.5, 1.0, F32)
    a, _ = oracle.dense_run(k, now, prev, 12)
    assert np.array_equal(s.read_field(0), a)
    s.close()


def test_batch_with_mixed_schedules_equals_solo():
    wls = [het(1, 6, 1, 1e-3, 0.8, 4), het(3, 26, 1, 1e-3, 0.8, 4), het(8, 26),
           het(5, 6, 0, 1e-3, 0.9, 2, shape=(20, 26, 33))]
    b = tcm.Batch(pool_bytes=30000 * tcm.tcm_slot_bytes(), max_bricks=40000, max_sims=8)
    sims = [b.add(wl) for wl in wls]
    b.step(17)
    late = b.add(het(4, 26, 0, 2e-3, 1.0, 0), n_steps=30)   # joins mid-interval of the others
    b.step(40)
    for wl, sim in zip(wls, sims):
        s = tcm.Sim.from_workload(wl)
        s.step(57)
        assert np.array_equal(sim.read_field(0), s.read_field(0))
        assert np.array_equal(sim.active_bricks(), s.active_bricks())
        s.close()
    s = tcm.Sim.from_workload(het(4, 26, 0, 2e-3, 1.0, 0))
    s.step(30)
    assert late.done() and np.array_equal(late.read_field(0), s.read_field(0))
    s.close()
    b.close()
