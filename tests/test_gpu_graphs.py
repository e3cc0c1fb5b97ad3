"""Step launches replayed from captured CUDA graphs give exactly the results
of launching every step directly (solo simulations, batches whose members
freeze at different steps, update schedules and the Eq. 7 shut-down)."""
import numpy as np
import pytest

from paper_1702_00216_gb300 import tcm
from paper_1702_00216_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def wl(shape=(36, 31, 44), interval=1, neighbours=6, lpf=None, seed=3):
    m = W.random_dense_media(shape, seed, 1.0, 2.0)
    dt = 0.5 / m.c_max()
    nz, ny, nx = shape
    return W.Workload("g", shape, m, 1.0, dt, [(nx // 3, ny // 2, nz // 4, W.ricker(1 / 8, dt))], 0,
                      thr_mode=1, tau=1e-4, decay_alpha=0.8, decay_steps=6, interval=interval,
                      neighbours=neighbours, lpf=lpf)


def test_solo_graphs_equal_direct_launches():
    outs = []
    for graphs in (True, False):
        s = tcm.Sim.from_workload(wl(), graphs=graphs)
        s.step(37)
        s.step(90)
        outs.append((s.read_field(0), s.read_field(1), s.active_bricks(), s.updates, s.launches,
                     s.graph_launches()))
        s.close()
    (a0, a1, ia, ua, la, ga), (b0, b1, ib, ub, lb, gb) = outs
    assert np.array_equal(a0, b0) and np.array_equal(a1, b1) and np.array_equal(ia, ib) and ua == ub
    assert la == lb == 127 and ga > 0 and gb == 0


def test_batch_graphs_with_freezes_and_variants():
    specs = [(wl(), 50), (wl((30, 30, 30), 3, 26, seed=5), 41), (wl((28, 33, 25), lpf=(0.25, 0.5), seed=7), 77),
             (wl((24, 24, 24), 8, 26, seed=9), 0)]
    res = []
    for graphs in (True, False):
        b = tcm.Batch(pool_bytes=20000 * tcm.tcm_slot_bytes(), max_bricks=40000, max_sims=8, graphs=graphs)
        sims = [b.add(w, n_steps=n) for w, n in specs]
        b.step(30)
        late = b.add(wl((26, 27, 28), seed=11), n_steps=25)
        b.step(60)
        res.append([(s.read_field(0), s.active_bricks(), s.updates, s.step_index) for s in sims + [late]])
        b.close()
    for x, y in zip(*res):
        assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1]) and x[2:] == y[2:]
    assert [r[3] for r in res[0]] == [50, 41, 77, 90, 25]
