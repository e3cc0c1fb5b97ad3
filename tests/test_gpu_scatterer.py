"""The sound-soft scatterer scenario (a sphere beside a cube with c = 0, a
directional Gaussian beam from the boundary, bi-polar pulse), scaled down:
GPU == oracle bit for bit, threshold-0 TCM == dense, the obstacles' nodes
stay exactly zero (k = 0 there), and the obstacle casts a shadow."""
import dataclasses

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


def oracle_of(wl, dense=False):
    o = oracle.OracleTCM(wl.shape, wl.media, wl.dx, wl.dt, thr_mode=wl.thr_mode, tau=wl.tau,
                         decay_alpha=wl.decay_alpha, decay_steps=wl.decay_steps, dense=dense)
    for x, y, z, w in wl.sources:
        o.add_source(x, y, z, np.asarray(w, F32))
    return o


def test_threshold0_tcm_equals_dense_and_obstacle_stays_zero():
    wl = W.scatterer(steps=220)
    s = tcm.Sim.from_workload(wl)
    d = tcm.Sim.from_workload(wl, dense=True)
    s.step(220)
    d.step(220)
    a = s.read_field(0)
    assert np.array_equal(a, d.read_field(0)) and np.array_equal(s.read_field(1), d.read_field(1))
    inside = wl.media.c == 0
    assert inside.sum() > 1000 and np.all(a[inside] == 0) and np.all(s.read_field(1)[inside] == 0)
    assert s.updates < d.updates
    o = oracle_of(wl, dense=True)
    o.step(220)
    assert np.array_equal(o.read_field(0), a)
    s.close()
    d.close()


def test_threshold_run_equals_oracle():
    wl = dataclasses.replace(W.scatterer(steps=200), thr_mode=1, tau=1e-4, decay_alpha=0.8, decay_steps=10)
    s = tcm.Sim.from_workload(wl)
    o = oracle_of(wl)
    for c in (60, 70, 70):
        s.step(c)
        o.step(c)
        assert np.array_equal(s.read_field(0), o.read_field(0))
        assert np.array_equal(s.active_bricks(), o.active_bricks())
    assert s.updates == o.updates
    s.close()


def test_obstacle_casts_a_shadow():
    wl = W.scatterer(steps=260)
    free = dataclasses.replace(wl, media=W.dense_media(np.full(wl.shape, 340.0, np.float32)))
    out = []
    for w in (wl, free):
        s = tcm.Sim.from_workload(w)
        e = np.zeros(w.shape)
        for _ in range(26):
            s.step(10)
            e += s.read_field(0).astype(np.float64) ** 2
        out.append(e)
        s.close()
    nz, ny, nx = wl.shape
    behind = (slice(int(nz * 0.3), int(nz * 0.55)), slice(int(ny * 0.4), int(ny * 0.6)),
              slice(int(nx * 0.75), int(nx * 0.9)))
    assert out[0][behind].sum() < 0.5 * out[1][behind].sum()
