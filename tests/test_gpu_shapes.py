"""Brick shapes 4x4x4 and 16x8x8 (8x8x8 is covered everywhere else): each
shape's build of the library equals the oracle run with the same cells, bit
for bit (fields, active sets, node updates), and the dense grid at
threshold 0."""
import numpy as np
import pytest

import oracle
from paper_1702_00216_gb300 import tcm
from paper_1702_00216_gb300 import workloads as W

pytestmark = pytest.mark.gpu
F32 = np.float32
SHAPES = [(4, 4, 4), (16, 8, 8)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def het(brick, thr_mode=0, tau=0.0, alpha=1.0, decay=0, shape=(37, 30, 45), interval=1, neighbours=6, lpf=None):
    m = W.random_dense_media(shape, 17, 1.0, 2.1)
    dt = 0.5 / m.c_max()
    w = W.ricker(1 / 8, dt)
    nz, ny, nx = shape
    return W.Workload("shape", shape, m, 1.0, dt, [(5, ny - 4, 6, w), (nx - 7, 3, nz - 5, w[:35] * 1.5)], 0,
                      brick=brick, thr_mode=thr_mode, tau=tau, decay_alpha=alpha, decay_steps=decay,
                      interval=interval, neighbours=neighbours, lpf=lpf)


def oracle_of(wl, storage="f32"):
    o = oracle.OracleTCM(wl.shape, wl.media, wl.dx, wl.dt, brick=wl.brick, thr_mode=wl.thr_mode, tau=wl.tau,
                         decay_alpha=wl.decay_alpha, decay_steps=wl.decay_steps, interval=wl.interval,
                         neighbours=wl.neighbours, lpf=wl.lpf, storage=storage)
    for x, y, z, w in wl.sources:
        o.add_source(x, y, z, np.asarray(w, F32))
    return o


def compare(s, o, chunks, exact=True):
    for c in chunks:
        s.step(c)
        o.step(c)
        a, b = s.read_field(0), o.read_field(0)
        if exact:
            assert np.array_equal(a, b) and np.array_equal(s.read_field(1), o.read_field(1))
        else:
            assert np.abs(a.astype(np.float64) - b).max() <= 1e-6 * max(np.abs(b).max(), 1e-30)
        assert np.array_equal(s.active_bricks(), o.active_bricks())
    assert s.updates == o.updates


@pytest.mark.parametrize("brick", SHAPES)
def test_threshold0_equals_oracle_and_dense(brick):
    wl = het(brick)
    s = tcm.Sim.from_workload(wl)
    compare(s, oracle_of(wl), [9, 31, 40])
    d = tcm.Sim.from_workload(het((8, 8, 8)), dense=True)
    d.step(80)
    assert np.array_equal(s.read_field(0), d.read_field(0))
    s.close()
    d.close()


@pytest.mark.parametrize("brick", SHAPES)
@pytest.mark.parametrize("mode,tau,alpha,decay", [(1, 1e-4, 0.8, 5), (0, 2e-3, 1.0, 0)])
def test_thresholds_equal_oracle(brick, mode, tau, alpha, decay):
    wl = het(brick, mode, tau, alpha, decay)
    s = tcm.Sim.from_workload(wl)
    compare(s, oracle_of(wl), [13, 27, 50])
    s.close()


@pytest.mark.parametrize("brick,storage", [((4, 4, 4), "bf16"), ((16, 8, 8), "f16")])
def test_16bit_storage_equals_oracle(brick, storage):
    wl = het(brick, 1, 1e-4, 0.8, 5)
    s = tcm.Sim.from_workload(wl, storage=storage)
    compare(s, oracle_of(wl, storage), [20, 40])
    s.close()


@pytest.mark.parametrize("brick,interval", [((4, 4, 4), 4), ((16, 8, 8), 8)])
def test_interval26_threshold0_equals_dense(brick, interval):
    wl = het(brick, interval=interval, neighbours=26)
    s = tcm.Sim.from_workload(wl)
    compare(s, oracle_of(wl), [17, 43])
    d = tcm.Sim.from_workload(het((8, 8, 8)), dense=True)
    d.step(60)
    assert np.array_equal(s.read_field(0), d.read_field(0))
    s.close()
    d.close()


def test_lpf_on_4cubed_matches_oracle_and_not_on_16x8x8():
    wl = het((4, 4, 4), 1, 2e-3, lpf=(0.25, 0.5))
    s = tcm.Sim.from_workload(wl)
    compare(s, oracle_of(wl), [10, 30, 30], exact=False)
    s.close()
    s = tcm.Sim.from_workload(het((16, 8, 8)))
    with pytest.raises(tcm.TCMError):
        s.set_lpf_shutdown(0.25, 0.5)
    s.close()


def test_batch_of_4cubed_sims_equals_solo():
    wls = [het((4, 4, 4), 1, 1e-4, 0.8, 5), het((4, 4, 4), shape=(20, 22, 19)),
           het((4, 4, 4), 0, 1e-3, interval=3, neighbours=26, shape=(25, 25, 25))]
    b = tcm.Batch(pool_bytes=60000 * tcm.tcm_slot_bytes((4, 4, 4)), max_bricks=100000, max_sims=4,
                  brick=(4, 4, 4))
    sims = [b.add(w) for w in wls]
    b.step(45)
    for w, sim in zip(wls, sims):
        s = tcm.Sim.from_workload(w)
        s.step(45)
        assert np.array_equal(sim.read_field(0), s.read_field(0))
        assert np.array_equal(sim.active_bricks(), s.active_bricks())
        s.close()
    with pytest.raises(tcm.TCMError):
        b.add(het((8, 8, 8)))          # a batch holds one brick shape
    b.close()


def test_set_field_16x8x8():
    shape = (13, 11, 37)
    v = W.eigenmode(shape, (1, 2, 3)).astype(F32)
    s = tcm.Sim(shape, W.homogeneous(1.0), 1.0, 0.5, brick=(16, 8, 8))
    s.set_field(v, v * F32(0.99))
    o = oracle.OracleTCM(shape, W.homogeneous(1.0), 1.0, 0.5, brick=(16, 8, 8))
    o.set_field(v, v * F32(0.99))
    compare(s, o, [5, 20])
    s.close()


@pytest.mark.parametrize("warps", [4, 8, 12])
@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_cta_blocking_builds_equal_the_oracle(warps, storage):
    """The 8x8x8 builds with 4, 8 and 12 warps per CTA of the step kernel
    (the autotuner's blocking axis; 12 holds the 16-bit columns as loaded and
    takes 4 update items per thread) give the oracle's fields, active sets
    and updates bit for bit, at a level above 0 with shut-down, in a single
    simulation and in a batch."""
    wl = het((8, 8, 8), thr_mode=1, tau=1e-4, alpha=0.7, decay=4)
    s = tcm.Sim.from_workload(wl, cta_warps=warps, storage=storage)
    compare(s, oracle_of(wl, storage), [1, 9, 30, 60])
    s.close()
    b = tcm.Batch(pool_bytes=4000 * tcm.tcm_slot_bytes(), max_bricks=1 << 14, max_sims=4, cta_warps=warps,
                  storage=storage)
    sims = [b.add(wl), b.add(het((8, 8, 8), shape=(21, 30, 17)))]
    b.step(50)
    for sm, w in zip(sims, (wl, het((8, 8, 8), shape=(21, 30, 17)))):
        o = oracle_of(w, storage)
        o.step(50)
        assert np.array_equal(sm.read_field(0), o.read_field(0))
        assert np.array_equal(sm.active_bricks(), o.active_bricks())
    b.close()


def test_cta_blocking_rejects_unbuilt_combinations():
    wl = het((4, 4, 4))
    with pytest.raises(tcm.TCMError) as e:
        tcm.Sim.from_workload(wl, cta_warps=16)
    assert e.value.status == tcm.TCM_EINVAL
    with pytest.raises(tcm.TCMError) as e:
        tcm.Sim.from_workload(het((8, 8, 8)), cta_warps=16)
    assert e.value.status == tcm.TCM_EINVAL


@pytest.mark.parametrize("warps", [4, 8, 12])
def test_mixed_storage_batch_in_every_blocking(warps):
    """A batch of mixed storage (FP32, BF16 and FP16 simulations stepped by
    one launch) in each CTA blocking of the 8x8x8 shape -- with 12 warps the
    16-bit bricks take the path that holds their columns as loaded -- equals
    the oracle in each simulation's storage form, bit for bit."""
    wls = [het((8, 8, 8), thr_mode=1, tau=1e-4, alpha=0.7, decay=4),
           het((8, 8, 8), thr_mode=1, tau=1e-4, alpha=0.7, decay=4, shape=(21, 30, 17)),
           het((8, 8, 8), shape=(26, 19, 33))]
    storages = ["bf16", "f32", "f16"]
    b = tcm.Batch(pool_bytes=6000 * tcm.tcm_slot_bytes(), max_bricks=1 << 15, max_sims=4, cta_warps=warps,
                  storage="mixed")
    sims = [b.add(w, storage=st) for w, st in zip(wls, storages)]
    b.step(45)
    for sm, w, st in zip(sims, wls, storages):
        o = oracle_of(w, st)
        o.step(45)
        assert np.array_equal(sm.read_field(0), o.read_field(0)), (warps, st)
        assert np.array_equal(sm.read_field(1), o.read_field(1)), (warps, st)
        assert np.array_equal(sm.active_bricks(), o.active_bricks())
        assert sm.updates == o.updates
    b.close()
