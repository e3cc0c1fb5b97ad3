"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Floating point: binary32 round-to-nearest on both sides with one fixed
grouping of Eq. 3, so fields must agree bit for bit (this is inside the
stated tolerance max|d phi| <= 1e-5 max|phi|, asserted as well).  Active
brick sets are compared as sorted id sets (box numbering depends on atomic
order and is never compared).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1702_00216_gb300 import tcm
from paper_1702_00216_gb300 import workloads as W

pytestmark = pytest.mark.gpu
F32 = np.float32
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def pair(wl, dense=False, pool_bytes=None, **okw):
    g = tcm.Sim.from_workload(wl, dense=dense, pool_bytes=pool_bytes)
    o = oracle.OracleTCM(wl.shape, wl.media, wl.dx, wl.dt, brick=wl.brick, thr_mode=wl.thr_mode,
                         tau=wl.tau, decay_alpha=wl.decay_alpha, decay_steps=wl.decay_steps,
                         dense=dense, **okw)
    for x, y, z, w in wl.sources:
        o.add_source(x, y, z, np.asarray(w, F32))
    return g, o


def assert_same(g, o, window=None):
    kw = {} if window is None else {"origin": window[0], "size": window[1]}
    for which in (0, 1):
        a, b = g.read_field(which, **kw), o.read_field(which, **kw)
        scale = max(float(np.max(np.abs(b))), 1e-30)
        assert float(np.max(np.abs(a - b))) <= TOL * scale
        assert np.array_equal(a, b), f"half {which}: max |d| = {float(np.max(np.abs(a - b)))}"
    assert np.array_equal(g.active_bricks(), o.active_bricks())


@pytest.mark.parametrize("dense", [False, True])
def test_small_config_64cubed(dense):
    """64^3, c = 1, Courant 0.5, centred Ricker, 100 steps, 8^3 bricks, threshold 0."""
    wl = W.small()
    g, o = pair(wl, dense=dense)
    done = 0
    for cp in (1, 2, 9, 33, 60, 100):
        g.step(cp - done)
        o.step(cp - done)
        done = cp
        assert_same(g, o)
        assert g.active_count() == o.active_count()
    assert g.updates == o.updates
    assert g.launches == 100


def test_threshold0_tcm_equals_dense_gpu():
    wl = W.small()
    g, _ = pair(wl)
    d = tcm.Sim.from_workload(wl, dense=True)
    g.step(100)
    d.step(100)
    assert np.array_equal(g.read_field(0), d.read_field(0))
    assert np.array_equal(g.read_field(1), d.read_field(1))


@pytest.mark.parametrize("shape", [(21, 29, 37), (8, 8, 8), (3, 5, 2), (17, 9, 33)])
def test_heterogeneous_ragged_multisource(shape):
    rng = np.random.default_rng(sum(shape))
    media = W.random_dense_media(shape, 7, 1.0, 2.0)
    dt = 0.5 / media.c_max()
    nz, ny, nx = shape
    srcs = [(int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(nz)),
             W.ricker(1 / rng.uniform(4, 10), dt)) for _ in range(3)]
    srcs.append((nx - 1, ny - 1, nz - 1, W.ricker(1 / 6, dt)))
    srcs.append((srcs[0][0], srcs[0][1], srcs[0][2], W.ricker(1 / 5, dt)))   # two at one node
    wl = W.Workload("het", shape, media, 1.0, dt, srcs, 70)
    g, o = pair(wl)
    for _ in range(7):
        g.step(10)
        o.step(10)
        assert_same(g, o)


@pytest.mark.parametrize("dx", [1.0, 0.25, 0.75])
def test_rules_media_bulking_matches_oracle(dx):
    """Heterogenic Bulking: the GPU's per-brick classification and scalar k
    equal the oracle's for layers cutting bricks and a sphere; node spacings
    that are powers of two (the quotient c dt / dx taken as an exact product)
    and one that is not (a division)."""
    shape = (40, 48, 56)
    media = W.Media(kind="rules", c_background=1.0, layers=[(12.0, 1.5), (29.5, 2.0)],
                    spheres=[(27.3, 20.0, 21.0, 9.5, 0.7), (8.0, 8.0, 8.0, 8.0, 2.2)])
    dt = 0.5 * dx / media.c_max()
    wl = W.Workload("rules", shape, media, dx, dt, [(20, 24, 18, W.ricker(1 / 8, dt / dx))], 80)
    g, o = pair(wl)
    nb = g.mx * g.my * g.mz
    kinds = set()
    for b in range(nb):
        gb, ob = g.brick_media(b), o.brick_media(b)
        kinds.add(gb[0])
        assert gb[0] == ob[0], b
        if gb[0] == 1:
            assert np.float32(gb[1]) == np.float32(ob[1]), b
    assert kinds == {1, 2}
    g.step(80)
    o.step(80)
    assert_same(g, o)


@pytest.mark.parametrize("dx", [0.5, 0.75])
def test_dense_media_node_spacing_matches_oracle(dx):
    """Per-node k from a dense velocity array (every brick bulked) with node
    spacings of both kinds: 50 steps bit-exact against the oracle."""
    shape = (24, 20, 28)
    media = W.random_dense_media(shape, 5, 1.0, 2.0)
    dt = 0.5 * dx / media.c_max()
    wl = W.Workload("dx", shape, media, dx, dt, [(9, 10, 12, W.ricker(1 / 8, dt / dx))], 50)
    g, o = pair(wl)
    g.step(50)
    o.step(50)
    assert_same(g, o)


@pytest.mark.parametrize("mode,tau,alpha,D", [(tcm.TCM_THR_ABSOLUTE, 3e-2, 1.0, 0),
                                               (tcm.TCM_THR_ABSOLUTE, 1e-2, 0.8, 5),
                                               (tcm.TCM_THR_RELATIVE, 1e-3, 0.7, 3),
                                               (tcm.TCM_THR_RELATIVE, 1e-6, 0.8, 20)])
def test_threshold_decay_retire_reuse(mode, tau, alpha, D):
    """Thresholds above 0: triggering, shut-down (Eq. 6), release and box
    reuse, step by step against the oracle."""
    shape = (40, 48, 56)
    media = W.Media(kind="rules", c_background=1.0, layers=[(20.0, 1.4)])
    dt = 0.5 / media.c_max()
    wl = W.Workload("thr", shape, media, 1.0, dt, [(20, 24, 10, W.ricker(1 / 8, dt))], 240,
                    thr_mode=mode, tau=tau, decay_alpha=alpha, decay_steps=D)
    g, o = pair(wl)
    counts = []
    for n in range(240):
        g.step(1)
        o.step(1)
        if n % 7 == 0 or n > 230:
            assert np.array_equal(g.active_bricks(), o.active_bricks()), n
        counts.append(o.active_count()[0])
    assert_same(g, o)
    assert g.updates == o.updates


def test_pool_exhaustion_reports_enomem():
    wl = W.small(n=48, steps=60)
    g = tcm.Sim.from_workload(wl, pool_bytes=5 * tcm.tcm_slot_bytes())
    with pytest.raises(tcm.TCMError) as e:
        g.step(60)
    assert e.value.status == tcm.TCM_ENOMEM
    with pytest.raises(tcm.TCMError) as e:
        g.step(1)
    assert e.value.status == tcm.TCM_ESTATE
    assert g.active_count()[0] <= 5      # still readable
    g.read_field(0)


def test_energy_matches_oracle_and_is_conserved():
    """FP64 energy reduction on the device equals the oracle's energy of the
    same (bit-equal) fields; at threshold 0 it is constant after the source."""
    shape = (24, 26, 30)
    media = W.random_dense_media(shape, 3, 1.0, 1.6)
    dt = 0.5 / media.c_max()
    w = W.ricker(1 / 6, dt)
    wl = W.Workload("energy", shape, media, 1.0, dt, [(12, 13, 11, w)], len(w) + 150)
    g, o = pair(wl)
    k = oracle.k_from_c(media.c, dt, 1.0, F32)
    es = []
    for n in (len(w) + 10, len(w) + 150):
        g.step(n - g.step_index)
        o.step(n - o.step_index)
        e_ref = oracle.energy(k, o.read_field(0), o.read_field(1))
        e_gpu = g.energy()
        assert e_gpu == pytest.approx(e_ref, rel=1e-12)
        es.append(e_gpu)
    assert abs(es[1] - es[0]) / es[0] < 1e-5      # FP32 recursion, FP64 sum


def test_set_field_eigenmode():
    """Initial fields from tcm_set_field (an eigenmode on a ragged grid)."""
    shape = (11, 9, 13)
    v = W.eigenmode(shape, (1, 2, 3)).astype(F32)
    wl = W.Workload("mode", shape, W.homogeneous(1.0), 1.0, 0.5, [], 50)
    g, o = pair(wl)
    g.set_field(v, (0.9 * v).astype(F32))
    o.set_field(v, (0.9 * v).astype(F32))
    g.step(50)
    o.step(50)
    assert_same(g, o)


def test_mirror_symmetry_gpu():
    n = 41
    wl = W.Workload("sym", (n, n, n), W.homogeneous(1.0), 1.0, 0.5,
                    [(20, 20, 20, W.ricker(1 / 8, 0.5))], 45)
    g = tcm.Sim.from_workload(wl)
    g.step(45)
    a = g.read_field(0)
    assert np.abs(a).max() > 0
    # x reflection exact (xm + xp is the first sum); the others to rounding
    assert np.array_equal(a, a[:, :, ::-1])
    for t in (a[::-1], a[:, ::-1], a.transpose(0, 2, 1)):
        assert np.abs(a - t).max() <= 1e-5 * np.abs(a).max()


def test_empty_simulation():
    wl = W.Workload("empty", (16, 24, 8), W.homogeneous(1.0), 1.0, 0.5, [], 5)
    g = tcm.Sim.from_workload(wl)
    g.step(5)
    assert g.active_count() == (0, 0)
    assert np.all(g.read_field(0) == 0)
    assert g.updates == 0


def test_causality_window_reads():
    """Windows that leave the domain read zeros there; the cone of a source
    ends at L1 distance n-1."""
    shape = (30, 31, 32)
    wl = W.Workload("cone", shape, W.homogeneous(1.0), 1.0, 0.5,
                    [(3, 29, 15, W.ricker(1 / 8, 0.5))], 9)
    g = tcm.Sim.from_workload(wl)
    g.step(9)
    win = g.read_field(0, origin=(-4, 20, 10), size=(12, 16, 12))
    assert np.all(win[:, :, :4] == 0) and np.all(win[:, 11:, :] == 0)
    full = g.read_field(0)
    zz, yy, xx = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
    dist = np.abs(xx - 3) + np.abs(yy - 29) + np.abs(zz - 15)
    assert np.all(full[dist > 8] == 0) and np.any(full[dist == 8] != 0)
    expect = np.zeros_like(win)
    expect[:, :11, 4:] = full[10:22, 20:31, 0:8]
    assert np.array_equal(win, expect)


def test_layered_512_first_steps_full_size():
    """The 512^3 layered, perturbed medium at full size in the benchmarked
    launch configuration: the first 160 steps (relative threshold 1e-6,
    20-step decay) against the oracle, on the window the wave occupies."""
    wl = W.layered(steps=160)
    g, o = pair(wl, pool_bytes=2 * 1024 ** 3)
    g.step(160)
    o.step(160)
    ids = o.active_bricks()
    assert np.array_equal(g.active_bricks(), ids)
    assert len(ids) > 8
    bx = ids % 64
    by = (ids // 64) % 64
    bz = ids // 4096
    lo = [int(v.min()) * 8 for v in (bx, by, bz)]
    hi = [int(v.max()) * 8 + 8 for v in (bx, by, bz)]
    assert_same(g, o, window=(lo, [h - l for h, l in zip(hi, lo)]))
    assert g.updates == o.updates


def test_virtual_4096_until_the_sphere():
    """The virtual 4096^3 domain (never allocated densely): the sphere-
    inclusion burst against the oracle (all host cores) at steps 120, 300 and
    800.  By step 800 the shell has reached the c = 1.8 sphere, so bulked
    bricks (per-node k on the sphere's surface) are boxed and compared; the
    fields are compared over the bounding box of the active bricks, in
    z-slabs."""
    import os
    oracle.set_threads(os.cpu_count() or 1)
    wl = W.virtual(steps=800, pool_bytes=8 * 1024 ** 3)
    g, o = pair(wl, pool_bytes=8 * 1024 ** 3)
    m = 512
    done = 0
    for cp in (120, 300, 800):
        g.step(cp - done)
        o.step(cp - done)
        done = cp
        ids = o.active_bricks()
        assert np.array_equal(g.active_bricks(), ids), cp
        bx, by, bz = ids % m, (ids // m) % m, ids // (m * m)
        lo = [int(v.min()) * 8 for v in (bx, by, bz)]
        hi = [int(v.max()) * 8 + 8 for v in (bx, by, bz)]
        for z0 in range(lo[2], hi[2], 64):
            dz = min(64, hi[2] - z0)
            kw = {"origin": (lo[0], lo[1], z0), "size": (hi[0] - lo[0], hi[1] - lo[1], dz)}
            for which in (0, 1):
                assert np.array_equal(g.read_field(which, **kw), o.read_field(which, **kw)), (cp, z0, which)
    assert g.updates == o.updates
    # bulked (heterogeneous) bricks took part
    sample = ids[:: max(1, len(ids) // 4000)]
    assert sum(1 for b in sample if g.brick_media(int(b))[0] == 2) > 0
    g.close()
    o.close()


@pytest.mark.parametrize("prefetch", [True, False])
def test_l2_prefetch_on_and_off_match_oracle(prefetch):
    """The L2 prefetch of the time stepping is a hint: with it on or off the
    fields and active sets equal the oracle's (relative threshold, decay,
    releases and claims on a ragged grid)."""
    shape = (40, 48, 56)
    media = W.random_dense_media(shape, 5, 1.0, 1.8)
    dt = 0.5 / media.c_max()
    wl = W.Workload("pf", shape, media, 1.0, dt, [(20, 24, 10, W.ricker(1 / 8, dt))], 150,
                    thr_mode=tcm.TCM_THR_RELATIVE, tau=1e-4, decay_alpha=0.8, decay_steps=5, prefetch=prefetch)
    g, o = pair(wl)
    for _ in range(3):
        g.step(50)
        o.step(50)
        assert_same(g, o)
    assert g.updates == o.updates


def test_layered_512_whole_benchmarked_run():
    """The benchmarked run itself: the 512^3 layered workload over all 1500
    steps (relative threshold 1e-6, 20-step decay, pool for every brick,
    steps in one call as the bench issues them) against the oracle run on
    all host cores; the final fields over the whole domain, the active set
    and the node-update count agree exactly."""
    import os
    wl = W.layered(steps=1500)
    pool = (512 // 8) ** 3 * tcm.tcm_slot_bytes(wl.brick)
    g, o = pair(wl, pool_bytes=pool)
    used = oracle.set_threads(os.cpu_count() or 1)
    assert used >= 1
    g.step(5)
    g.step(1495)
    o.step(1500)
    assert g.updates == o.updates
    assert np.array_equal(g.active_bricks(), o.active_bricks())
    for which in (0, 1):
        a, b = g.read_field(which), o.read_field(which)
        assert np.array_equal(a, b), f"half {which}: max |d| = {float(np.max(np.abs(a - b)))}"
    g.close()


def test_page_locked_host_buffers_equal_pageable():
    """A dense velocity model in page-locked host memory is read in place by
    the bulking kernels, and a page-locked destination is written directly by
    the field gather: the results equal those through pageable buffers (and
    the oracle's) bit for bit."""
    import torch
    shape = (36, 28, 44)
    media = W.random_dense_media(shape, 17, 1.0, 2.5)
    dt = 0.5 / media.c_max()
    pinned_c = torch.empty(shape, dtype=torch.float32, pin_memory=True)
    pinned_c.numpy()[...] = media.c
    src = [(12, 14, 20, W.ricker(1 / 8, dt))]
    runs = []
    for c in (media.c.copy(), pinned_c.numpy()):
        wl = W.Workload("pin", shape, W.dense_media(c), 1.0, dt, src, 60)
        s = tcm.Sim.from_workload(wl)
        s.step(60)
        pinned_out = torch.empty(shape, dtype=torch.float32, pin_memory=True)
        nz, ny, nx = shape
        rc = tcm.lib().tcm_read_field(s.handle, 0, 0, 0, 0, nx, ny, nz, tcm.C.c_void_p(pinned_out.data_ptr()))
        assert rc == 0
        runs.append((s.read_field(0), pinned_out.numpy().copy()))
        s.close()
    assert np.array_equal(runs[0][0], runs[1][0])          # pinned model == pageable model
    assert np.array_equal(runs[0][0], runs[0][1])          # pinned destination == pageable destination
    assert np.array_equal(runs[1][0], runs[1][1])
    g, o = pair(W.Workload("pin", shape, media, 1.0, dt, src, 60))
    o.step(60)
    assert np.array_equal(runs[1][0], o.read_field(0))
    g.close()
