"""Pins of the CPU oracle to facts the paper and the mathematics fix.

Nothing here compares the oracle with itself: every check is a closed form
(the Dirichlet eigenmode recursion of Eq. 3, the leapfrog energy, the CFL
bound of Eq. 4 on a finite grid, lattice-point counts), an invariant
(causality, mirror symmetry, energy conservation), or an identity between the
two oracle programs that the method guarantees (the TCM at threshold 0 skips
only nodes that hold no wave, so it equals the dense grid bit for bit), plus a
dense-array restatement of the box bookkeeping at thresholds above 0.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1702_00216_gb300 import workloads as W

F32, F64 = np.float32, np.float64


def homog_k(shape, courant, dtype):
    """k = (c dt/dx)^2 with c = 1, dx = 1, dt = courant."""
    return oracle.k_from_c(np.ones(shape, np.float32), courant, 1.0, dtype)


def mode_sum(shape, p):
    nz, ny, nx = shape
    return sum(math.sin(math.pi * pd / (2 * (nd + 1))) ** 2 for pd, nd in zip(p, (nx, ny, nz)))


# ---------------------------------------------------------------- coefficient
@pytest.mark.parametrize("dtype", [F32, F64])
def test_k_exact_values(dtype):
    # (c dt / dx)^2 for exactly representable quotients (Eq. 3 coefficient)
    c = np.array([1.0, 3.0, 2.0, 0.0], np.float32)
    k = oracle.k_from_c(c, 0.5, 1.5, dtype)
    assert k.tolist() == [1.0 / 9.0 if dtype == F64 else float(np.float32(1.0 / 9.0)), 1.0,
                          float(dtype(4.0 / 9.0)), 0.0]
    assert oracle.k_from_c(np.array([1.0], np.float32), 0.5, 1.0, dtype)[0] == 0.25


# ---------------------------------------------------------------- dispersion
@pytest.mark.parametrize("shape,p", [((11, 9, 7), (1, 2, 3)), ((6, 10, 8), (5, 1, 4))])
def test_dispersion_eigenmode_f64(shape, p):
    """Eq. 3 on a Dirichlet eigenmode: phi^n = cos(n theta) v exactly, with
    sin^2(theta/2) = C^2 sum_d sin^2(pi p_d / (2(N_d+1))).  A dropped or
    mis-signed term, a wrong coefficient or a transposed axis breaks it."""
    C = 0.5
    k = homog_k(shape, C, F64)
    v = W.eigenmode(shape, p)
    theta = 2.0 * math.asin(C * math.sqrt(mode_sum(shape, p)))
    steps = 300
    a, b = oracle.dense_run(k, v, math.cos(theta) * v, steps)
    assert np.max(np.abs(a - math.cos(steps * theta) * v)) < 1e-11
    assert np.max(np.abs(b - math.cos((steps - 1) * theta) * v)) < 1e-11


def test_dispersion_eigenmode_f32():
    shape, p, C = (11, 9, 7), (2, 1, 3), 0.5
    k = homog_k(shape, C, F32)
    v = W.eigenmode(shape, p)
    theta = 2.0 * math.asin(C * math.sqrt(mode_sum(shape, p)))
    a, _ = oracle.dense_run(k, v.astype(F32), (math.cos(theta) * v).astype(F32), 200)
    assert np.max(np.abs(a - math.cos(200 * theta) * v)) < 5e-5


def test_dispersion_detects_transposed_axes():
    """The same mode on the transposed grid does not satisfy the relation:
    the check above really distinguishes the axes."""
    shape, p, C = (11, 9, 7), (1, 2, 3), 0.5
    v = W.eigenmode(shape, p)
    theta_wrong = 2.0 * math.asin(C * math.sqrt(mode_sum(shape, p[::-1])))
    a, _ = oracle.dense_run(homog_k(shape, C, F64), v, math.cos(theta_wrong) * v, 300)
    assert np.max(np.abs(a - math.cos(300 * theta_wrong) * v)) > 1e-3


# ---------------------------------------------------------------- energy
def test_energy_closed_form_for_a_mode():
    """E(a v, b v) = |v|^2 [ (a-b)^2 / k + 4 S a b ] for an eigenvector v."""
    shape, p, C = (7, 8, 9), (2, 3, 1), 0.5
    k = homog_k(shape, C, F64)
    v = W.eigenmode(shape, p)
    S = mode_sum(shape, p)
    for a, b in [(1.0, 0.5), (-0.3, 0.7), (0.0, 1.0)]:
        expect = float(np.sum(v * v)) * ((a - b) ** 2 / (C * C) + 4.0 * S * a * b)
        assert oracle.energy(k, a * v, b * v) == pytest.approx(expect, rel=1e-13)


def test_energy_conserved_heterogeneous_f64():
    """Leapfrog energy is invariant for any symmetric K and positive k."""
    rng = np.random.default_rng(5)
    shape = (10, 12, 14)
    c = rng.uniform(1.0, 2.0, shape).astype(np.float32)
    k = oracle.k_from_c(c, 0.5 / float(c.max()), 1.0, F64)
    a, b = rng.standard_normal(shape), rng.standard_normal(shape)
    E = []
    for _ in range(8):
        E.append(oracle.energy(k, a, b))
        a, b = oracle.dense_run(k, a, b, 60)
    E = np.array(E)
    assert E[0] > 0
    assert np.max(np.abs(E - E[0])) / E[0] < 1e-12


def test_energy_constant_after_source_stops():
    rng = np.random.default_rng(11)
    shape = (24, 20, 22)
    c = rng.uniform(1.0, 1.5, shape).astype(np.float32)
    dt = 0.5 / float(c.max())
    k = oracle.k_from_c(c, dt, 1.0, F64)
    w = W.ricker(1.0 / 8.0, dt)
    z = np.zeros(shape)
    a, b = oracle.dense_run(k, z, z, len(w), sources=[(10, 9, 12, w)])
    E0 = oracle.energy(k, *oracle.dense_run(k, a, b, 1))
    a, b = oracle.dense_run(k, a, b, 200, step0=len(w))
    E1 = oracle.energy(k, a, b)
    assert E0 > 0 and abs(E1 - E0) / E0 < 1e-12


# ---------------------------------------------------------------- CFL (Eq. 4)
@pytest.mark.parametrize("C,unstable", [(0.5, False), (0.58, False), (0.59, True), (0.6, True)])
def test_cfl_bound_finite_grid(C, unstable):
    """Eq. 4: stable iff C^2 * S_max <= 1.  On a 10^3 Dirichlet grid
    S_max = 3 sin^2(10 pi / 22), so the bound is C <= 0.5833 (1/sqrt(3) as
    N -> infinity)."""
    n = 10
    smax = 3 * math.sin(10 * math.pi / 22) ** 2
    assert (C * C * smax > 1.0) == unstable
    rng = np.random.default_rng(3)
    v = rng.uniform(-1, 1, (n, n, n))
    a, _ = oracle.dense_run(homog_k((n, n, n), C, F64), v, v, 300)
    growth = np.max(np.abs(a)) / np.max(np.abs(v))
    if unstable:
        assert growth > 1e6
    else:
        assert growth < 50


# ---------------------------------------------------------------- causality
@pytest.mark.parametrize("dtype", [F32, F64])
def test_causality_l1_ball(dtype):
    """A source first inserted into phi^1 reaches L1 distance n-1 by phi^n and
    no further (7-point stencil, one cell per step)."""
    rng = np.random.default_rng(7)
    shape = (20, 22, 24)
    c = rng.uniform(1.0, 2.0, shape).astype(np.float32)
    dt = 0.5 / float(c.max())
    k = oracle.k_from_c(c, dt, 1.0, dtype)
    w = W.ricker(1.0 / 8.0, dt).astype(dtype)
    x, y, z = 5, 9, 13
    zz, yy, xx = np.meshgrid(np.arange(20), np.arange(22), np.arange(24), indexing="ij")
    dist = np.abs(xx - x) + np.abs(yy - y) + np.abs(zz - z)
    zero = np.zeros(shape, dtype)
    for n in (1, 4, 9):
        a, _ = oracle.dense_run(k, zero, zero, n, sources=[(x, y, z, w)])
        assert np.all(a[dist > n - 1] == 0)
        assert np.all(a[(dist == n - 1) & (xx == x) & (yy == y)] != 0)
        tcm = oracle.OracleTCM(shape, W.dense_media(c), 1.0, dt, dtype=dtype)
        tcm.add_source(x, y, z, w)
        tcm.step(n)
        assert np.array_equal(tcm.read_field(0), a)


# ---------------------------------------------------------------- symmetry
@pytest.mark.parametrize("dtype", [F32, F64])
def test_mirror_symmetry_centred_source(dtype):
    """Centred source, homogeneous odd grid: the field is invariant under the
    x reflection bit for bit (the sum starts with xm + xp, which commutes),
    and under the y and z reflections and the axis exchanges to rounding
    (the left-to-right sum ((((xm+xp)+ym)+yp)+zm)+zp adds ym before yp)."""
    n, steps = 33, 40
    shape = (n, n, n)
    k = homog_k(shape, 0.5, dtype)
    w = W.ricker(1.0 / 8.0, 0.5).astype(dtype)
    zero = np.zeros(shape, dtype)
    a, _ = oracle.dense_run(k, zero, zero, steps, sources=[(16, 16, 16, w)])
    assert np.abs(a).max() > 0
    assert np.array_equal(a, a[:, :, ::-1])
    tol = 1e-5 if dtype == F32 else 1e-13
    for b in (a[::-1, :, :], a[:, ::-1, :], a.transpose(0, 2, 1), a.transpose(2, 1, 0)):
        assert np.max(np.abs(a - b)) <= tol * np.abs(a).max()
    # an indexing slip (a shifted halo) breaks the symmetry far above rounding
    off = oracle.dense_run(k, zero, zero, steps, sources=[(16, 16, 15, w)])[0]
    assert np.max(np.abs(off - off[::-1, :, :])) > 1e-2 * np.abs(off).max()
    # the TCM (8^3 cells; 33 = 4*8 + 1 leaves a ragged last cell) keeps it
    tcm = oracle.OracleTCM(shape, W.homogeneous(1.0), 1.0, 0.5, dtype=dtype)
    tcm.add_source(16, 16, 16, w)
    tcm.step(steps)
    assert np.array_equal(tcm.read_field(0), a)


# ---------------------------------------------------------------- TCM == dense at threshold 0
def _dense_reference(shape, media, dt, sources, steps, dtype, checkpoints):
    c = media.c if media.kind == "dense" else oracle.rules_c(shape, media)
    k = oracle.k_from_c(c, dt, 1.0, dtype)
    a = np.zeros(shape, dtype)
    b = np.zeros(shape, dtype)
    out, done = {}, 0
    for cp in checkpoints:
        a, b = oracle.dense_run(k, a, b, cp - done, sources=sources, step0=done)
        done = cp
        out[cp] = (a.copy(), b.copy())
    return out


@pytest.mark.parametrize("dtype", [F32, F64])
def test_tcm_threshold0_equals_dense_small_config(dtype):
    """64^3, c = 1, Courant 0.5, Ricker at the centre, 100 steps, 8^3 cells."""
    wl = W.small()
    src = [(x, y, z, w.astype(dtype)) for x, y, z, w in wl.sources]
    cps = [1, 17, 50, 100]
    ref = _dense_reference(wl.shape, wl.media, wl.dt, src, wl.steps, dtype, cps)
    tcm = oracle.OracleTCM(wl.shape, wl.media, wl.dx, wl.dt, brick=wl.brick, dtype=dtype)
    for x, y, z, w in src:
        tcm.add_source(x, y, z, w)
    done, seen = 0, []
    for cp in cps:
        tcm.step(cp - done)
        done = cp
        assert np.array_equal(tcm.read_field(0), ref[cp][0])
        assert np.array_equal(tcm.read_field(1), ref[cp][1])
        seen.append(tcm.active_count()[0])
    # at threshold 0 the boxed region is the numerical light cone (L1 radius n):
    # the source node (32,32,32) is the low corner of cell (4,4,4), so its three
    # low faces trigger three neighbours after the first step; the whole
    # 8^3-cell grid is boxed once the cone reaches the faces
    assert seen[0] == 4 and seen[0] < seen[1] < seen[2] and seen[-1] == 512


@pytest.mark.parametrize("brick", [(8, 8, 8), (16, 8, 8), (4, 4, 4), (5, 3, 7)])
def test_tcm_threshold0_equals_dense_heterogeneous_ragged(brick):
    """Random per-node media (every cell bulked), three sources, a domain that
    is not a multiple of the cell size."""
    rng = np.random.default_rng(1702)
    shape = (21, 29, 37)
    media = W.random_dense_media(shape, 99, 1.0, 2.0)
    dt = 0.5 / media.c_max()
    srcs = [(3, 4, 5, W.ricker(1 / 8, dt).astype(F32)),
            (36, 28, 20, W.ricker(1 / 10, dt).astype(F32)),
            (int(rng.integers(37)), int(rng.integers(29)), int(rng.integers(21)),
             W.ricker(1 / 6, dt).astype(F32))]
    steps = 60
    ref = _dense_reference(shape, media, dt, srcs, steps, F32, [steps])
    tcm = oracle.OracleTCM(shape, media, 1.0, dt, brick=brick)
    for s in srcs:
        tcm.add_source(*s)
    tcm.step(steps)
    assert np.array_equal(tcm.read_field(0), ref[steps][0])
    assert np.array_equal(tcm.read_field(1), ref[steps][1])


def test_tcm_threshold0_equals_dense_layered_rules():
    """Rules media whose layer boundaries cut some cells: homogenic and bulked
    cells side by side (Heterogenic Bulking leaves the results unchanged)."""
    shape = (40, 24, 24)
    media = W.Media(kind="rules", c_background=1.0, layers=[(12.0, 1.5), (29.5, 2.0)],
                    spheres=[(11.0, 12.0, 20.0, 5.5, 0.7)])
    dt = 0.5 / media.c_max()
    src = [(12, 12, 18, W.ricker(1 / 8, dt).astype(F32))]
    ref = _dense_reference(shape, media, dt, src, 70, F32, [70])
    tcm = oracle.OracleTCM(shape, media, 1.0, dt)
    tcm.add_source(*src[0])
    tcm.step(70)
    assert np.array_equal(tcm.read_field(0), ref[70][0])
    kinds = {tcm.brick_media(b)[0] for b in range(tcm.mx * tcm.my * tcm.mz)}
    assert kinds == {1, 2}


def test_tcm_brute_force_every_source_position():
    """Every source node of a 3 x 2 x 1 cell grid (4^3 cells), 12 steps each."""
    shape = (4, 8, 12)
    dt = 0.5
    w = W.ricker(1 / 4, dt, t0=1.0).astype(F32)
    k = homog_k(shape, dt, F32)
    zero = np.zeros(shape, F32)
    for z in range(shape[0]):
        for y in range(shape[1]):
            for x in range(shape[2]):
                a, b = oracle.dense_run(k, zero, zero, 12, sources=[(x, y, z, w)])
                tcm = oracle.OracleTCM(shape, W.homogeneous(1.0), 1.0, dt, brick=(4, 4, 4))
                tcm.add_source(x, y, z, w)
                tcm.step(12)
                assert np.array_equal(tcm.read_field(0), a), (x, y, z)
                assert np.array_equal(tcm.read_field(1), b), (x, y, z)


def test_tcm_set_field_matches_dense():
    """Initial fields instead of a source: only cells holding values are boxed."""
    shape = (24, 16, 16)
    v = np.zeros(shape, F32)
    v[10:14, 6:9, 5:9] = np.random.default_rng(1).uniform(-1, 1, (4, 3, 4)).astype(F32)
    k = homog_k(shape, 0.5, F32)
    a, b = oracle.dense_run(k, v, v, 25)
    tcm = oracle.OracleTCM(shape, W.homogeneous(1.0), 1.0, 0.5)
    tcm.set_field(v, v)
    assert tcm.active_count()[0] == 4   # z cell 1; y and x each straddle cells 0|1
    tcm.step(25)
    assert np.array_equal(tcm.read_field(0), a) and np.array_equal(tcm.read_field(1), b)


def test_oracle_thread_count_does_not_change_results():
    def run():
        tcm = oracle.OracleTCM((24, 24, 24), W.homogeneous(1.0), 1.0, 0.5, thr_mode=1, tau=1e-3,
                               decay_alpha=0.9, decay_steps=3)
        tcm.add_source(12, 12, 12, W.ricker(1 / 8, 0.5).astype(F32))
        tcm.step(40)
        return tcm.read_field(0), tcm.active_bricks()
    try:
        oracle.set_threads(1)
        f1, a1 = run()
        oracle.set_threads(4)
        f4, a4 = run()
    finally:
        oracle.set_threads(1)
    assert np.array_equal(f1, f4) and np.array_equal(a1, a4)


# ---------------------------------------------------------------- thresholds above 0
def _eq3_numpy(a, b, k):
    """Eq. 3 with the oracle's grouping, on dense float32 arrays (zero ghosts)."""
    p = np.pad(a, 1)
    xm, xp = p[1:-1, 1:-1, :-2], p[1:-1, 1:-1, 2:]
    ym, yp = p[1:-1, :-2, 1:-1], p[1:-1, 2:, 1:-1]
    zm, zp = p[:-2, 1:-1, 1:-1], p[2:, 1:-1, 1:-1]
    s = ((((xm + xp) + ym) + yp) + zm) + zp
    lap = s - a.dtype.type(6) * a
    return (a.dtype.type(2) * a - b) + k * lap


def _cell_mask(ids, shape, brick, m):
    nz, ny, nx = shape
    bx, by, bz = brick
    mx, my, mz = m
    cm = np.zeros(mx * my * mz, bool)
    cm[np.asarray(ids, dtype=np.int64)] = True
    cm = cm.reshape(mz, my, mx)
    full = cm.repeat(bz, 0).repeat(by, 1).repeat(bx, 2)
    return full[:nz, :ny, :nx]


def _cell_max(arr, brick, m):
    bx, by, bz = brick
    mx, my, mz = m
    pad = np.zeros((mz * bz, my * by, mx * bx), arr.dtype)
    pad[:arr.shape[0], :arr.shape[1], :arr.shape[2]] = arr
    return pad.reshape(mz, bz, my, by, mx, bx), pad


@pytest.mark.parametrize("mode,tau,reuse", [(oracle.THR_ABSOLUTE, 3e-2, True),
                                            (oracle.THR_RELATIVE, 0.3, False)])
def test_tcm_box_bookkeeping_matches_masked_dense(mode, tau, reuse):
    """With no decay, one step of the TCM is: Eq. 3 on the boxed cells, then
    the cells chosen by the update procedure keep their values and all others
    hold zero.  Restated here on dense arrays (masks), step by step, from the
    oracle's own previous state: it pins Cell2box/Box2cell, box reuse and
    re-initialisation, the halo padding and the triggering rule."""
    shape = (32, 24, 40)
    brick = (8, 8, 8)
    dt = 0.5
    w = W.ricker(1 / 8, dt).astype(F32)
    src = (9, 11, 14)
    k = homog_k(shape, dt, F32)
    tcm = oracle.OracleTCM(shape, W.homogeneous(1.0), 1.0, dt, brick=brick, thr_mode=mode, tau=tau)
    tcm.add_source(*src, w)
    m = (tcm.mx, tcm.my, tcm.mz)
    ever, peak, retired_any = set(), 0, False
    for n in range(90):
        A = tcm.active_bricks()
        a, b = tcm.read_field(0), tcm.read_field(1)
        tcm.step(1)
        A1 = tcm.active_bricks()
        a1, b1 = tcm.read_field(0), tcm.read_field(1)
        mA, mA1 = _cell_mask(A, shape, brick, m), _cell_mask(A1, shape, brick, m)
        q = _eq3_numpy(a, b, k)
        if n < len(w):
            q[src[2], src[1], src[0]] = q[src[2], src[1], src[0]] + w[n]
        q = np.where(mA, q, F32(0))
        assert np.array_equal(a1, np.where(mA1, q, F32(0)))
        assert np.array_equal(b1, np.where(mA1, a, F32(0)))
        # the update procedure on cell maxima
        G = float(np.max(np.abs(q)))
        thr = tau * G if mode == oracle.THR_RELATIVE else tau
        qc, _ = _cell_max(np.abs(q), brick, m)
        ac, _ = _cell_max(np.abs(a), brick, m)
        mcell = np.maximum(qc.max(axis=(1, 3, 5)), ac.max(axis=(1, 3, 5)))
        faces = {  # face maxima per cell, same (mz, my, mx) layout
            (0, -1): qc[:, :, :, :, :, 0].max(axis=(1, 3)), (0, 1): qc[:, :, :, :, :, -1].max(axis=(1, 3)),
            (1, -1): qc[:, :, :, 0, :, :].max(axis=(1, 4)), (1, 1): qc[:, :, :, -1, :, :].max(axis=(1, 4)),
            (2, -1): qc[:, 0, :, :, :, :].max(axis=(2, 4)), (2, 1): qc[:, -1, :, :, :, :].max(axis=(2, 4)),
        }
        act = _cell_mask(A, (m[2], m[1], m[0]), (1, 1, 1), m)
        hot_face_into = np.zeros_like(act)   # cell receives a face above the level
        for (ax, sgn), fm in faces.items():
            hot = (fm.astype(np.float64) > thr) & act
            axis = 2 - ax                     # array axis of x/y/z
            sh = np.roll(hot, sgn, axis=axis)
            sl = [slice(None)] * 3
            sl[axis] = 0 if sgn == 1 else -1
            sh[tuple(sl)] = False
            hot_face_into |= sh
        forced = np.zeros_like(act)
        if n + 1 < len(w):
            forced[src[2] // 8, src[1] // 8, src[0] // 8] = True
        keep = act & ((mcell.astype(np.float64) > thr) | hot_face_into | forced)
        new = ~act & (hot_face_into | forced)
        expect = np.flatnonzero((keep | new).ravel())
        assert np.array_equal(np.sort(A1), expect), n
        retired_any |= bool(np.any(act & ~keep))
        ever |= set(A1.tolist())
        peak = max(peak, len(A1))
    if reuse:
        assert retired_any, "scenario must retire cells"
        assert len(ever) > peak, "scenario must reuse boxes"


def test_tcm_decay_scales_shutdown_cells():
    """Eq. 6: a cell in shut-down is multiplied by alpha each step for n steps,
    total A = alpha^n, then released.  Pin: a lone initial value in one cell
    with an absolute level above it decays by exactly alpha per step (on top
    of Eq. 3) and the cell is gone after decay_steps + 1 updates."""
    shape = (8, 8, 8)
    v = np.zeros(shape, F32)
    v[4, 4, 4] = 1.0
    alpha, D = 0.5, 3
    tcm = oracle.OracleTCM(shape, W.homogeneous(1.0), 1.0, 0.5, tau=10.0, decay_alpha=alpha,
                           decay_steps=D)
    tcm.set_field(v, v)
    k = homog_k(shape, 0.5, F32)
    a, b = v, v
    for n in range(D + 1):
        assert tcm.active_count()[0] == 1
        q = _eq3_numpy(a, b, k)
        if n > 0:
            q = F32(alpha) * q
        tcm.step(1)
        if n < D:
            assert np.array_equal(tcm.read_field(0), q)
        a, b = q, a
    assert tcm.active_count()[0] == 0


def test_tcm_pool_cap_sets_enomem():
    tcm = oracle.OracleTCM((32, 32, 32), W.homogeneous(1.0), 1.0, 0.5, max_slots=3)
    tcm.add_source(16, 16, 16, W.ricker(1 / 8, 0.5).astype(F32))
    tcm.step(40)
    assert tcm.status == -2
    assert tcm.active_count()[0] == 3


# ---------------------------------------------------------------- media rules
def test_sphere_rule_lattice_counts():
    """Nodes with |x - centre|^2 <= r^2 around a node: 1 + 6 (r=1), +12 (r^2=2),
    +8 (r^2=3), +6 (r^2=4)."""
    for r2, count in [(1, 7), (2, 19), (3, 27), (4, 33)]:
        media = W.Media(kind="rules", c_background=1.0,
                        spheres=[(5.0, 5.0, 5.0, math.sqrt(r2) + 1e-9, 2.0)])
        c = oracle.rules_c((11, 11, 11), media)
        assert int(np.sum(c == 2.0)) == count


def test_layer_rule_and_bulking_classification():
    shape = (32, 16, 16)
    media = W.Media(kind="rules", c_background=1.0, layers=[(0.0, 1.25), (12.0, 2.0)])
    c = oracle.rules_c(shape, media)
    assert np.all(c[:12] == np.float32(1.25)) and np.all(c[12:] == 2.0)
    tcm = oracle.OracleTCM(shape, media, 1.0, 0.2)
    # cells along z: [0,8) c=1.25, [8,16) straddles z=12, [16,24), [24,32) c=2
    assert tcm.brick_media(0) == (1, float(np.float32((1.25 * 0.2) ** 2)))
    assert tcm.brick_media(4)[0] == 2 and tcm.brick_media(5)[0] == 2
    assert tcm.brick_media(8) == (1, float(np.float32((2.0 * 0.2) ** 2)))
