"""Pins of the oracle's update schedule: the procedure run every `interval`
steps (Eq. 5) with activation of all 26 neighbours of a triggered cell
(steps 4-5 of the update, Fig. 3).

Facts that fix it: the discrete light cone of Eq. 3 grows by one node per
step along each axis, so between two runs of the procedure (interval <= the
cell edge) a wave can leave a cell only into its 26 neighbours; at threshold
0 the TCM must then equal the dense grid bit for bit, and with an interval
longer than the cell edge it must not.  At thresholds above 0 the schedule
is restated on dense arrays (masks) step by step.
"""
import numpy as np
import pytest
from scipy import ndimage

import oracle
from paper_1702_00216_gb300 import workloads as W

F32 = np.float32


def dense_of(shape, media, dt, sources, steps):
    k = oracle.k_from_c(oracle.rules_c(shape, media) if media.kind == "rules" else media.c, dt, 1.0, F32)
    z = np.zeros(shape, F32)
    return oracle.dense_run(k, z, z, steps, sources=[(x, y, zz, np.asarray(w, F32), st)
                                                     for x, y, zz, w, st in sources])


def tcm_of(shape, media, dt, sources, steps, brick=(8, 8, 8), **kw):
    t = oracle.OracleTCM(shape, media, 1.0, dt, brick=brick, **kw)
    pending = sorted(sources, key=lambda s: s[4])
    done = 0
    for x, y, z, w, st in pending:
        t.step(st - done)
        done = st
        t.add_source(x, y, z, np.asarray(w, F32))
    t.step(steps - done)
    return t


@pytest.mark.parametrize("interval", [1, 2, 5, 8])
def test_interval_26_threshold0_equals_dense(interval):
    shape = (27, 33, 38)
    m = W.random_dense_media(shape, 4, 1.0, 2.0)
    dt = 0.5 / m.c_max()
    w = W.ricker(1 / 8, dt)
    srcs = [(5, 30, 3, w, 0), (35, 2, 25, w[:25], 7)]
    steps = 70
    a, b = dense_of(shape, m, dt, srcs, steps)
    t = tcm_of(shape, m, dt, srcs, steps, interval=interval, neighbours=26)
    assert np.array_equal(t.read_field(0), a) and np.array_equal(t.read_field(1), b)
    early = tcm_of(shape, m, dt, srcs[:1], 12, interval=interval, neighbours=26)
    assert 0 < early.active_count()[0] < early.mx * early.my * early.mz


def test_interval_beyond_cell_edge_loses_the_front():
    # one node per step along an axis: 9 steps from a cell's far face reach
    # past its 26 neighbours, so the front is cut and TCM != dense
    # (the front is at x = 20 + n after step n; after the run at n = 35 it
    # sits on the last node of a cell, and 9 more steps cross two cells)
    shape = (40, 40, 96)
    m = W.homogeneous(1.0)
    dt = 0.5
    w = W.ricker(1 / 8, dt)
    srcs = [(20, 20, 20, w, 0)]
    a, _ = dense_of(shape, m, dt, srcs, 50)
    t9 = tcm_of(shape, m, dt, srcs, 50, interval=9, neighbours=26)
    t8 = tcm_of(shape, m, dt, srcs, 50, interval=8, neighbours=26)
    assert np.array_equal(t8.read_field(0), a)
    assert not np.array_equal(t9.read_field(0), a)
    # with face activation only, interval 2 loses part of the spread
    t2f = tcm_of(shape, m, dt, srcs, 50, interval=2, neighbours=6)
    assert not np.array_equal(t2f.read_field(0), a)


@pytest.mark.parametrize("interval", [2, 4])
def test_interval_26_brute_force_every_source_node(interval):
    # every source node of a 3x2x2-cell grid of 4^3 cells, threshold 0
    shape = (8, 8, 12)
    m = W.homogeneous(1.0)
    dt = 0.5
    w = W.ricker(1 / 4, dt)[:12]
    for z in range(0, 8, 3):
        for y in range(0, 8, 3):
            for x in range(12):
                srcs = [(x, y, z, w, 0)]
                a, b = dense_of(shape, m, dt, srcs, 18)
                t = tcm_of(shape, m, dt, srcs, 18, brick=(4, 4, 4), interval=interval, neighbours=26)
                assert np.array_equal(t.read_field(0), a), (x, y, z)
                assert np.array_equal(t.read_field(1), b), (x, y, z)


def test_schedule_arguments():
    with pytest.raises(ValueError):
        oracle.OracleTCM((8, 8, 8), W.homogeneous(1.0), 1.0, 0.5, interval=0, neighbours=26)
    with pytest.raises(ValueError):
        oracle.OracleTCM((8, 8, 8), W.homogeneous(1.0), 1.0, 0.5, interval=2, neighbours=18)


def _eq3(a, b, k):
    p = np.pad(a, 1)
    s = ((((p[1:-1, 1:-1, :-2] + p[1:-1, 1:-1, 2:]) + p[1:-1, :-2, 1:-1]) + p[1:-1, 2:, 1:-1]) +
         p[:-2, 1:-1, 1:-1]) + p[2:, 1:-1, 1:-1]
    return (F32(2) * a - b) + k * (s - F32(6) * a)


def _cells(ids, m):
    mx, my, mz = m
    c = np.zeros(mx * my * mz, bool)
    c[np.asarray(ids, dtype=np.int64)] = True
    return c.reshape(mz, my, mx)


def _nodes(cells, shape, brick):
    bx, by, bz = brick
    return cells.repeat(bz, 0).repeat(by, 1).repeat(bx, 2)[:shape[0], :shape[1], :shape[2]]


def _cellmax(v, m, brick):
    bx, by, bz = brick
    mx, my, mz = m
    p = np.zeros((mz * bz, my * by, mx * bx), v.dtype)
    p[:v.shape[0], :v.shape[1], :v.shape[2]] = v
    return p.reshape(mz, bz, my, by, mx, bx).max(axis=(1, 3, 5))


@pytest.mark.parametrize("interval,mode,tau", [(3, oracle.THR_ABSOLUTE, 3e-2),
                                               (5, oracle.THR_RELATIVE, 0.35)])
def test_interval_26_restated_on_masks(interval, mode, tau):
    """No decay: between runs the boxed set stays and Eq. 3 runs on it; a run
    after step n calls a boxed cell triggered when its maximum is above the
    level or a source feeds it in n+1..n+interval; it keeps the triggered
    cells and their boxed 26-neighbours and boxes the rest of their 26
    neighbours (and unboxed source cells still to be fed)."""
    shape = (30, 26, 36)
    brick = (6, 6, 6)
    dt = 0.5
    w = W.ricker(1 / 7, dt).astype(F32)
    src = (17, 12, 14)
    k = oracle.k_from_c(np.ones(shape, F32), dt, 1.0, F32)
    t = oracle.OracleTCM(shape, W.homogeneous(1.0), 1.0, dt, brick=brick, thr_mode=mode, tau=tau,
                         interval=interval, neighbours=26)
    t.add_source(*src, w)
    m = (t.mx, t.my, t.mz)
    s3 = np.ones((3, 3, 3), bool)
    released = False
    for n in range(80):
        A = _cells(t.active_bricks(), m)
        a, b = t.read_field(0), t.read_field(1)
        t.step(1)
        A1 = _cells(t.active_bricks(), m)
        q = _eq3(a, b, k)
        if n < len(w):
            q[src[2], src[1], src[0]] += w[n]
        q = np.where(_nodes(A, shape, brick), q, F32(0))
        if (n + 1) % interval:
            assert np.array_equal(A1, A), n
        else:
            thr = tau * float(np.abs(q).max()) if mode == oracle.THR_RELATIVE else tau
            mc = np.maximum(_cellmax(np.abs(q), m, brick), _cellmax(np.abs(a), m, brick))
            forced = np.zeros_like(A)
            if any(n + 1 <= j < len(w) for j in range(n + 1, n + 1 + interval)):
                forced[src[2] // 6, src[1] // 6, src[0] // 6] = True
            hot = A & ((mc.astype(np.float64) > thr) | forced)
            near = ndimage.binary_dilation(hot, structure=s3)
            expect = (A & (near | forced)) | (~A & (near | forced))
            released |= bool(np.any(A & ~expect))
            assert np.array_equal(A1, expect), n
        nm = _nodes(A1, shape, brick)
        assert np.array_equal(t.read_field(0), np.where(nm, q, F32(0))), n
        assert np.array_equal(t.read_field(1), np.where(nm, a, F32(0))), n
    assert released, "scenario must release cells"


@pytest.mark.parametrize("interval,neighbours", [(1, 6), (4, 26)])
def test_initial_field_on_cell_faces_threshold0_equals_dense(interval, neighbours):
    # initial values on the faces, edges and corners of one cell: the update
    # procedure run on the initial state boxes the cells they spread into
    shape = (24, 24, 24)
    m = W.homogeneous(1.0)
    dt = 0.5
    now = np.zeros(shape, F32)
    prev = np.zeros(shape, F32)
    now[8, 8:16, 8:16] = 1.0          # z- face of cell (1,1,1)
    now[8:16, 15, 15] = -0.5          # an x+/y+ edge
    prev[15, 15, 15] = 0.25           # a corner, phi^{-1} only
    k = oracle.k_from_c(np.ones(shape, F32), dt, 1.0, F32)
    a, b = oracle.dense_run(k, now, prev, 12)
    t = oracle.OracleTCM(shape, m, 1.0, dt, interval=interval, neighbours=neighbours)
    t.set_field(now, prev)
    t.step(12)
    assert np.array_equal(t.read_field(0), a) and np.array_equal(t.read_field(1), b)
