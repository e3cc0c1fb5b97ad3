"""Pins of the oracle's update procedure at thresholds above 0.

The paper fixes the procedure in words (Simulation section, "updating active
cells", steps 1-8 with Fig. 3; Shut-down section, Eq. 6; Boxes section,
Fig. 1) and shows its effect only in figures, so there is no printed value to
compare with.  These tests pin the oracle to what the procedure implies,
using nothing but what the oracle exposes -- its boxed cells and its two
field levels before and after every step -- and the dense program for one
step of Eq. 3, which is pinned on its own (eigenmode closed form, energy,
causality, symmetry, CFL; test_oracle_pins.py).  Checked after every step of
randomised runs (media, sources, absolute and relative levels, shut-down
lengths, neighbour sets, update intervals, both precisions):

 I1  a kept cell carries phi^n over unchanged (two-level rotation of Eq. 3);
 I2  a kept cell's phi^{n+1} is one step of Eq. 3 on the field padded by its
     neighbours' boundaries (zero where unboxed), optionally times alpha
     (Time stepping; Eq. 6) -- nothing else changes a value;
 I3  a cell whose maximal |value| is above the level is not released and
     does not shut down (step 3);
 I4  every cell across a face above the level is boxed after the update, and
     does not shut down (step 4, Fig. 3a; with the 26-neighbour set, every
     neighbour of a triggered cell, Fig. 3a-d);
 I5  a boxed cell that is not triggered shuts down: for the next D steps its
     phi^{n+1} is multiplied by alpha, then it is released, so its values are
     attenuated by A = alpha^D in total (steps 6-7, Eq. 6); with D = 0 it is
     released at once; a trigger cancels the shut-down;
 I6  a newly boxed cell starts from zero in both levels (steps 8, Fig. 1),
     and an unboxed cell reads zero;
 I7  a source's cell is boxed while the source still inserts samples
     (Source insertion).

Worked examples pin the readings where a plausible alternative exists:
strict "above" at a level equal to a cell's maximum; the cell maximum taken
over both phi^{n+1} and phi^n (threshold 0 must stay equal to the dense grid
when a cell's phi^{n+1} vanishes while phi^n does not); a cell kept by its
neighbour's touching face keeps its values and does not decay; with an
update interval dividing D the shut-down still lasts exactly D steps.  A
threshold sweep pins convergence: the deviation from the dense grid shrinks
as the level drops and is exactly zero at threshold 0.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1702_00216_gb300 import workloads as W

F32, F64 = np.float32, np.float64


class Cells:
    """Brick geometry on (nz, ny, nx) arrays; brick ids z*my*mx + y*mx + x."""

    def __init__(self, shape, brick):
        self.shape = shape
        nz, ny, nx = shape
        self.bx, self.by, self.bz = brick
        self.mx, self.my, self.mz = -(-nx // self.bx), -(-ny // self.by), -(-nz // self.bz)
        self.n = self.mx * self.my * self.mz
        ids = np.arange(self.n)
        self.cx, self.cy, self.cz = ids % self.mx, (ids // self.mx) % self.my, ids // (self.mx * self.my)

    def blocks(self, a):
        """(n_cells, bz, by, bx) view of a zero-padded copy."""
        p = np.zeros((self.mz * self.bz, self.my * self.by, self.mx * self.bx), a.dtype)
        p[:a.shape[0], :a.shape[1], :a.shape[2]] = a
        p = p.reshape(self.mz, self.bz, self.my, self.by, self.mx, self.bx)
        return p.transpose(0, 2, 4, 1, 3, 5).reshape(self.n, self.bz, self.by, self.bx)

    def unblocks(self, c):
        """Inverse of blocks: (n_cells, bz, by, bx) -> (nz, ny, nx)."""
        p = c.reshape(self.mz, self.my, self.mx, self.bz, self.by, self.bx).transpose(0, 3, 1, 4, 2, 5)
        p = p.reshape(self.mz * self.bz, self.my * self.by, self.mx * self.bx)
        return p[:self.shape[0], :self.shape[1], :self.shape[2]]

    def absmax(self, a):
        return np.abs(self.blocks(a)).reshape(self.n, -1).max(axis=1)

    def face_absmax(self, a):
        """(n_cells, 6): max |value| on the faces x-, x+, y-, y+, z-, z+ (in-domain nodes only:
        the padding is zero)."""
        b = np.abs(self.blocks(a))
        return np.stack([b[:, :, :, 0].reshape(self.n, -1).max(1), b[:, :, :, -1].reshape(self.n, -1).max(1),
                         b[:, :, 0, :].reshape(self.n, -1).max(1), b[:, :, -1, :].reshape(self.n, -1).max(1),
                         b[:, 0, :, :].reshape(self.n, -1).max(1), b[:, -1, :, :].reshape(self.n, -1).max(1)], 1)

    def at(self, cx, cy, cz):
        ok = (cx >= 0) & (cy >= 0) & (cz >= 0) & (cx < self.mx) & (cy < self.my) & (cz < self.mz)
        return np.where(ok, (cz * self.my + cy) * self.mx + cx, -1)

    def face_neighbours(self):
        """(n_cells, 6) neighbour ids across the faces, -1 outside."""
        d = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
        return np.stack([self.at(self.cx + a, self.cy + b, self.cz + c) for a, b, c in d], 1)

    def all_neighbours(self):
        """(n_cells, 26) neighbour ids, -1 outside."""
        d = [(a, b, c) for c in (-1, 0, 1) for b in (-1, 0, 1) for a in (-1, 0, 1) if (a, b, c) != (0, 0, 0)]
        return np.stack([self.at(self.cx + a, self.cy + b, self.cz + c) for a, b, c in d], 1)

    def mask(self, cells):
        """Node mask of the given cells (bool per cell)."""
        m = cells.reshape(self.mz, self.my, self.mx)
        full = m.repeat(self.bz, 0).repeat(self.by, 1).repeat(self.bx, 2)
        return full[:self.shape[0], :self.shape[1], :self.shape[2]]


def k_array(media, shape, dt, dtype):
    c = media.c if media.kind == "dense" else oracle.rules_c(shape, media)
    return oracle.k_from_c(np.asarray(c, np.float32), dt, 1.0, dtype)


class Scenario:
    def __init__(self, name, shape, media, dt, sources, steps, thr_mode, tau, alpha, D,
                 neighbours=6, interval=1, dtype=F32, brick=(8, 8, 8), init=None, cancels=True):
        self.__dict__.update(locals())
        del self.__dict__["self"]


def scenarios():
    """Runs long and loud enough (levels chosen so) that cells are claimed,
    kept by a neighbour's face, shut down, re-triggered and released."""
    rng = np.random.default_rng(1702)
    out = []
    out.append(Scenario("homogeneous-relative-release", (40, 40, 40), W.homogeneous(1.0), 0.5,
                        [(13, 17, 19, W.ricker(1 / 8, 0.5))], 160, 1, 0.1, 1.0, 0))
    lay = W.Media(kind="rules", c_background=1.0, layers=[(20.0, 1.6)])
    dt = 0.5 / lay.c_max()
    out.append(Scenario("layered-absolute-decay", (64, 40, 32), lay, dt,
                        [(16, 20, 12, W.ricker(1 / 6, dt))], 200, 0, 3e-2, 0.7, 5))
    m = W.random_dense_media((33, 35, 41), 9, 1.0, 2.0)
    dt = 0.5 / m.c_max()
    two = [(5, 6, 7, W.ricker(1 / 6, dt)), (30, 28, 25, W.ricker(1 / 10, dt))]
    out.append(Scenario("ragged-absolute-decay-two-sources", (33, 35, 41), m, dt, two, 160, 0, 2e-2, 0.5, 3))
    out.append(Scenario("ragged-absolute-decay-two-sources-f64", (33, 35, 41), m, dt, two, 160, 0, 2e-2, 0.5, 3,
                        dtype=F64))
    out.append(Scenario("homogeneous-26-neighbours", (40, 40, 40), W.homogeneous(1.0), 0.5,
                        [(20, 21, 19, W.ricker(1 / 8, 0.5))], 160, 1, 0.1, 0.8, 4, neighbours=26))
    out.append(Scenario("interval-4-26-neighbours", (40, 40, 48), W.homogeneous(1.0), 0.5,
                        [(20, 21, 19, W.ricker(1 / 8, 0.5))], 200, 0, 3e-2, 0.8, 8, neighbours=26,
                        interval=4, cancels=False))
    out.append(Scenario("interval-3-faces", (40, 40, 40), W.homogeneous(1.0), 0.5,
                        [(11, 21, 19, W.ricker(1 / 8, 0.5))], 160, 0, 1.5e-2, 0.6, 6, interval=3))
    # initial fields with values everywhere in a block, random signs
    init = np.zeros((32, 32, 40), F32)
    init[9:20, 6:25, 10:33] = rng.standard_normal((11, 19, 23)).astype(F32) * F32(0.01)
    out.append(Scenario("initial-field-absolute", (32, 32, 40), W.homogeneous(1.0), 0.5, [], 160, 0, 1e-2, 0.9,
                        2, init=(init, (init * F32(0.5)).astype(F32))))
    out.append(Scenario("brick-4x4x4", (24, 28, 32), W.homogeneous(1.0), 0.5,
                        [(10, 11, 9, W.ricker(1 / 8, 0.5))], 150, 1, 0.1, 0.7, 3, brick=(4, 4, 4)))
    out.append(Scenario("brick-16x8x8", (40, 40, 64), W.homogeneous(1.0), 0.5,
                        [(20, 21, 19, W.ricker(1 / 8, 0.5))], 200, 1, 0.1, 0.7, 3, brick=(16, 8, 8)))
    return out


def make_oracle(sc):
    o = oracle.OracleTCM(sc.shape, sc.media, 1.0, sc.dt, brick=sc.brick, thr_mode=sc.thr_mode, tau=sc.tau,
                         decay_alpha=sc.alpha, decay_steps=sc.D, dtype=sc.dtype, interval=sc.interval,
                         neighbours=sc.neighbours)
    for x, y, z, w in sc.sources:
        o.add_source(x, y, z, np.asarray(w, sc.dtype))
    if sc.init is not None:
        o.set_field(*sc.init)
    return o


def observe(sc, o=None):
    """Step the oracle one step at a time and check I1-I7 after every step.

    Returns (violations: {invariant: [messages]}, counts of what happened)."""
    o = o or make_oracle(sc)
    cells = Cells(sc.shape, sc.brick)
    k = k_array(sc.media, sc.shape, sc.dt, sc.dtype)
    srcs = [(x, y, z, np.asarray(w, sc.dtype), 0) for x, y, z, w in sc.sources]
    src_cell = [cells.at(np.array(x // sc.brick[0]), np.array(y // sc.brick[1]), np.array(z // sc.brick[2]))
                for x, y, z, _, _ in srcs]
    fnb = cells.face_neighbours()
    anb = cells.all_neighbours()
    alpha = sc.dtype(sc.alpha)
    I, D = sc.interval, sc.D
    rounds = -(-D // I) if D > 0 else 0      # updates a shut-down lasts
    quiet = np.zeros(cells.n, np.int64)      # consecutive updates a boxed cell was not triggered
    bad = {f"I{i}": [] for i in range(1, 8)}
    cnt = dict(kept=0, released=0, claimed=0, decayed_steps=0, cancelled=0, triggered_by_face=0)

    def fail(inv, n, msg):
        if len(bad[inv]) < 5:
            bad[inv].append(f"step {n}: {msg}")

    def act_set():
        a = np.zeros(cells.n, bool)
        a[o.active_bricks()] = True
        return a

    for n in range(sc.steps):
        P0, P1 = o.read_field(0), o.read_field(1)
        A0 = act_set()
        if n == 0:
            # the update on the initial state (runs inside the first step call;
            # it releases nothing): level from max |phi^0|; 6 neighbours: the
            # cell across each face of phi^0 above it; 26: every neighbour of a
            # cell above it in max(|phi^0|, |phi^-1|) or fed in steps 0..I-1
            level0 = sc.tau * float(np.max(np.abs(P0))) if sc.thr_mode == 1 else sc.tau
            if sc.neighbours == 6:
                fm0 = cells.face_absmax(P0).astype(np.float64)
                for f in range(6):
                    dst = fnb[np.flatnonzero(A0 & (fm0[:, f] > level0)), f]
                    A0[dst[dst >= 0]] = True
            else:
                hot = A0 & (np.maximum(cells.absmax(P0), cells.absmax(P1)).astype(np.float64) > level0)
                for (x, y, z, w, s0), c in zip(srcs, src_cell):
                    if len(w) and s0 <= I - 1:
                        hot[int(c)] = True
                nb = anb[np.flatnonzero(hot)]
                A0[nb[nb >= 0]] = True
        Dn, _ = oracle.dense_run(k, P0, P1, 1, srcs, step0=n)
        o.step(1)
        A1 = act_set()
        Q0, Q1 = o.read_field(0), o.read_field(1)
        bq0, bq1, bp0, bd = cells.blocks(Q0), cells.blocks(Q1), cells.blocks(P0), cells.blocks(Dn)
        upd = (n + 1) % I == 0
        K, R, N = A0 & A1, A0 & ~A1, ~A0 & A1
        # expected decay this step: shut-down started at an earlier update
        decaying = (quiet >= 1) & (quiet <= rounds) & A0 if D > 0 else np.zeros(cells.n, bool)
        flat = lambda b: b.reshape(cells.n, -1)
        plain = np.all(flat(bq0) == flat(bd), axis=1)
        scaled = np.all(flat(bq0) == flat(alpha * bd), axis=1)
        # I1 rotation
        for b in np.flatnonzero(K & ~np.all(flat(bq1) == flat(bp0), axis=1)):
            fail("I1", n, f"cell {b}: phi^n changed")
        # I2 / I5: Eq. 3, times alpha exactly in shut-down
        for b in np.flatnonzero(K & decaying & ~scaled):
            fail("I5", n, f"cell {b} in shut-down not scaled by alpha")
        for b in np.flatnonzero(K & ~decaying & ~plain):
            fail("I2", n, f"cell {b} differs from one Eq. 3 step" + (" (scaled?)" if scaled[b] else ""))
        cnt["decayed_steps"] += int(np.sum(K & decaying & ~plain))
        # I6: new boxes start at zero; unboxed cells read zero
        for b in np.flatnonzero(N & (np.any(flat(bq0) != 0, 1) | np.any(flat(bq1) != 0, 1))):
            fail("I6", n, f"new cell {b} not zero")
        if np.any(Q0[~cells.mask(A1)] != 0) or np.any(Q1[~cells.mask(A1)] != 0):
            fail("I6", n, "unboxed node holds a value")
        if not upd:
            if not np.array_equal(A0, A1):
                fail("I5", n, "boxed cells changed between updates")
            continue
        # the state the update sees: phi^{n+1} of every cell boxed during the step
        nxt = np.where((R & decaying)[:, None, None, None], alpha * bd, bd)
        nxt = np.where(K[:, None, None, None], bq0, nxt)
        nxt_full = cells.unblocks(nxt)
        nxt_full = np.where(cells.mask(A0), nxt_full, sc.dtype(0))
        G = float(np.max(np.abs(nxt_full)))
        level = sc.tau * G if sc.thr_mode == 1 else sc.tau
        mB = np.maximum(cells.absmax(nxt_full), cells.absmax(P0)).astype(np.float64)
        fm = cells.face_absmax(nxt_full).astype(np.float64)
        own = A0 & (mB > level)
        forced = np.zeros(cells.n, bool)
        for (x, y, z, w, s0), c in zip(srcs, src_cell):
            if n + 1 + I - 1 >= s0 and n + 1 < s0 + len(w):
                forced[int(c)] = True
        if sc.neighbours == 6:
            hot_in = np.zeros(cells.n, bool)    # receives a face above the level from a boxed cell
            for f in range(6):
                src = np.flatnonzero(A0 & (fm[:, f] > level))
                dst = fnb[src, f]
                hot_in[dst[dst >= 0]] = True
            trig = own | hot_in | forced
            must_box = hot_in | forced
            cnt["triggered_by_face"] += int(np.sum(A0 & hot_in & ~own & ~forced))
        else:
            t26 = own | forced
            near = t26.copy()
            nb = anb[np.flatnonzero(t26)]
            near[nb[nb >= 0]] = True
            trig = near
            must_box = near
        # I3: above the level => not released
        for b in np.flatnonzero(own & ~A1):
            fail("I3", n, f"cell {b} above the level released")
        # I4: triggered neighbours boxed
        for b in np.flatnonzero(must_box & ~A1 & ~forced):
            fail("I4", n, f"cell {b} triggered but not boxed")
        # I7: source cells boxed while feeding
        for b in np.flatnonzero(forced & ~A1):
            fail("I7", n, f"source cell {b} not boxed")
        # I5: shut-down bookkeeping
        q_new = np.where(A0 & ~trig, quiet + 1, 0)
        cnt["cancelled"] += int(np.sum(A0 & trig & (quiet > 0)))
        release = A0 & (q_new == rounds + 1)
        for b in np.flatnonzero(release & A1 & ~must_box):
            fail("I5", n, f"cell {b} finished its shut-down but stays boxed")
        for b in np.flatnonzero(A0 & ~release & ~A1):
            fail("I5", n, f"cell {b} released before the end of its shut-down (quiet {q_new[b]})")
        quiet = np.where(A1 & ~release, q_new, 0)
        quiet[N] = 0
        cnt["kept"] += int(np.sum(K))
        cnt["released"] += int(np.sum(R))
        cnt["claimed"] += int(np.sum(N))
    return {k: v for k, v in bad.items() if v}, cnt


@pytest.mark.parametrize("sc", scenarios(), ids=lambda s: s.name)
def test_update_procedure_invariants(sc):
    bad, cnt = observe(sc)
    assert not bad, bad
    # the scenario exercised what it pins
    assert cnt["released"] > 0 and cnt["claimed"] > 0 and cnt["kept"] > 0, cnt
    if sc.D > 0:
        assert cnt["decayed_steps"] > 0 and (cnt["cancelled"] > 0 or not sc.cancels), cnt
    if sc.neighbours == 6:
        assert cnt["triggered_by_face"] > 0, cnt


# ------------------------------------------------------------ worked examples
def single_node_state(v=1.0):
    """phi^0 = v at the centre node (12,12,12) of the middle cell of a 24^3
    domain (3^3 cells of 8^3), phi^{-1} = v there: with c = 1, dt = 0.5
    (k = 1/4) one step gives phi^1 = v/2 - ... exactly representable values."""
    now = np.zeros((24, 24, 24), F32)
    now[12, 12, 12] = F32(v)
    return now, now.copy()


@pytest.mark.parametrize("tau,kept", [(1.0, False), (float(np.nextafter(F32(1.0), F32(0))), True)])
def test_level_equal_to_cell_maximum_is_not_above(tau, kept):
    """Step 3 keeps cells whose maximal |value| is above the level: at a level
    equal to the maximum (here |phi^0| = 1 at the only non-zero node; phi^1 =
    -1/2 there, +1/4 at its six neighbours, all inside the cell) the cell is
    released (D = 0); one ulp below it, it stays."""
    now, prev = single_node_state()
    o = oracle.OracleTCM((24, 24, 24), W.homogeneous(1.0), 1.0, 0.5, thr_mode=oracle.THR_ABSOLUTE, tau=tau)
    o.set_field(now, prev)
    o.step(1)
    assert o.read_field(1)[12, 12, 12] == (1.0 if kept else 0.0)
    assert (o.active_bricks().tolist() == [13]) == kept
    if not kept:
        assert o.active_count()[0] == 0


def test_cell_maximum_covers_phi_n_at_threshold_zero():
    """A cell whose phi^{n+1} vanishes while phi^n does not still holds a wave
    (the leapfrog state is the pair of levels); at threshold 0 the TCM must
    not drop it.  phi^0 = 1 at one node, phi^{-1} = 1/2 there and 1/4 at its
    six neighbours: then phi^1 = 0 at every node exactly (k = 1/4), phi^2 =
    -phi^0.  The TCM must equal the dense grid at every step."""
    now = np.zeros((24, 24, 24), F32)
    prev = np.zeros_like(now)
    now[12, 12, 12] = 1.0
    prev[12, 12, 12] = 0.5
    for d in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
        prev[12 + d[0], 12 + d[1], 12 + d[2]] = 0.25
    k = oracle.k_from_c(np.ones(now.shape, np.float32), 0.5, 1.0, F32)
    a1, _ = oracle.dense_run(k, now, prev, 1)
    assert not a1.any()                                  # phi^1 = 0 exactly
    o = oracle.OracleTCM(now.shape, W.homogeneous(1.0), 1.0, 0.5)
    o.set_field(now, prev)
    for n in range(1, 12):
        o.step(1)
        a, b = oracle.dense_run(k, now, prev, n)
        assert np.array_equal(o.read_field(0), a), n
        assert np.array_equal(o.read_field(1), b), n
    assert o.read_field(0).any()


def test_cell_kept_by_neighbour_face_keeps_values_and_does_not_decay():
    """Steps 3-4 then 6: a cell triggered only because the touching face of a
    triggered neighbour is above the level is triggered, so it neither shuts
    down nor loses its values.  Cell A (x 0..7) gets phi^1 = 1 on its x+ face
    (phi^0 = 0, phi^{-1} = -1 there); cell B (x 8..15) holds 1e-4 everywhere,
    far below the level 1e-2, and stays below it after the step."""
    shape = (8, 8, 16)
    now = np.zeros(shape, F32)
    prev = np.zeros(shape, F32)
    now[:, :, 8:] = F32(1e-4)
    prev[:, :, 8:] = F32(1e-4)
    prev[:, :, 7] = F32(-1.0)
    o = oracle.OracleTCM(shape, W.homogeneous(1.0), 1.0, 0.5, thr_mode=oracle.THR_ABSOLUTE, tau=1e-2,
                         decay_alpha=0.5, decay_steps=5)
    o.set_field(now, prev)
    k = oracle.k_from_c(np.ones(shape, np.float32), 0.5, 1.0, F32)
    a1, b1 = oracle.dense_run(k, now, prev, 1)
    assert np.max(np.abs(a1[:, :, 8:])) < 1e-2 and np.max(np.abs(a1[:, :, 7])) > 1e-2
    o.step(1)
    assert o.active_bricks().tolist() == [0, 1]
    assert np.array_equal(o.read_field(0), a1) and np.array_equal(o.read_field(1), b1)
    # B is not in shut-down: the next step is plain Eq. 3, no alpha
    a2, _ = oracle.dense_run(k, a1, b1, 1)
    o.step(1)
    assert np.array_equal(o.read_field(0)[:, :, 8:], a2[:, :, 8:])


def _in(sl, shape):
    m = np.zeros(shape, bool)
    m[sl] = True
    return m


@pytest.mark.parametrize("interval,D,decayed", [(1, 6, 6), (3, 6, 6), (2, 6, 6), (4, 6, 8)])
def test_shutdown_length_with_an_update_interval(interval, D, decayed):
    """Eq. 6 with the Eq. 5 interval: a lone quiet cell decays by alpha per
    time step while in shut-down and is released when the count (in time
    steps) runs out.  With an interval dividing D the shut-down lasts exactly
    D steps (A = alpha^D); otherwise it lasts the next multiple of the
    interval (the count is only inspected at updates)."""
    now, prev = single_node_state(1e-3)
    o = oracle.OracleTCM((24, 24, 24), W.homogeneous(1.0), 1.0, 0.5, thr_mode=oracle.THR_ABSOLUTE, tau=1.0,
                         decay_alpha=0.5, decay_steps=D, interval=interval)
    o.set_field(now, prev)
    k = oracle.k_from_c(np.ones(now.shape, np.float32), 0.5, 1.0, F32)
    cell = (slice(8, 16), slice(8, 16), slice(8, 16))
    a, b = now, prev
    n_decayed = 0
    for n in range(40):
        if o.active_count()[0] == 0:
            break
        q, _ = oracle.dense_run(k, a, b, 1)
        q[~_in(cell, q.shape)] = 0       # the only boxed cell: nothing outside it
        o.step(1)
        got = o.read_field(0)
        if o.active_count()[0]:
            assert o.active_bricks().tolist() == [13]
            if np.array_equal(got, F32(0.5) * q):
                n_decayed += 1
            else:
                assert np.array_equal(got, q), n
            a, b = got, a
        else:
            n_decayed += 1          # the releasing update follows a decayed step
    # the first update (after step interval-1) finds the cell quiet; it then
    # decays for `decayed` steps and is released at the update that ends them
    assert n_decayed == decayed, n_decayed
    assert o.active_count()[0] == 0


# ------------------------------------------------------------ threshold sweep
@pytest.mark.parametrize("case", ["homogeneous", "heterogeneous"])
def test_deviation_from_dense_shrinks_with_the_level(case):
    """The TCM drops only what is below the level: as the relative level
    falls from 1e-2 to 1e-6 the largest deviation from the dense grid falls
    with it; from 1e-6 to 1e-8 it stays within 1e-5 max|phi| (rounding at the
    front, where dropped values of ~1e-8 max|phi| change the last bits of
    sums); at level 0 it is exactly zero."""
    if case == "homogeneous":
        shape, media, dt = (48, 48, 48), W.homogeneous(1.0), 0.5
        srcs = [(24, 24, 24, W.ricker(1 / 12, dt))]
    else:
        shape = (40, 44, 36)
        media = W.random_dense_media(shape, 4, 1.0, 2.2)
        dt = 0.5 / media.c_max()
        srcs = [(10, 30, 22, W.ricker(1 / 10, dt))]
    steps = 110
    k = k_array(media, shape, dt, F32)
    z = np.zeros(shape, F32)
    ref, _ = oracle.dense_run(k, z, z, steps, [(x, y, zz, np.asarray(w, F32)) for x, y, zz, w in srcs])
    gmax = float(np.max(np.abs(ref)))
    errs = []
    for tau in (1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-7, 1e-8, 0.0):
        o = oracle.OracleTCM(shape, media, 1.0, dt, thr_mode=oracle.THR_RELATIVE, tau=tau,
                             decay_alpha=0.8, decay_steps=10)
        for x, y, zz, w in srcs:
            o.add_source(x, y, zz, np.asarray(w, F32))
        o.step(steps)
        errs.append(float(np.max(np.abs(o.read_field(0) - ref))))
        o.close()
    assert errs[-1] == 0.0
    assert errs[0] > 0.0
    # down to 1e-6 the deviation falls with the level (about tenfold per decade)
    for a, b in zip(errs[:4], errs[1:5]):
        assert b < a / 3, errs
    # below that, what is dropped no longer dominates: the deviation is the
    # rounding that the missing tiny values change at the front, within the
    # binary32 tolerance of 1e-5 max|phi|
    for e in errs[4:7]:
        assert e <= 1e-5 * gmax, (errs, gmax)
