"""Pins of the oracle's 16-bit storage form (field stored as bfloat16 or
binary16, arithmetic in binary32).

The rounding routines are pinned to independent library conversions (numpy's
binary16 cast, torch's bfloat16 cast, both round to nearest even).  The
16-bit storage uses the velocity form of Eq. 3 (phi^n and v^n = phi^n -
phi^{n-1} per box).  Its algebra is pinned by equality to rounding with the
leapfrog form (the plain Eq. 3, pinned elsewhere against closed forms) in
binary64 and binary32; the storage form is pinned as a composition of pinned
parts: one binary32 velocity-form step followed by the library rounding,
repeated step by step, must give the 16-bit run bit for bit; at threshold 0
the 16-bit TCM must equal the 16-bit dense grid (the method skips only nodes
that hold no wave, in any storage).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1702_00216_gb300 import workloads as W

F32 = np.float32


def lib_round(v, storage, scale=1.0):
    """Library rounding: numpy binary16 / torch bfloat16, as binary32."""
    v = np.asarray(v, F32)
    if storage == "f16":
        with np.errstate(over="ignore"):
            return ((v / F32(scale)).astype(np.float16).astype(F32) * F32(scale)).astype(F32)
    torch = pytest.importorskip("torch")
    return torch.from_numpy(v.copy()).to(torch.bfloat16).to(torch.float32).numpy()


def edge_values():
    rng = np.random.default_rng(16)
    v = [0.0, -0.0, 1.0, -1.0, 65504.0, 65519.99, 65520.0, 65536.0, 2.0 ** -24, 2.0 ** -25,
         1.5 * 2.0 ** -24, 2.0 ** -14, 2.0 ** -15 * 3, 1 + 2.0 ** -8, 1 + 2.0 ** -11, 1 + 3 * 2.0 ** -12,
         3.3895314e38, 3.39e38, 3.4e38, 1e-40, 1e-45, 2.0 ** -126, 2.0 ** -133, 2.0 ** -134,
         np.inf, -np.inf]
    # ties: exact midpoints between neighbours of both formats
    for e in range(-20, 20):
        for m in (1, 3, 5, 255):
            v.append((1 + m * 2.0 ** -9) * 2.0 ** e)     # bf16 ties
            v.append((1 + m * 2.0 ** -12) * 2.0 ** e)    # f16 ties
    v += list(rng.standard_normal(4000) * 10.0 ** rng.uniform(-30, 30, 4000))
    v += list(rng.uniform(-70000, 70000, 2000))
    v += list(rng.uniform(-1, 1, 2000) * 2.0 ** -14)     # f16 subnormals
    bits = rng.integers(0, 2 ** 32, 4000, dtype=np.uint64).astype(np.uint32).view(F32)
    with np.errstate(over="ignore"):
        a = np.concatenate([np.array(v, dtype=np.float64).astype(F32), bits])   # every bit class
    return a[~np.isnan(a)]


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_rounding_matches_library_cast(storage):
    v = edge_values()
    got = oracle.round_storage(v, storage)
    ref = lib_round(v, storage)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_rounding_detects_truncation():
    # truncation instead of nearest-even would fail here
    assert oracle.round_storage([1 + 3 * 2.0 ** -9], "bf16")[0] == F32(1 + 2.0 ** -7)
    assert oracle.round_storage([1 + 3 * 2.0 ** -12], "f16")[0] == F32(1 + 2.0 ** -10)
    assert oracle.round_storage([1 + 2.0 ** -8], "bf16")[0] == 1.0          # tie to even
    assert oracle.round_storage([2.0 ** -25], "f16")[0] == 0.0              # tie to even (zero)


def dense_case():
    m = W.random_dense_media((19, 21, 26), 7, 1.0, 2.0)
    dt = 0.5 / m.c_max()
    return m, dt


def composed_run(m, dt, storage, src, steps):
    """binary32 velocity-form step of the oracle, then library rounding of
    phi^{n+1} and v^{n+1}, repeated."""
    shape = m.c.shape
    x, y, z, w = src
    w = np.asarray(w, F32)
    scale = 1.0
    if storage == "f16":
        e = math.frexp(float(np.max(np.abs(w))))[1] - 8
        scale = 2.0 ** e
    now = np.zeros(shape, F32)
    v = np.zeros(shape, F32)
    for n in range(steps):
        o = oracle.OracleTCM(shape, m, 1.0, dt, dense=True, velocity=True)
        o.set_field_velocity(now, v)
        if n < len(w):
            o.add_source(x, y, z, w[n:n + 1])
        o.step(1)
        now, v = lib_round(o.read_field(0), storage, scale), lib_round(o.read_velocity(), storage, scale)
        o.close()
    return now, v, scale


@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-12), (F32, 2e-5)])
def test_velocity_form_equals_leapfrog_to_rounding(dtype, tol):
    # the velocity form is Eq. 3 rearranged: equal to rounding in binary64 and
    # binary32, so a dropped term or a wrong sign would show
    m, dt = dense_case()
    w = W.ricker(1 / 6, dt)
    runs = []
    for vel in (False, True):
        o = oracle.OracleTCM(m.c.shape, m, 1.0, dt, dtype=dtype, velocity=vel, thr_mode=1, tau=1e-4,
                             decay_alpha=0.8, decay_steps=4)
        o.add_source(11, 9, 8, w)
        o.step(90)
        runs.append((o.read_field(0), o.read_field(1), o.active_bricks()))
    (a0, a1, ia), (b0, b1, ib) = runs
    g = np.abs(a0).max()
    assert g > 0 and np.abs(a0 - b0).max() <= tol * g and np.abs(a1 - b1).max() <= tol * g
    assert np.array_equal(ia, ib)
    if dtype == F32:
        assert not np.array_equal(a0, b0)          # not the same program


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_storage_run_equals_velocity_step_then_library_rounding(storage):
    m, dt = dense_case()
    w = W.ricker(1 / 6, dt).astype(F32) * F32(3.7)
    src = (11, 9, 8, w)
    steps = 40
    now, v, scale = composed_run(m, dt, storage, src, steps)
    o = oracle.OracleTCM(m.c.shape, m, 1.0, dt, dense=True, storage=storage)
    o.add_source(*src[:3], w)
    o.step(steps)
    assert o.storage_scale == scale
    assert np.array_equal(o.read_field(0), now)
    assert np.array_equal(o.read_velocity(), v)
    assert np.array_equal(o.read_field(1), (now - v).astype(F32))
    # and the rounding is really there: the binary32 run differs
    o32 = oracle.OracleTCM(m.c.shape, m, 1.0, dt, dense=True, velocity=True)
    o32.add_source(*src[:3], w)
    o32.step(steps)
    assert not np.array_equal(o32.read_field(0), now)


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_storage_threshold0_tcm_equals_dense(storage):
    m, dt = dense_case()
    w = W.ricker(1 / 8, dt).astype(F32)
    runs = []
    for dense in (False, True):
        o = oracle.OracleTCM(m.c.shape, m, 1.0, dt, dense=dense, storage=storage)
        o.add_source(4, 17, 3, w)
        o.add_source(20, 2, 15, w[:30])
        o.step(60)
        runs.append((o.read_field(0), o.read_field(1), o.active_count()))
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    assert runs[0][2][0] < runs[1][2][0] or runs[0][2] == runs[1][2]


def test_f16_scale_rule_and_initial_field_rounding():
    m, dt = dense_case()
    rng = np.random.default_rng(3)
    now = np.zeros(m.c.shape, F32)
    now[5:9, 6:10, 7:12] = rng.standard_normal((4, 4, 5)).astype(F32) * F32(1000.0)
    prev = now * F32(0.999)
    o = oracle.OracleTCM(m.c.shape, m, 1.0, dt, storage="f16")
    o.set_field(now, prev)
    o.step(1)
    peak = float(max(np.abs(now).max(), np.abs(prev).max()))
    e = math.frexp(peak)[1] - 8
    s = 2.0 ** e
    assert o.storage_scale == s and 128 <= peak / s < 256
    # one velocity-form step from phi^0 and v^0 = phi^0 - phi^{-1}, each rounded
    r = oracle.OracleTCM(m.c.shape, m, 1.0, dt, velocity=True)
    r.set_field_velocity(lib_round(now, "f16", s), lib_round(now - prev, "f16", s))
    r.step(1)
    assert np.array_equal(o.read_field(0), lib_round(r.read_field(0), "f16", s))
    assert np.array_equal(o.read_velocity(), lib_round(r.read_velocity(), "f16", s))


def test_f64_program_refuses_16bit_storage():
    with pytest.raises(ValueError):
        oracle.OracleTCM((8, 8, 8), W.homogeneous(1.0), 1.0, 0.5, dtype=np.float64, storage="bf16")
