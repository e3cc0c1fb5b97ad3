"""CPU oracle for the Triggered Cells Method (Naeh, arXiv:1702.00216).

TEST INFRASTRUCTURE ONLY: only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_1702_00216_gb300``) never imports it and shares no code with it.

This module is argument marshalling over the plain C programs in
``tcm_oracle.c`` (dense FDTD of Eq. 3, and the TCM algorithm in the paper's
order); see ``tcm_oracle.h`` for what each function computes and where in the
paper it comes from.

Parity status of each function (what pins it, see tests/test_oracle_pins.py):
  dense_run      pinned: Dirichlet eigenmode closed form (dispersion of Eq. 3),
                 energy invariant, causality, mirror symmetry, CFL (Eq. 4)
  energy         pinned: constant under the exact leapfrog recursion; closed
                 form for one eigenmode
  k_from_c       pinned: exact values for representable inputs
  OracleTCM      pinned: equal, bit for bit, to dense_run at threshold 0 (the
                 TCM skips only where no wave is present); brute force over
                 every source position on 1-3 cell grids; box reuse; masked
                 dense recursion with the recorded active sets at threshold > 0
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_LIB = None

ORC_MEDIA_DENSE, ORC_MEDIA_RULES = 0, 1
STORAGE_F32, STORAGE_BF16, STORAGE_F16 = 0, 1, 2
_STORAGE_NAMES = {"f32": STORAGE_F32, "bf16": STORAGE_BF16, "f16": STORAGE_F16}
THR_ABSOLUTE, THR_RELATIVE = 0, 1

_i64 = C.c_int64
_vp = C.c_void_p
_d = C.c_double


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = C.CDLL(path)
        for sfx in ("f32", "f64"):
            getattr(L, f"orc_dense_run_{sfx}").argtypes = [
                _i64, _i64, _i64, _vp, _vp, _vp, C.c_int, _vp, _vp, _vp, _vp, _i64, _i64, _i64]
            getattr(L, f"orc_dense_run_{sfx}").restype = C.c_int
            getattr(L, f"orc_energy_{sfx}").argtypes = [_i64, _i64, _i64, _vp, _vp, _vp]
            getattr(L, f"orc_energy_{sfx}").restype = _d
            getattr(L, f"orc_k_from_c_{sfx}").argtypes = [_vp, _i64, _d, _d, _vp]
            getattr(L, f"orc_k_from_c_{sfx}").restype = None
            f = getattr(L, f"orc_tcm_create_{sfx}")
            f.argtypes = [_i64, _i64, _i64, C.c_int, C.c_int, C.c_int, C.c_int, _vp, C.c_float,
                          C.c_int, _vp, _vp, C.c_int, _vp, _vp, _d, _d, C.c_int, _d, _d, C.c_int,
                          _i64, C.c_int]
            f.restype = _vp
            getattr(L, f"orc_tcm_add_source_{sfx}").argtypes = [_vp, _i64, _i64, _i64, _vp, _i64]
            getattr(L, f"orc_tcm_set_field_{sfx}").argtypes = [_vp, _vp, _vp]
            getattr(L, f"orc_tcm_step_{sfx}").argtypes = [_vp, _i64]
            getattr(L, f"orc_tcm_read_field_{sfx}").argtypes = [
                _vp, C.c_int, _i64, _i64, _i64, _i64, _i64, _i64, _vp]
            getattr(L, f"orc_tcm_active_count_{sfx}").argtypes = [_vp, _vp]
            getattr(L, f"orc_tcm_active_count_{sfx}").restype = _i64
            getattr(L, f"orc_tcm_active_bricks_{sfx}").argtypes = [_vp, _vp, _i64]
            getattr(L, f"orc_tcm_active_bricks_{sfx}").restype = _i64
            for name in ("updates", "step_index"):
                getattr(L, f"orc_tcm_{name}_{sfx}").argtypes = [_vp]
                getattr(L, f"orc_tcm_{name}_{sfx}").restype = _i64
            getattr(L, f"orc_tcm_status_{sfx}").argtypes = [_vp]
            getattr(L, f"orc_tcm_set_storage_{sfx}").argtypes = [_vp, C.c_int]
            getattr(L, f"orc_tcm_set_schedule_{sfx}").argtypes = [_vp, C.c_int, C.c_int]
            getattr(L, f"orc_tcm_set_velocity_form_{sfx}").argtypes = [_vp, C.c_int]
            getattr(L, f"orc_tcm_set_field_velocity_{sfx}").argtypes = [_vp, _vp, _vp]
            getattr(L, f"orc_tcm_read_velocity_{sfx}").argtypes = [_vp, _i64, _i64, _i64, _i64, _i64, _i64, _vp]
            getattr(L, f"orc_tcm_set_lpf_{sfx}").argtypes = [_vp, _d, _d]
            getattr(L, f"orc_tcm_storage_scale_{sfx}").argtypes = [_vp]
            getattr(L, f"orc_tcm_storage_scale_{sfx}").restype = _d
            getattr(L, f"orc_tcm_brick_media_{sfx}").argtypes = [_vp, _i64, _vp]
            getattr(L, f"orc_tcm_destroy_{sfx}").argtypes = [_vp]
            getattr(L, f"orc_tcm_destroy_{sfx}").restype = None
        L.orc_rules_c.argtypes = [_i64, _i64, _i64, C.c_float, C.c_int, _vp, _vp, C.c_int, _vp,
                                  _vp, _vp]
        L.orc_rules_c.restype = None
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_fft.argtypes = [_vp, _vp, C.c_int, C.c_int]
        L.orc_fft.restype = None
        L.orc_lpf_response.argtypes = [C.c_int, C.c_int, _d, _d]
        L.orc_lpf_response.restype = _d
        L.orc_lpf_region.argtypes = [_vp, C.c_int, C.c_int, _d, _d]
        L.orc_lpf_region.restype = None
        for name in ("orc_round_bf16", "orc_round_f16"):
            getattr(L, name).argtypes = [C.c_float]
            getattr(L, name).restype = C.c_float
        _LIB = L
    return _LIB


def set_threads(n: int) -> int:
    """OpenMP threads for the oracle's per-node loops; returns the count in use."""
    return int(lib().orc_set_threads(int(n)))


def _sfx(dtype) -> str:
    dt = np.dtype(dtype)
    if dt == np.float32:
        return "f32"
    if dt == np.float64:
        return "f64"
    raise ValueError(f"oracle supports float32/float64, not {dt}")


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(_vp)


def k_from_c(c: np.ndarray, dt: float, dx: float, dtype=np.float32) -> np.ndarray:
    """Eq. 3 coefficient (c*dt/dx)^2, formed in FP64 and rounded to dtype."""
    c = np.ascontiguousarray(c, dtype=np.float32)
    out = np.empty(c.shape, dtype=dtype)
    getattr(lib(), f"orc_k_from_c_{_sfx(dtype)}")(_ptr(c), c.size, float(dt), float(dx), _ptr(out))
    return out


def rules_c(shape, media) -> np.ndarray:
    """Evaluate rules media at every node of a (nz, ny, nx) grid."""
    nz, ny, nx = shape
    lz, lc, sp, sc = _rules_arrays(media)
    out = np.empty((nz, ny, nx), dtype=np.float32)
    lib().orc_rules_c(nx, ny, nz, float(media.c_background), len(lc), _ptr(lz), _ptr(lc),
                      len(sc), _ptr(sp), _ptr(sc), _ptr(out))
    return out


def _rules_arrays(media):
    lz = np.ascontiguousarray([z for z, _ in media.layers] or [0.0], dtype=np.float64)
    lc = np.ascontiguousarray([c for _, c in media.layers], dtype=np.float32)
    sp = np.ascontiguousarray([s[:4] for s in media.spheres] or [[0.0] * 4], dtype=np.float64)
    sc = np.ascontiguousarray([s[4] for s in media.spheres], dtype=np.float32)
    return lz, lc, sp, sc


def dense_run(k: np.ndarray, now: np.ndarray, prev: np.ndarray, steps: int, sources=(),
              step0: int = 0):
    """Advance the dense FDTD of Eq. 3 by `steps` steps (copies; returns (now, prev)).

    Arrays are (nz, ny, nx).  `sources` is a sequence of (x, y, z, w[, start]).
    """
    dtype = k.dtype
    sfx = _sfx(dtype)
    nz, ny, nx = k.shape
    k = np.ascontiguousarray(k)
    now = np.array(now, dtype=dtype, order="C", copy=True)
    prev = np.array(prev, dtype=dtype, order="C", copy=True)
    ns = len(sources)
    idx = np.zeros(max(ns, 1), np.int64)
    start = np.zeros(max(ns, 1), np.int64)
    ln = np.zeros(max(ns, 1), np.int64)
    wl = max([len(s[3]) for s in sources] + [1])
    W = np.zeros((max(ns, 1), wl), dtype=dtype)
    for i, s in enumerate(sources):
        x, y, z, w = s[:4]
        idx[i] = (z * ny + y) * nx + x
        start[i] = s[4] if len(s) > 4 else 0
        ln[i] = len(w)
        W[i, :len(w)] = np.asarray(w, dtype=dtype)
    rc = getattr(lib(), f"orc_dense_run_{sfx}")(nx, ny, nz, _ptr(k), _ptr(now), _ptr(prev), ns,
                                               _ptr(idx), _ptr(start), _ptr(ln), _ptr(W), wl,
                                               int(step0), int(steps))
    if rc != 0:
        raise RuntimeError(f"orc_dense_run failed: {rc}")
    return now, prev


def round_storage(v, storage) -> np.ndarray:
    """Round binary32 values to bfloat16 ("bf16") or binary16 ("f16"), nearest
    even, returned as binary32 (the oracle's element-wise C routine)."""
    fn = getattr(lib(), "orc_round_" + storage)
    a = np.asarray(v, dtype=np.float32)
    return np.array([fn(float(x)) for x in a.ravel()], dtype=np.float32).reshape(a.shape)


def fft(x, sign: int = -1) -> np.ndarray:
    """The oracle's radix-2 DFT of a complex vector (length a power of two)."""
    x = np.asarray(x, dtype=np.complex128)
    re = np.ascontiguousarray(x.real)
    im = np.ascontiguousarray(x.imag)
    lib().orc_fft(_ptr(re), _ptr(im), len(x), int(sign))
    return re + 1j * im


def lpf_response(kappa: int, M: int, pass_: float, stop: float) -> float:
    return float(lib().orc_lpf_response(int(kappa), int(M), float(pass_), float(stop)))


def lpf_region(v: np.ndarray, M: int, pass_: float, stop: float) -> np.ndarray:
    """Eq. 7 on a cubic region (zero-padded to M per axis); returns a copy."""
    v = np.array(v, dtype=np.float64, order="C", copy=True)
    L = v.shape[0]
    assert v.shape == (L, L, L)
    lib().orc_lpf_region(_ptr(v), L, int(M), float(pass_), float(stop))
    return v


def energy(k: np.ndarray, a: np.ndarray, b: np.ndarray) -> float:
    """Leapfrog discrete energy between phi^{n+1} = a and phi^n = b (FP64 sum)."""
    sfx = _sfx(k.dtype)
    nz, ny, nx = k.shape
    a = np.ascontiguousarray(a, dtype=k.dtype)
    b = np.ascontiguousarray(b, dtype=k.dtype)
    return float(getattr(lib(), f"orc_energy_{sfx}")(nx, ny, nz, _ptr(np.ascontiguousarray(k)),
                                                     _ptr(a), _ptr(b)))


class OracleTCM:
    """The Triggered Cells Method on the CPU (plain C, one box at a time)."""

    def __init__(self, shape, media, dx: float, dt: float, brick=(8, 8, 8),
                 thr_mode: int = THR_ABSOLUTE, tau: float = 0.0, decay_alpha: float = 1.0,
                 decay_steps: int = 0, max_slots: int = 0, dense: bool = False,
                 dtype=np.float32, storage="f32", interval: int = 1, neighbours: int = 6,
                 lpf=None, velocity=None):
        self.dtype = np.dtype(dtype)
        self._s = _sfx(dtype)
        self.shape = tuple(int(v) for v in shape)
        nz, ny, nx = self.shape
        self.brick = tuple(int(v) for v in brick)
        bx, by, bz = self.brick
        L = lib()
        self._keep = []
        if media.kind == "dense":
            c = np.ascontiguousarray(media.c, dtype=np.float32)
            assert c.shape == self.shape
            self._keep.append(c)
            h = getattr(L, f"orc_tcm_create_{self._s}")(
                nx, ny, nz, bx, by, bz, ORC_MEDIA_DENSE, _ptr(c), 0.0, 0, None, None, 0, None,
                None, float(dx), float(dt), int(thr_mode), float(tau), float(decay_alpha),
                int(decay_steps), int(max_slots), int(bool(dense)))
        else:
            lz, lc, sp, sc = _rules_arrays(media)
            h = getattr(L, f"orc_tcm_create_{self._s}")(
                nx, ny, nz, bx, by, bz, ORC_MEDIA_RULES, None, float(media.c_background),
                len(lc), _ptr(lz), _ptr(lc), len(sc), _ptr(sp), _ptr(sc), float(dx), float(dt),
                int(thr_mode), float(tau), float(decay_alpha), int(decay_steps), int(max_slots),
                int(bool(dense)))
        if not h:
            raise ValueError("orc_tcm_create rejected its arguments")
        self._h = h
        st = _STORAGE_NAMES[storage] if isinstance(storage, str) else int(storage)
        if st != STORAGE_F32 and self._f("set_storage")(h, st) != 0:
            self.close()
            raise ValueError("storage not supported by this program")
        if (interval, neighbours) != (1, 6) and self._f("set_schedule")(h, int(interval),
                                                                         int(neighbours)) != 0:
            self.close()
            raise ValueError("invalid update schedule")
        if velocity is not None and self._f("set_velocity_form")(h, int(bool(velocity))) != 0:
            self.close()
            raise ValueError("velocity form not available here")
        if lpf is not None and self._f("set_lpf")(h, float(lpf[0]), float(lpf[1])) != 0:
            self.close()
            raise ValueError("invalid low-pass shut-down")
        self.mx = -(-nx // bx)
        self.my = -(-ny // by)
        self.mz = -(-nz // bz)

    def _f(self, name):
        return getattr(lib(), f"orc_tcm_{name}_{self._s}")

    def close(self):
        if getattr(self, "_h", None):
            self._f("destroy")(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_source(self, x, y, z, w):
        w = np.ascontiguousarray(w, dtype=self.dtype)
        rc = self._f("add_source")(self._h, int(x), int(y), int(z), _ptr(w), len(w))
        if rc != 0:
            raise RuntimeError(f"orc_tcm_add_source failed: {rc}")

    def set_field(self, now, prev):
        now = np.ascontiguousarray(now, dtype=self.dtype)
        prev = np.ascontiguousarray(prev, dtype=self.dtype)
        assert now.shape == self.shape and prev.shape == self.shape
        rc = self._f("set_field")(self._h, _ptr(now), _ptr(prev))
        if rc != 0:
            raise RuntimeError(f"orc_tcm_set_field failed: {rc}")

    def step(self, n: int = 1) -> int:
        return int(self._f("step")(self._h, int(n)))

    def read_field(self, which: int = 0, origin=(0, 0, 0), size=None) -> np.ndarray:
        """Window of phi^n (which=0) or phi^{n-1} (which=1); origin/size are (x, y, z)."""
        if size is None:
            size = (self.shape[2], self.shape[1], self.shape[0])
        wx, wy, wz = (int(v) for v in size)
        out = np.zeros((wz, wy, wx), dtype=self.dtype)
        rc = self._f("read_field")(self._h, int(which), int(origin[0]), int(origin[1]),
                                   int(origin[2]), wx, wy, wz, _ptr(out))
        if rc != 0:
            raise RuntimeError(f"orc_tcm_read_field failed: {rc}")
        return out

    def set_field_velocity(self, now, v):
        now = np.ascontiguousarray(now, dtype=self.dtype)
        v = np.ascontiguousarray(v, dtype=self.dtype)
        rc = self._f("set_field_velocity")(self._h, _ptr(now), _ptr(v))
        if rc != 0:
            raise RuntimeError(f"orc_tcm_set_field_velocity failed: {rc}")

    def read_velocity(self) -> np.ndarray:
        out = np.zeros(self.shape, dtype=self.dtype)
        nz, ny, nx = self.shape
        rc = self._f("read_velocity")(self._h, 0, 0, 0, nx, ny, nz, _ptr(out))
        if rc != 0:
            raise RuntimeError(f"orc_tcm_read_velocity failed: {rc}")
        return out

    def active_count(self):
        nodes = np.zeros(1, np.int64)
        n = self._f("active_count")(self._h, _ptr(nodes))
        return int(n), int(nodes[0])

    def active_bricks(self) -> np.ndarray:
        n = self._f("active_bricks")(self._h, None, 0)
        ids = np.zeros(max(n, 1), np.int64)
        self._f("active_bricks")(self._h, _ptr(ids), n)
        return ids[:n].copy()

    @property
    def updates(self) -> int:
        return int(self._f("updates")(self._h))

    @property
    def step_index(self) -> int:
        return int(self._f("step_index")(self._h))

    @property
    def storage_scale(self) -> float:
        return float(self._f("storage_scale")(self._h))

    @property
    def status(self) -> int:
        return int(self._f("status")(self._h))

    def brick_media(self, b: int):
        """(1, k) for a homogenic cell, (2, None) for a bulked (heterogenic) one."""
        k = np.zeros(1, np.float64)
        r = int(self._f("brick_media")(self._h, int(b), _ptr(k)))
        return (r, float(k[0])) if r == 1 else (r, None)
