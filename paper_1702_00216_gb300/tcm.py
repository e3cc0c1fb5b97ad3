"""Thin ctypes binding of libtcm (C ABI in include/tcm.h).

Argument marshalling only: every step of the method runs in the CUDA library.
The module-level functions carry the C names; ``Sim`` bundles them for
convenience.  PyTorch, when present, only provides the device memory of the
box pool and the CUDA stream.  There is no CPU fallback: if the library has
not been built, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# TCM_CHECKED=1: the bounds-checked build of the same sources (see build.py)
LIB_PATH = os.path.join(HERE, "libtcm_checked.so" if os.environ.get("TCM_CHECKED", "") == "1" else "libtcm.so")

TCM_OK, TCM_EINVAL, TCM_ECFL, TCM_ENOMEM, TCM_EDEVICE, TCM_ETIMEOUT, TCM_ESTATE = range(7)
TCM_MEDIA_DENSE, TCM_MEDIA_RULES = 0, 1
TCM_THR_ABSOLUTE, TCM_THR_RELATIVE = 0, 1
TCM_STORAGE_F32, TCM_STORAGE_BF16, TCM_STORAGE_F16, TCM_STORAGE_MIXED = 0, 1, 2, 3
STORAGES = {"f32": TCM_STORAGE_F32, "bf16": TCM_STORAGE_BF16, "f16": TCM_STORAGE_F16, "mixed": TCM_STORAGE_MIXED}


def storage_code(storage) -> int:
    """TCM_STORAGE_* from a code or a name ('f32', 'bf16', 'f16')."""
    return STORAGES[storage] if isinstance(storage, str) else int(storage)

EXPORTS = ["tcm_slot_bytes", "tcm_create", "tcm_add_source", "tcm_set_field", "tcm_step",
           "tcm_step_async", "tcm_sync", "tcm_set_schedule", "tcm_schedule", "tcm_set_lpf_shutdown", "tcm_read_field", "tcm_read_field_device",
           "tcm_active_count", "tcm_active_bricks", "tcm_updates", "tcm_energy",
           "tcm_energy_noalloc",
           "tcm_brick_media", "tcm_pool_info", "tcm_phase_ns", "tcm_launch_count", "tcm_graph_launch_count", "tcm_step_index",
           "tcm_status_string", "tcm_destroy", "tcm_batch_create", "tcm_batch_add",
           "tcm_batch_step", "tcm_batch_step_async", "tcm_batch_sync", "tcm_sim_done",
           "tcm_batch_remove", "tcm_batch_info", "tcm_batch_destroy", "tcm_barrier_selftest",
           "tcm_set_storage", "tcm_batch_pause", "tcm_batch_resume", "tcm_batch_headroom", "tcm_lpf_info"]


class tcm_domain(C.Structure):
    _fields_ = [("nx", C.c_int64), ("ny", C.c_int64), ("nz", C.c_int64)]


class tcm_velocity_model(C.Structure):
    _fields_ = [("kind", C.c_int), ("c", C.c_void_p), ("c_background", C.c_float),
                ("n_layers", C.c_int), ("layer_z", C.c_void_p), ("layer_c", C.c_void_p),
                ("n_spheres", C.c_int), ("sphere_xyzr", C.c_void_p), ("sphere_c", C.c_void_p)]


class tcm_brick(C.Structure):
    _fields_ = [("bx", C.c_int), ("by", C.c_int), ("bz", C.c_int)]


class tcm_options(C.Structure):
    _fields_ = [("threshold_mode", C.c_int), ("decay_alpha", C.c_float), ("decay_steps", C.c_int),
                ("pool_ptr", C.c_void_p), ("pool_bytes", C.c_size_t), ("stream", C.c_void_p),
                ("storage", C.c_int), ("dense", C.c_int), ("device", C.c_int), ("no_graphs", C.c_int),
                ("no_prefetch", C.c_int), ("cta_warps", C.c_int)]


class tcm_batch_options(C.Structure):
    _fields_ = [("pool_ptr", C.c_void_p), ("pool_bytes", C.c_size_t), ("stream", C.c_void_p),
                ("device", C.c_int), ("storage", C.c_int), ("max_bricks", C.c_int64),
                ("max_sims", C.c_int), ("no_graphs", C.c_int), ("brick", tcm_brick), ("no_prefetch", C.c_int),
                ("cta_warps", C.c_int)]


class TCMError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {tcm_status_string(status)} ({status})")


_LIB = None
_vp, _i64 = C.c_void_p, C.c_int64


def lib():
    """The loaded libtcm.so.  Raises if it has not been built (no fallback)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: run __graft_entry__.build() "
                               "(the CUDA library is the only implementation)")
        L = C.CDLL(LIB_PATH)
        sig = {
            "tcm_slot_bytes": ([tcm_brick, C.c_int, _vp], C.c_int),
            "tcm_create": ([_vp, _vp, C.c_double, C.c_double, C.c_double, tcm_brick, _vp, _vp], C.c_int),
            "tcm_add_source": ([_vp, _i64, _i64, _i64, _vp, _i64], C.c_int),
            "tcm_set_field": ([_vp, _vp, _vp], C.c_int),
            "tcm_set_schedule": ([_vp, C.c_int, C.c_int], C.c_int),
            "tcm_schedule": ([_vp, _vp, _vp], C.c_int),
            "tcm_set_lpf_shutdown": ([_vp, C.c_double, C.c_double], C.c_int),
            "tcm_step": ([_vp, _i64], C.c_int),
            "tcm_step_async": ([_vp, _i64], C.c_int),
            "tcm_sync": ([_vp], C.c_int),
            "tcm_read_field": ([_vp, C.c_int, _i64, _i64, _i64, _i64, _i64, _i64, _vp], C.c_int),
            "tcm_read_field_device": ([_vp, C.c_int, _i64, _i64, _i64, _i64, _i64, _i64, _vp], C.c_int),
            "tcm_active_count": ([_vp, _vp, _vp], C.c_int),
            "tcm_active_bricks": ([_vp, _vp, _i64, _vp], C.c_int),
            "tcm_updates": ([_vp, _vp], C.c_int),
            "tcm_energy": ([_vp, _vp], C.c_int),
            "tcm_energy_noalloc": ([_vp, _vp], C.c_int),
            "tcm_brick_media": ([_vp, _i64, _vp, _vp], C.c_int),
            "tcm_pool_info": ([_vp, _vp, _vp], C.c_int),
            "tcm_phase_ns": ([_vp, _vp, _vp, _vp], C.c_int),
            "tcm_launch_count": ([_vp], _i64),
            "tcm_graph_launch_count": ([_vp], _i64),
            "tcm_step_index": ([_vp], _i64),
            "tcm_status_string": ([C.c_int], C.c_char_p),
            "tcm_destroy": ([_vp], None),
            "tcm_batch_create": ([_vp, _vp], C.c_int),
            "tcm_batch_add": ([_vp, _vp, _vp, C.c_double, C.c_double, C.c_double, tcm_brick, C.c_int,
                               C.c_float, C.c_int, C.c_int, _i64, _vp], C.c_int),
            "tcm_batch_step": ([_vp, _i64], C.c_int),
            "tcm_batch_step_async": ([_vp, _i64], C.c_int),
            "tcm_batch_sync": ([_vp], C.c_int),
            "tcm_sim_done": ([_vp, _vp], C.c_int),
            "tcm_batch_remove": ([_vp, _vp], C.c_int),
            "tcm_batch_info": ([_vp, _vp, _vp, _vp], C.c_int),
            "tcm_batch_destroy": ([_vp], None),
            "tcm_barrier_selftest": ([C.c_int, C.c_int, C.c_double, _vp], C.c_int),
            "tcm_set_storage": ([_vp, C.c_int], C.c_int),
            "tcm_batch_pause": ([_vp], C.c_int),
            "tcm_batch_resume": ([_vp], C.c_int),
            "tcm_batch_headroom": ([_vp, _i64, _vp], C.c_int),
            "tcm_lpf_info": ([_vp, _vp, _vp, _vp], C.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _LIB = L
    return _LIB


def tcm_barrier_selftest(device: int = 0, skew: int = 0, timeout_s: float = 0.05):
    """Run the bounded device-wide barrier once (skew 1: one arrival missing);
    returns (status, device error bits) without raising."""
    err = C.c_uint(0)
    rc = lib().tcm_barrier_selftest(int(device), int(skew), float(timeout_s), C.byref(err))
    return int(rc), int(err.value)


def _chk(rc: int, what: str):
    if rc != TCM_OK:
        raise TCMError(rc, what)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_vp)


# ---- the C functions, same names --------------------------------------------
def tcm_status_string(status: int) -> str:
    return lib().tcm_status_string(int(status)).decode()


def tcm_slot_bytes(brick=(8, 8, 8), storage: int = TCM_STORAGE_F32) -> int:
    out = C.c_size_t(0)
    _chk(lib().tcm_slot_bytes(tcm_brick(*brick), storage, C.byref(out)), "tcm_slot_bytes")
    return int(out.value)


def velocity_model(media):
    """tcm_velocity_model for a workloads.Media (keeps its arrays alive)."""
    keep = []
    vm = tcm_velocity_model()
    if media.kind == "dense":
        c = np.ascontiguousarray(media.c, dtype=np.float32)
        keep.append(c)
        vm.kind = TCM_MEDIA_DENSE
        vm.c = c.ctypes.data
    else:
        vm.kind = TCM_MEDIA_RULES
        vm.c_background = float(media.c_background)
        lz = np.ascontiguousarray([z for z, _ in media.layers], dtype=np.float64)
        lc = np.ascontiguousarray([c for _, c in media.layers], dtype=np.float32)
        sp = np.ascontiguousarray([s[:4] for s in media.spheres], dtype=np.float64).reshape(-1)
        sc = np.ascontiguousarray([s[4] for s in media.spheres], dtype=np.float32)
        keep += [lz, lc, sp, sc]
        vm.n_layers = len(lc)
        vm.layer_z = lz.ctypes.data if len(lc) else None
        vm.layer_c = lc.ctypes.data if len(lc) else None
        vm.n_spheres = len(sc)
        vm.sphere_xyzr = sp.ctypes.data if len(sc) else None
        vm.sphere_c = sc.ctypes.data if len(sc) else None
    return vm, keep


def tcm_create(shape, media, dx, dt, threshold, brick, options) -> int:
    nz, ny, nx = shape
    dom = tcm_domain(nx, ny, nz)
    vm, keep = velocity_model(media)
    out = _vp()
    rc = lib().tcm_create(C.byref(dom), C.byref(vm), float(dx), float(dt), float(threshold),
                          tcm_brick(*brick), C.byref(options), C.byref(out))
    del keep
    _chk(rc, "tcm_create")
    return out.value


def tcm_add_source(h, x, y, z, wavelet):
    w = np.ascontiguousarray(wavelet, dtype=np.float32)
    _chk(lib().tcm_add_source(h, int(x), int(y), int(z), _ptr(w), len(w)), "tcm_add_source")


def tcm_set_field(h, now, prev):
    now = np.ascontiguousarray(now, dtype=np.float32)
    prev = np.ascontiguousarray(prev, dtype=np.float32)
    _chk(lib().tcm_set_field(h, _ptr(now), _ptr(prev)), "tcm_set_field")


def tcm_set_schedule(h, interval=1, neighbours=6):
    _chk(lib().tcm_set_schedule(h, int(interval), int(neighbours)), "tcm_set_schedule")


def tcm_set_lpf_shutdown(h, pass_, stop):
    _chk(lib().tcm_set_lpf_shutdown(h, float(pass_), float(stop)), "tcm_set_lpf_shutdown")


def tcm_schedule(h):
    iv, nb = C.c_int(0), C.c_int(0)
    _chk(lib().tcm_schedule(h, C.byref(iv), C.byref(nb)), "tcm_schedule")
    return iv.value, nb.value


def tcm_step(h, n=1):
    _chk(lib().tcm_step(h, int(n)), "tcm_step")


def tcm_step_async(h, n=1):
    _chk(lib().tcm_step_async(h, int(n)), "tcm_step_async")


def tcm_sync(h):
    _chk(lib().tcm_sync(h), "tcm_sync")


def tcm_read_field(h, which, origin, size) -> np.ndarray:
    wx, wy, wz = (int(v) for v in size)
    out = np.zeros((wz, wy, wx), dtype=np.float32)
    _chk(lib().tcm_read_field(h, int(which), int(origin[0]), int(origin[1]), int(origin[2]),
                              wx, wy, wz, _ptr(out)), "tcm_read_field")
    return out


def tcm_read_field_device(h, which, origin, size, device_ptr: int):
    wx, wy, wz = (int(v) for v in size)
    _chk(lib().tcm_read_field_device(h, int(which), int(origin[0]), int(origin[1]),
                                     int(origin[2]), wx, wy, wz, _vp(device_ptr)),
         "tcm_read_field_device")


def tcm_active_count(h):
    b, c = C.c_int64(0), C.c_int64(0)
    _chk(lib().tcm_active_count(h, C.byref(b), C.byref(c)), "tcm_active_count")
    return b.value, c.value


def tcm_active_bricks(h) -> np.ndarray:
    n = C.c_int64(0)
    _chk(lib().tcm_active_bricks(h, None, 0, C.byref(n)), "tcm_active_bricks")
    ids = np.zeros(max(n.value, 1), np.int64)
    _chk(lib().tcm_active_bricks(h, _ptr(ids), n.value, C.byref(n)), "tcm_active_bricks")
    return ids[:n.value].copy()


def tcm_updates(h) -> int:
    u = C.c_int64(0)
    _chk(lib().tcm_updates(h, C.byref(u)), "tcm_updates")
    return u.value


def tcm_energy(h) -> float:
    e = C.c_double(0)
    _chk(lib().tcm_energy(h, C.byref(e)), "tcm_energy")
    return e.value


def tcm_energy_noalloc(h, device_out_ptr: int):
    """Energy into one device double at device_out_ptr; allocates nothing."""
    _chk(lib().tcm_energy_noalloc(h, _vp(device_out_ptr)), "tcm_energy_noalloc")


def tcm_brick_media(h, b):
    kind, k = C.c_int(0), C.c_float(0)
    _chk(lib().tcm_brick_media(h, int(b), C.byref(kind), C.byref(k)), "tcm_brick_media")
    return (1, float(k.value)) if kind.value == 1 else (2, None)


def tcm_pool_info(h):
    s, f = C.c_int64(0), C.c_int64(0)
    _chk(lib().tcm_pool_info(h, C.byref(s), C.byref(f)), "tcm_pool_info")
    return s.value, f.value


def tcm_phase_ns(h):
    """(time stepping, updating active cells, compaction) cumulative device ns."""
    a, b, c = C.c_int64(0), C.c_int64(0), C.c_int64(0)
    _chk(lib().tcm_phase_ns(h, C.byref(a), C.byref(b), C.byref(c)), "tcm_phase_ns")
    return a.value, b.value, c.value


def tcm_lpf_info(h):
    """(ns, bricks filtered, binary32 multiply-adds per brick) of the Eq. 7 filter so far."""
    a, b, c = C.c_int64(0), C.c_int64(0), C.c_int64(0)
    _chk(lib().tcm_lpf_info(h, C.byref(a), C.byref(b), C.byref(c)), "tcm_lpf_info")
    return a.value, b.value, c.value


def tcm_launch_count(h) -> int:
    return int(lib().tcm_launch_count(h))


def tcm_step_index(h) -> int:
    return int(lib().tcm_step_index(h))


def tcm_destroy(h):
    lib().tcm_destroy(h)


def tcm_batch_create(options) -> int:
    out = _vp()
    _chk(lib().tcm_batch_create(C.byref(options), C.byref(out)), "tcm_batch_create")
    return out.value


def tcm_batch_add(b, shape, media, dx, dt, threshold, brick, thr_mode, decay_alpha, decay_steps,
                  dense=False, n_steps=0) -> int:
    nz, ny, nx = shape
    dom = tcm_domain(nx, ny, nz)
    vm, keep = velocity_model(media)
    out = _vp()
    rc = lib().tcm_batch_add(b, C.byref(dom), C.byref(vm), float(dx), float(dt), float(threshold),
                             tcm_brick(*brick), int(thr_mode), float(decay_alpha), int(decay_steps),
                             int(bool(dense)), int(n_steps), C.byref(out))
    del keep
    _chk(rc, "tcm_batch_add")
    return out.value


def tcm_batch_step(b, n=1):
    _chk(lib().tcm_batch_step(b, int(n)), "tcm_batch_step")


def tcm_batch_step_async(b, n=1):
    _chk(lib().tcm_batch_step_async(b, int(n)), "tcm_batch_step_async")


def tcm_batch_sync(b):
    _chk(lib().tcm_batch_sync(b), "tcm_batch_sync")


def tcm_sim_done(h) -> bool:
    d = C.c_int(0)
    _chk(lib().tcm_sim_done(h, C.byref(d)), "tcm_sim_done")
    return bool(d.value)


def tcm_batch_remove(b, h):
    _chk(lib().tcm_batch_remove(b, h), "tcm_batch_remove")


def tcm_batch_info(b):
    s, f, n = C.c_int64(0), C.c_int64(0), C.c_int(0)
    _chk(lib().tcm_batch_info(b, C.byref(s), C.byref(f), C.byref(n)), "tcm_batch_info")
    return s.value, f.value, n.value


def tcm_batch_destroy(b):
    lib().tcm_batch_destroy(b)


def tcm_set_storage(h, storage):
    _chk(lib().tcm_set_storage(h, storage_code(storage)), "tcm_set_storage")


def tcm_batch_pause(h):
    _chk(lib().tcm_batch_pause(h), "tcm_batch_pause")


def tcm_batch_resume(h):
    _chk(lib().tcm_batch_resume(h), "tcm_batch_resume")


def tcm_batch_headroom(b, steps) -> int:
    n = C.c_int64(0)
    _chk(lib().tcm_batch_headroom(b, int(steps), C.byref(n)), "tcm_batch_headroom")
    return n.value


# ---- convenience wrapper ----------------------------------------------------
def _torch():
    try:
        import torch
        return torch
    except Exception:  # pragma: no cover
        return None


class Sim:
    """One simulation on the GPU (tcm_create ... tcm_destroy)."""

    def __init__(self, shape, media, dx, dt, threshold=0.0, brick=(8, 8, 8),
                 thr_mode=TCM_THR_ABSOLUTE, decay_alpha=1.0, decay_steps=0, pool_bytes=None,
                 dense=False, device=0, stream=None, pool_tensor=None, storage=TCM_STORAGE_F32,
                 graphs=True, prefetch=True, cta_warps=0):
        self.shape = tuple(int(v) for v in shape)
        self.storage = storage_code(storage)
        nz, ny, nx = self.shape
        bx, by, bz = brick
        self.brick = (bx, by, bz)
        self.mx, self.my, self.mz = -(-nx // bx), -(-ny // by), -(-nz // bz)
        slot = tcm_slot_bytes(brick, self.storage)
        if pool_bytes is None:
            pool_bytes = self.mx * self.my * self.mz * slot
        torch = _torch()
        self._pool = None
        opts = tcm_options()
        opts.threshold_mode = int(thr_mode)
        opts.decay_alpha = float(decay_alpha)
        opts.decay_steps = int(decay_steps)
        opts.pool_bytes = int(pool_bytes)
        opts.storage = self.storage
        opts.no_graphs = 0 if graphs else 1
        opts.no_prefetch = 0 if prefetch else 1
        opts.cta_warps = int(cta_warps)
        opts.dense = int(bool(dense))
        opts.device = int(device)
        if pool_tensor is not None:
            self._pool = pool_tensor
            opts.pool_ptr = int(pool_tensor.data_ptr())
            opts.pool_bytes = int(pool_tensor.numel() * pool_tensor.element_size())
        elif torch is not None and torch.cuda.is_available():
            self._pool = torch.empty(int(pool_bytes), dtype=torch.uint8, device=f"cuda:{device}")
            opts.pool_ptr = int(self._pool.data_ptr())
        if stream is None and torch is not None and torch.cuda.is_available():
            stream = torch.cuda.current_stream(device).cuda_stream
        opts.stream = stream or None
        self._h = None
        self._h = tcm_create(self.shape, media, dx, dt, threshold, brick, opts)

    @classmethod
    def _wrap(cls, handle, shape, brick):
        s = cls.__new__(cls)
        s.shape = tuple(int(v) for v in shape)
        nz, ny, nx = s.shape
        bx, by, bz = brick
        s.brick = (bx, by, bz)
        s.mx, s.my, s.mz = -(-nx // bx), -(-ny // by), -(-nz // bz)
        s._pool = None
        s._h = handle
        s._borrowed = True
        return s

    @classmethod
    def from_workload(cls, wl, dense=False, **kw):
        pool = kw.pop("pool_bytes", wl.pool_bytes)
        kw.setdefault("prefetch", wl.prefetch)
        kw.setdefault("cta_warps", getattr(wl, "cta_warps", 0))
        s = cls(wl.shape, wl.media, wl.dx, wl.dt, threshold=wl.tau, brick=wl.brick,
                thr_mode=wl.thr_mode, decay_alpha=wl.decay_alpha, decay_steps=wl.decay_steps,
                pool_bytes=pool, dense=dense, **kw)
        for x, y, z, w in wl.sources:
            s.add_source(x, y, z, np.asarray(w, dtype=np.float32))
        if (wl.interval, wl.neighbours) != (1, 6):
            s.set_schedule(wl.interval, wl.neighbours)
        if wl.lpf is not None:
            s.set_lpf_shutdown(*wl.lpf)
        return s

    @property
    def handle(self):
        return self._h

    def add_source(self, x, y, z, w):
        tcm_add_source(self._h, x, y, z, w)

    def set_field(self, now, prev):
        tcm_set_field(self._h, now, prev)

    def set_schedule(self, interval=1, neighbours=6):
        tcm_set_schedule(self._h, interval, neighbours)

    def schedule(self):
        return tcm_schedule(self._h)

    def set_lpf_shutdown(self, pass_, stop):
        tcm_set_lpf_shutdown(self._h, pass_, stop)

    def step(self, n=1):
        tcm_step(self._h, n)

    def step_async(self, n=1):
        tcm_step_async(self._h, n)

    def sync(self):
        tcm_sync(self._h)

    def read_field(self, which=0, origin=(0, 0, 0), size=None):
        if size is None:
            size = (self.shape[2], self.shape[1], self.shape[0])
        return tcm_read_field(self._h, which, origin, size)

    def active_count(self):
        return tcm_active_count(self._h)

    def active_bricks(self):
        return tcm_active_bricks(self._h)

    @property
    def updates(self):
        return tcm_updates(self._h)

    def energy(self):
        return tcm_energy(self._h)

    def brick_media(self, b):
        return tcm_brick_media(self._h, b)

    def pool_info(self):
        return tcm_pool_info(self._h)

    def phase_ns(self):
        return tcm_phase_ns(self._h)

    @property
    def launches(self):
        return tcm_launch_count(self._h)

    def graph_launches(self):
        return int(lib().tcm_graph_launch_count(self._h))

    @property
    def step_index(self):
        return tcm_step_index(self._h)

    def done(self):
        return tcm_sim_done(self._h)

    def close(self):
        if self._h and not getattr(self, "_borrowed", False):
            tcm_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Many simulations stepped together by one launch per step (tcm_batch_*)."""

    def __init__(self, pool_bytes, max_bricks, max_sims=64, device=0, stream=None,
                 pool_tensor=None, storage=TCM_STORAGE_F32, graphs=True, brick=(8, 8, 8), prefetch=True,
                 cta_warps=0):
        torch = _torch()
        self.storage = storage_code(storage)
        self.brick = tuple(int(v) for v in brick)
        o = tcm_batch_options()
        o.no_graphs = 0 if graphs else 1
        o.no_prefetch = 0 if prefetch else 1
        o.cta_warps = int(cta_warps)
        o.brick = tcm_brick(*self.brick)
        o.pool_bytes = int(pool_bytes)
        o.device = int(device)
        o.storage = self.storage
        o.max_bricks = int(max_bricks)
        o.max_sims = int(max_sims)
        self._pool = None
        if pool_tensor is not None:
            self._pool = pool_tensor
        elif torch is not None and torch.cuda.is_available():
            self._pool = torch.empty(int(pool_bytes), dtype=torch.uint8, device=f"cuda:{device}")
        if self._pool is not None:
            o.pool_ptr = int(self._pool.data_ptr())
            o.pool_bytes = int(self._pool.numel() * self._pool.element_size())
        if stream is None and torch is not None and torch.cuda.is_available():
            stream = torch.cuda.current_stream(device).cuda_stream
        o.stream = stream or None
        self._h = None
        self._h = tcm_batch_create(o)
        self._sims = []

    def add(self, wl, n_steps=0, dense=False, storage=None):
        """Add a workloads.Workload (with its sources); returns a Sim bound to the
        batch.  storage: the simulation's field storage in a mixed batch."""
        h = tcm_batch_add(self._h, wl.shape, wl.media, wl.dx, wl.dt, wl.tau, wl.brick, wl.thr_mode,
                          wl.decay_alpha, wl.decay_steps, dense=dense, n_steps=n_steps)
        sim = Sim._wrap(h, wl.shape, wl.brick)
        if storage is not None:
            tcm_set_storage(h, storage)
        for x, y, z, w in wl.sources:
            sim.add_source(x, y, z, np.asarray(w, dtype=np.float32))
        if (getattr(wl, "interval", 1), getattr(wl, "neighbours", 6)) != (1, 6):
            sim.set_schedule(wl.interval, wl.neighbours)
        if getattr(wl, "lpf", None) is not None:
            sim.set_lpf_shutdown(*wl.lpf)
        self._sims.append(sim)
        return sim

    def step(self, n=1):
        tcm_batch_step(self._h, n)

    def step_async(self, n=1):
        tcm_batch_step_async(self._h, n)

    def sync(self):
        tcm_batch_sync(self._h)

    def remove(self, sim):
        tcm_batch_remove(self._h, sim._h)
        sim._h = None
        self._sims = [s for s in self._sims if s is not sim]

    def info(self):
        """(boxes in the pool, free boxes, simulations alive)."""
        return tcm_batch_info(self._h)

    def pause(self, sim):
        tcm_batch_pause(sim._h)

    def resume(self, sim):
        tcm_batch_resume(sim._h)

    def headroom(self, steps) -> int:
        """Upper bound on the boxes the stepping simulations can claim in `steps` steps."""
        return tcm_batch_headroom(self._h, steps)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            for s in self._sims:
                s._h = None
            tcm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
