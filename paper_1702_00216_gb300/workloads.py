"""Seeded synthetic inputs for the Triggered Cells Method (Naeh, arXiv:1702.00216).

This module only *describes* inputs -- velocity models, source wavelets,
source positions, step counts and the request stream of the serving form.
It holds none of the method's arithmetic: the Eq. 3 coefficient
k = (c*dt/dx)^2, the update, the triggering and the bulking are computed
separately by the CUDA library and by the CPU oracle from these inputs.

The paper's own scenarios (a sphere beside a cube in a 340 m/s medium, a
Gaussian beam from the boundary; "Numerical stability" and "Results") are
described only in prose and figures, so the workloads below are synthetic
stand-ins with the same structure: pulse sources in large, mostly quiet
domains, homogeneous or layered media with inclusions.

Recipes (all seeds fixed):
  small      64^3, c = 1, dx = 1, dt = 0.5 (Courant 0.5), Ricker f = 1/16
             (16 cells per wavelength) at the centre, 100 steps, 8^3 cells,
             threshold 0.
  layered    512^3, 4 horizontal layers c = 1.0/1.5/2.0/2.5 (z slabs of 128),
             times (1 + p), p a Gaussian-filtered (sigma 8 cells, periodic)
             N(0,1) field from default_rng(1702) scaled to max|p| = 0.10;
             dt = 0.5/max(c); Ricker f = 1/16 at (256, 256, 64); relative
             threshold 1e-6; 20-step decay; 1500 steps.
  virtual    4096^3 (never allocated densely), c = 1 with a sphere of c = 1.8,
             radius 300, centred at (1012, 512, 512) + integer jitter in
             [-32, 32]^3 from default_rng(1702); dt = 0.5/1.8; a 3-cycle
             Ricker burst (f = 1/16) at (512, 512, 512); relative threshold
             1e-6; box pool capped at 120 GB; 2500 steps.
  precision  the small medium and source on 256^3, 800 steps.
  serving    5000 requests from default_rng(216): grid edge log-uniform in
             [64, 512], 2-6 layers with c in [1, 3], Ricker at a random node
             with 8-32 cells per wavelength, 200-3000 steps, FP32 or BF16
             storage, Poisson arrivals.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np


# --------------------------------------------------------------------------
# velocity models
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Media:
    """Velocity model: a dense array (nz, ny, nx) or rules.

    Rules: c = c_background; then for each layer (z0, c) in order, c where
    z >= z0; then for each sphere (x, y, z, r, c) in order, c where
    (i-x)^2 + (j-y)^2 + (l-z)^2 <= r^2 (node indices, FP64).
    """
    kind: str = "rules"                      # "dense" | "rules"
    c: Optional[np.ndarray] = None           # dense: float32 (nz, ny, nx)
    c_background: float = 1.0
    layers: List[Tuple[float, float]] = dataclasses.field(default_factory=list)
    spheres: List[Tuple[float, float, float, float, float]] = dataclasses.field(default_factory=list)

    def c_max(self) -> float:
        if self.kind == "dense":
            return float(np.max(self.c))
        vals = [self.c_background] + [c for _, c in self.layers] + [s[4] for s in self.spheres]
        return float(max(np.float32(v) for v in vals))


def homogeneous(c: float = 1.0) -> Media:
    return Media(kind="rules", c_background=float(c))


def dense_media(c: np.ndarray) -> Media:
    return Media(kind="dense", c=np.ascontiguousarray(c, dtype=np.float32))


def gaussian_noise_field(shape, sigma: float, seed: int, amplitude: float) -> np.ndarray:
    """N(0,1) noise from default_rng(seed), Gaussian-filtered (periodic, via FFT)
    with standard deviation `sigma` cells, scaled so that max|p| = amplitude."""
    import scipy.fft as sfft

    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(shape)
    spec = sfft.rfftn(noise, workers=-1)
    del noise
    nz, ny, nx = shape
    fz = np.fft.fftfreq(nz)[:, None, None]
    fy = np.fft.fftfreq(ny)[None, :, None]
    fx = np.fft.rfftfreq(nx)[None, None, :]
    g = np.exp(-2.0 * (math.pi ** 2) * sigma * sigma * (fz * fz + fy * fy + fx * fx))
    spec *= g
    p = sfft.irfftn(spec, s=shape, workers=-1)
    del spec
    p *= amplitude / np.max(np.abs(p))
    return p


def layered_perturbed(shape=(512, 512, 512), layer_c=(1.0, 1.5, 2.0, 2.5), sigma: float = 8.0,
                      amplitude: float = 0.10, seed: int = 1702) -> Media:
    """Horizontal layers (equal z slabs) times (1 + Gaussian-filtered noise)."""
    nz, ny, nx = shape
    p = gaussian_noise_field(shape, sigma, seed, amplitude)
    nl = len(layer_c)
    zc = np.empty(nz, dtype=np.float64)
    for m, cv in enumerate(layer_c):
        zc[m * nz // nl:(m + 1) * nz // nl] = cv
    c = (zc[:, None, None] * (1.0 + p)).astype(np.float32)
    return dense_media(c)


def random_dense_media(shape, seed: int, lo: float = 1.0, hi: float = 2.0) -> Media:
    """Uniform random c per node (small test grids)."""
    rng = np.random.default_rng(seed)
    return dense_media(rng.uniform(lo, hi, size=shape).astype(np.float32))


def sphere_inclusion_media(seed: int = 1702, centre=(1012, 512, 512), jitter: int = 32,
                           radius: float = 300.0, c_in: float = 1.8, c_out: float = 1.0) -> Media:
    rng = np.random.default_rng(seed)
    d = rng.integers(-jitter, jitter + 1, size=3)
    cx, cy, cz = (float(centre[i] + d[i]) for i in range(3))
    return Media(kind="rules", c_background=c_out, spheres=[(cx, cy, cz, float(radius), c_in)])


def random_layered_media(rng: np.random.Generator, nz: int, n_layers: int, c_lo=1.0, c_hi=3.0) -> Media:
    """n_layers horizontal layers at sorted random depths (first at z = 0)."""
    tops = np.sort(rng.integers(1, max(nz, 2), size=n_layers - 1)) if n_layers > 1 else []
    cs = rng.uniform(c_lo, c_hi, size=n_layers).astype(np.float32)
    layers = [(0.0, float(cs[0]))] + [(float(t), float(c)) for t, c in zip(tops, cs[1:])]
    return Media(kind="rules", c_background=float(cs[0]), layers=layers)


# --------------------------------------------------------------------------
# source wavelets (inputs: computed in FP64, handed to both sides)
# --------------------------------------------------------------------------
def ricker(f: float, dt: float, t0: Optional[float] = None, n: Optional[int] = None,
           amplitude: float = 1.0) -> np.ndarray:
    """Ricker wavelet A(1 - 2 pi^2 f^2 (t-t0)^2) exp(-pi^2 f^2 (t-t0)^2) at t = i*dt,
    t0 = 1.5/f by default, truncated after ceil(2 t0 / dt) samples (FP64)."""
    if t0 is None:
        t0 = 1.5 / f
    if n is None:
        n = int(math.ceil(2.0 * t0 / dt))
    t = np.arange(n, dtype=np.float64) * dt - t0
    a = (math.pi * f * t) ** 2
    return amplitude * (1.0 - 2.0 * a) * np.exp(-a)


def ricker_burst(f: float, dt: float, cycles: int = 3) -> np.ndarray:
    """Sum of `cycles` Ricker wavelets one period apart (FP64)."""
    t0 = 1.5 / f
    n = int(math.ceil((2.0 * t0 + (cycles - 1) / f) / dt))
    w = np.zeros(n, dtype=np.float64)
    for j in range(cycles):
        w += ricker(f, dt, t0=t0 + j / f, n=n)
    return w


# --------------------------------------------------------------------------
# workload configurations
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    shape: Tuple[int, int, int]              # (nz, ny, nx)
    media: Media
    dx: float
    dt: float
    sources: List[Tuple[int, int, int, np.ndarray]]   # (x, y, z, w FP64)
    steps: int
    brick: Tuple[int, int, int] = (8, 8, 8)          # (bx, by, bz)
    thr_mode: int = 0                                # 0 absolute, 1 relative
    tau: float = 0.0
    decay_alpha: float = 1.0
    decay_steps: int = 0
    pool_bytes: Optional[int] = None
    interval: int = 1                                # update procedure every `interval` steps
    neighbours: int = 6                              # 6 (faces) or 26
    lpf: Optional[Tuple[float, float]] = None        # Eq. 7 shut-down (pass, stop), else Eq. 6
    prefetch: bool = True                            # L2 prefetch in the time stepping
    cta_warps: int = 0                               # warps per CTA of the step kernel (0: 8)

    @property
    def nx(self):
        return self.shape[2]

    @property
    def ny(self):
        return self.shape[1]

    @property
    def nz(self):
        return self.shape[0]


def small(n: int = 64, steps: int = 100) -> Workload:
    """64^3 homogeneous pulse, threshold 0 (TCM must equal the dense grid)."""
    dt = 0.5
    f = 1.0 / 16.0
    c = n // 2
    return Workload("small-64^3-homogeneous-ricker", (n, n, n), homogeneous(1.0), 1.0, dt,
                    [(c, c, c, ricker(f, dt))], steps)


def layered(n: int = 512, steps: int = 1500, media: Optional[Media] = None) -> Workload:
    """512^3 layered + perturbed medium, relative threshold 1e-6, 20-step decay."""
    if media is None:
        media = layered_perturbed((n, n, n))
    dt = 0.5 / media.c_max()
    f = 1.0 / 16.0
    src = (n // 2, n // 2, n // 8)
    return Workload(f"layered-{n}^3-perturbed-ricker", (n, n, n), media, 1.0, dt,
                    [(src[0], src[1], src[2], ricker(f, dt))], steps,
                    thr_mode=1, tau=1e-6, decay_alpha=0.8, decay_steps=20)


def virtual(n: int = 4096, steps: int = 2500, pool_bytes: int = 120 * 2**30) -> Workload:
    """Virtual 4096^3 domain with a spherical inclusion, 3-cycle Ricker burst."""
    media = sphere_inclusion_media()
    dt = 0.5 / media.c_max()
    f = 1.0 / 16.0
    return Workload(f"virtual-{n}^3-sphere-burst", (n, n, n), media, 1.0, dt,
                    [(512, 512, 512, ricker_burst(f, dt, 3))], steps,
                    thr_mode=1, tau=1e-6, decay_alpha=0.8, decay_steps=20, pool_bytes=pool_bytes)


def gaussian_derivative(sigma: float, dt: float, t0: Optional[float] = None) -> np.ndarray:
    """Bi-polar pulse: the derivative of a Gaussian, -(t - t0)/sigma * exp(-(t - t0)^2 /
    (2 sigma^2)) at t = i*dt, t0 = 4 sigma, truncated after 2 t0 (peak 1/sqrt(e); FP64)."""
    if t0 is None:
        t0 = 4.0 * sigma
    n = int(math.ceil(2.0 * t0 / dt))
    t = np.arange(n, dtype=np.float64) * dt - t0
    return -(t / sigma) * np.exp(-0.5 * (t / sigma) ** 2)


def scatterer(shape=(64, 64, 112), steps: int = 260, beam_sigma: float = 5.0, pulse_sigma: float = 0.01,
              threshold: float = 0.0) -> Workload:
    """The sound-soft scatterer scenario of the stability study, scaled down: c = 340 m/s,
    dx = 1 m, dt = 1e-3 s (Courant 0.34); a sphere beside a cube, both with c = 0 (k = 0,
    so their nodes never leave zero); a directional Gaussian beam from the x- boundary:
    point sources on the plane x = 2 with Gaussian weights (sigma = beam_sigma cells),
    all fed the derivative of a Gaussian (sigma = pulse_sigma s)."""
    nz, ny, nx = shape
    c = np.full(shape, 340.0, dtype=np.float64)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cx, cy, cz, r = nx * 0.55, ny * 0.5, nz * 0.42, min(nx, ny, nz) * 0.14
    c[(x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2 <= r * r] = 0.0
    half = r * 0.9
    cube = (np.abs(x - cx) <= half) & (np.abs(y - cy) <= half) & (z >= cz + r - 1) & (z <= cz + r - 1 + 2 * half)
    c[cube] = 0.0
    dt = 1e-3
    w = gaussian_derivative(pulse_sigma, dt)
    srcs = []
    for yy in range(ny):
        for zz in range(nz):
            g = math.exp(-((yy - cy) ** 2 + (zz - cz) ** 2) / (2 * beam_sigma ** 2))
            if g > 0.1:
                srcs.append((2, yy, zz, w * g))
    return Workload(f"scatterer-{nx}x{ny}x{nz}-beam", shape, dense_media(c), 1.0, dt, srcs, steps,
                    thr_mode=1 if threshold > 0 else 0, tau=threshold)


def precision(n: int = 256, steps: int = 800) -> Workload:
    """The medium and source of small() -- homogeneous c = 1, dx = 1, dt = 0.5,
    Ricker f = 1/16 at the grid centre -- on a 256^3 grid, with the relative
    threshold 1e-6 and 20-step decay of layered() (the storage-precision
    comparison)."""
    dt = 0.5
    f = 1.0 / 16.0
    c = n // 2
    return Workload(f"precision-{n}^3-homogeneous-ricker", (n, n, n), homogeneous(1.0), 1.0, dt,
                    [(c, c, c, ricker(f, dt))], steps,
                    thr_mode=1, tau=1e-6, decay_alpha=0.8, decay_steps=20)


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float                # seconds after the stream starts
    workload: Workload
    storage: str                  # "f32" | "bf16"


def serving_stream(n_requests: int = 5000, seed: int = 216, rate_hz: float = 50.0,
                   edge_lo: int = 64, edge_hi: int = 512, steps_lo: int = 200,
                   steps_hi: int = 3000, bf16_fraction: float = 0.5) -> List[Request]:
    """Poisson-arrival stream of simulation requests (serving form)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for rid in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        edge = int(round(math.exp(rng.uniform(math.log(edge_lo), math.log(edge_hi)))))
        nl = int(rng.integers(2, 7))
        media = random_layered_media(rng, edge, nl)
        dt = 0.5 / media.c_max()
        x, y, z = (int(v) for v in rng.integers(0, edge, size=3))
        cells_per_wl = rng.uniform(8.0, 32.0)
        f = media.c_max() / cells_per_wl
        steps = int(rng.integers(steps_lo, steps_hi + 1))
        storage = "bf16" if rng.uniform() < bf16_fraction else "f32"
        wl = Workload(f"req{rid}", (edge, edge, edge), media, 1.0, dt,
                      [(x, y, z, ricker(f, dt))], steps)
        out.append(Request(rid, t, wl, storage))
    return out


def eigenmode(shape, p: Sequence[int]) -> np.ndarray:
    """Dirichlet eigenvector sin(pi p_x (i+1)/(nx+1)) sin(..y..) sin(..z..) (FP64),
    an input for the dispersion and energy checks."""
    nz, ny, nx = shape
    px, py, pz = p
    sx = np.sin(math.pi * px * (np.arange(nx) + 1) / (nx + 1))
    sy = np.sin(math.pi * py * (np.arange(ny) + 1) / (ny + 1))
    sz = np.sin(math.pi * pz * (np.arange(nz) + 1) / (nz + 1))
    return sz[:, None, None] * sy[None, :, None] * sx[None, None, :]
