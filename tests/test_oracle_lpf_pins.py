"""Pins of the oracle's frequency-domain shut-down (Eq. 7).

The transform is pinned to numpy's FFT, the filter response to its
definition's fixed points, the region filter to the same definition built on
numpy's FFT, and the shut-down itself to (a) the dense grid at threshold 0
(releasing all-zero cells filters nothing), (b) a worked release whose
filtered neighbours are recomputed from the dense step with numpy's FFT, and
(c) its purpose: less high-frequency content than a hard release.
"""
import numpy as np
import pytest

import oracle
from paper_1702_00216_gb300 import workloads as W

F32 = np.float32


@pytest.mark.parametrize("n", [1, 2, 4, 8, 64, 256])
def test_fft_matches_numpy(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert np.allclose(oracle.fft(x, -1), np.fft.fft(x), atol=1e-12 * n)
    assert np.allclose(oracle.fft(x, 1) / n, np.fft.ifft(x), atol=1e-12)


def test_lpf_response_fixed_points():
    M, p, s = 64, 0.25, 0.5
    h = np.array([oracle.lpf_response(k, M, p, s) for k in range(M)])
    assert h[0] == 1.0 and h[8] == 1.0 and h[16] == 0.0 and h[32] == 0.0   # nu = 0, .25, .5, 1
    assert np.array_equal(h[1:], h[1:][::-1])                             # H(k) = H(M - k)
    assert abs(h[12] - 0.5) < 1e-15                                        # nu = 0.375: mid-taper
    assert np.all(np.diff(h[:33]) <= 0)


def numpy_region(v, M, p, s):
    L = v.shape[0]
    pad = np.zeros((M, M, M))
    pad[:L, :L, :L] = v
    k = np.minimum(np.arange(M), M - np.arange(M)) / (M / 2)
    h = np.where(k <= p, 1.0, np.where(k >= s, 0.0, 0.5 * (1 + np.cos(np.pi * (k - p) / (s - p)))))
    H = h[:, None, None] * h[None, :, None] * h[None, None, :]
    return np.real(np.fft.ifftn(np.fft.fftn(pad) * H))[:L, :L, :L]


def test_region_filter_matches_numpy_definition():
    rng = np.random.default_rng(7)
    v = rng.standard_normal((24, 24, 24))
    got = oracle.lpf_region(v, 64, 0.3, 0.6)
    assert np.allclose(got, numpy_region(v, 64, 0.3, 0.6), atol=1e-12)
    # transposed axes would fail on an anisotropic input
    a = np.zeros((24, 24, 24))
    a[:, :, ::2] = 1.0
    assert not np.allclose(oracle.lpf_region(a, 64, 0.3, 0.6),
                           oracle.lpf_region(a.transpose(2, 1, 0), 64, 0.3, 0.6))


def test_region_filter_passes_low_and_removes_nyquist():
    L, M = 24, 64
    z, y, x = np.meshgrid(*(np.arange(L),) * 3, indexing="ij")
    env = np.exp(-((x - 11.5) ** 2 + (y - 11.5) ** 2 + (z - 11.5) ** 2) / (2 * 4.0 ** 2))
    low = env * np.cos(np.pi * 0.08 * x)                  # nu = 0.08 << pass
    out = oracle.lpf_region(low, M, 0.3, 0.6)
    c = slice(8, 16)
    assert np.abs(out[c, c, c] - low[c, c, c]).max() < 1e-3 * np.abs(low).max()
    nyq = (-1.0) ** (x + y + z)
    assert np.abs(oracle.lpf_region(nyq, M, 0.3, 0.6)[c, c, c]).max() < 1e-6   # edges of the padding leak a little


def test_lpf_threshold0_equals_dense():
    shape = (26, 30, 35)
    m = W.random_dense_media(shape, 8, 1.0, 2.0)
    dt = 0.5 / m.c_max()
    w = W.ricker(1 / 8, dt).astype(F32)
    k = oracle.k_from_c(m.c, dt, 1.0, F32)
    z = np.zeros(shape, F32)
    a, _ = oracle.dense_run(k, z, z, 60, sources=[(6, 20, 9, w), (30, 3, 20, w[:20])])
    for interval, nb in ((1, 6), (4, 26)):
        t = oracle.OracleTCM(shape, m, 1.0, dt, interval=interval, neighbours=nb, lpf=(0.25, 0.5))
        t.add_source(6, 20, 9, w)
        t.add_source(30, 3, 20, w[:20])
        t.step(60)
        assert np.array_equal(t.read_field(0), a)


def released_scenario(lpf):
    """3^3 cells of 8^3: a hot centre cell, a weak corner cell below the level
    (released after step 0), the centre's face neighbours boxed by the update
    on the initial state."""
    shape = (24, 24, 24)
    rng = np.random.default_rng(11)
    now = np.zeros(shape, F32)
    now[8:16, 8:16, 8:16] = rng.uniform(0.5, 1.0, (8, 8, 8)).astype(F32)
    now[0:8, 0:8, 0:8] = rng.uniform(-0.05, 0.05, (8, 8, 8)).astype(F32)
    prev = (now * F32(0.9)).astype(F32)
    t = oracle.OracleTCM(shape, W.homogeneous(1.0), 1.0, 0.5, tau=0.2, lpf=lpf)
    t.set_field(now, prev)
    return t, now, prev


def test_lpf_worked_release_matches_numpy():
    t, now, prev = released_scenario((0.25, 0.5))
    t.step(1)
    ids = set(t.active_bricks().tolist())
    assert 0 not in ids and 13 in ids          # corner released, centre kept
    k = oracle.k_from_c(np.ones(now.shape, F32), 0.5, 1.0, F32)
    a, b = oracle.dense_run(k, now, prev, 1)  # phi^1, phi^0 before the update
    boxed = np.zeros((3, 3, 3), bool)
    for c in (13, 4, 10, 12, 14, 16, 22):      # centre + its six face neighbours
        boxed[c // 9, (c // 3) % 3, c % 3] = True
    mask = boxed.repeat(8, 0).repeat(8, 1).repeat(8, 2)
    got0, got1 = t.read_field(0), t.read_field(1)
    for lev, (src, got) in enumerate(((a, got0), (b, got1))):
        f = np.where(mask, src, 0).astype(np.float64)
        for c in (13, 4, 10, 12):               # kept cells diagonal/adjacent to the corner
            cz, cy, cx = c // 9, (c // 3) % 3, c % 3
            region = np.zeros((24, 24, 24))
            for dz in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        zz, yy, xx = cz + dz, cy + dy, cx + dx
                        if 0 <= zz < 3 and 0 <= yy < 3 and 0 <= xx < 3:
                            region[(dz + 1) * 8:(dz + 2) * 8, (dy + 1) * 8:(dy + 2) * 8,
                                   (dx + 1) * 8:(dx + 2) * 8] = f[zz * 8:zz * 8 + 8, yy * 8:yy * 8 + 8,
                                                                  xx * 8:xx * 8 + 8]
            want = numpy_region(region, 64, 0.25, 0.5)[8:16, 8:16, 8:16]
            cell = got[cz * 8:cz * 8 + 8, cy * 8:cy * 8 + 8, cx * 8:cx * 8 + 8]
            assert np.allclose(cell, want, rtol=0, atol=2e-7 * np.abs(want).max()), (lev, c)
        # cells away from the corner keep the plain step
        for c in (14, 16, 22):
            cz, cy, cx = c // 9, (c // 3) % 3, c % 3
            sl = (slice(cz * 8, cz * 8 + 8), slice(cy * 8, cy * 8 + 8), slice(cx * 8, cx * 8 + 8))
            assert np.array_equal(got[sl], src[sl])


def test_lpf_release_leaves_less_high_frequency_than_hard_release():
    def hf_energy(t):
        f = t.read_field(0).astype(np.float64)
        S = np.abs(np.fft.fftn(f)) ** 2
        k = np.sqrt(sum(np.fft.fftfreq(n)[s] ** 2 for n, s in zip(
            f.shape, np.ix_(range(f.shape[0]), range(f.shape[1]), range(f.shape[2])))))
        return S[k > 0.3].sum()
    soft, _, _ = released_scenario((0.2, 0.4))
    hard, _, _ = released_scenario(None)
    soft.step(1)
    hard.step(1)
    assert hf_energy(soft) < 0.5 * hf_energy(hard)
