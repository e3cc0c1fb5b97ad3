"""Degenerate and boundary cases through the C ABI against the oracle:
one-node and one-line domains, a domain of one partial brick, sources on
every corner and edge, a source that starts and ends within the first steps,
zero-length wavelets, and the sizes at which a 32-bit node count would
overflow (large brick ids)."""
import numpy as np
import pytest

import oracle
from paper_1702_00216_gb300 import tcm
from paper_1702_00216_gb300 import workloads as W

pytestmark = pytest.mark.gpu
F32 = np.float32


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def run_both(shape, sources, steps, **kw):
    m = W.homogeneous(1.0)
    dt = 0.5
    s = tcm.Sim(shape, m, 1.0, dt, **kw)
    o = oracle.OracleTCM(shape, m, 1.0, dt, thr_mode=kw.get("thr_mode", 0), tau=kw.get("threshold", 0.0))
    for x, y, z, w in sources:
        s.add_source(x, y, z, np.asarray(w, F32))
        o.add_source(x, y, z, np.asarray(w, F32))
    s.step(steps)
    o.step(steps)
    out = (s.read_field(0), o.read_field(0), s.read_field(1), o.read_field(1), s.active_bricks(),
           o.active_bricks(), s.updates, o.updates)
    s.close()
    return out


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 19), (1, 17, 1), (23, 1, 1), (3, 5, 7), (9, 8, 8)])
def test_degenerate_domains(shape):
    nz, ny, nx = shape
    w = W.ricker(1 / 4, 0.5)
    srcs = [(nx // 2, ny // 2, nz // 2, w)]
    a, b, a1, b1, ia, ib, ua, ub = run_both(shape, srcs, 25)
    assert np.array_equal(a, b) and np.array_equal(a1, b1) and np.array_equal(ia, ib) and ua == ub


def test_sources_on_corners_and_edges():
    shape = (17, 18, 19)
    nz, ny, nx = shape
    w = W.ricker(1 / 5, 0.5)
    corners = [(x, y, z, w) for x in (0, nx - 1) for y in (0, ny - 1) for z in (0, nz - 1)]
    a, b, a1, b1, ia, ib, ua, ub = run_both(shape, corners + [(8, 0, 9, w[:3])], 40,
                                             thr_mode=tcm.TCM_THR_RELATIVE, threshold=1e-3)
    assert np.array_equal(a, b) and np.array_equal(a1, b1) and np.array_equal(ia, ib) and ua == ub


def test_short_and_empty_wavelets():
    shape = (20, 20, 20)
    a, b, a1, b1, ia, ib, ua, ub = run_both(shape, [(5, 5, 5, np.array([1.0])), (14, 14, 14, np.array([]))], 30)
    assert np.array_equal(a, b) and np.array_equal(ia, ib)
    assert np.abs(a).max() > 0


def test_large_brick_ids():
    # 2^31 nodes would overflow a 32-bit node index; the brick table and
    # every node address use 64-bit arithmetic (a 2048 x 2048 x 600 domain,
    # 4.9e6 bricks, only the source's neighbourhood ever boxed)
    shape = (600, 2048, 2048)
    w = W.ricker(1 / 8, 0.5)
    src = (2040, 2041, 595, w)
    s = tcm.Sim(shape, W.homogeneous(1.0), 1.0, 0.5, pool_bytes=4096 * tcm.tcm_slot_bytes())
    s.add_source(*src[:3], np.asarray(w, F32))
    s.step(30)
    # after 30 steps the wave is within L1 distance 30 of the source, so a
    # window reaching 40 nodes below it (and to the domain's upper faces) is
    # the same run on a small grid
    win = (2000, 2001, 555)
    size = (48, 47, 45)
    got = s.read_field(0, origin=win, size=size)
    o = oracle.OracleTCM(size[::-1], W.homogeneous(1.0), 1.0, 0.5)
    o.add_source(src[0] - win[0], src[1] - win[1], src[2] - win[2], np.asarray(w, F32))
    o.step(30)
    assert np.abs(got).max() > 0 and np.array_equal(got, o.read_field(0))
    s.close()
