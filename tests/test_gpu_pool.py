"""Box-pool exhaustion far beyond the pool's size (Boxes, Fig. 1; update
procedure step 8).

A sheet of boxed bricks with initial values on every node triggers every
brick across its faces (or, with the 26-neighbour set, its whole
neighbourhood) at the first update, while only a handful of vacant boxes are
left: won claims outnumber the vacant boxes many times over.  The step must
finish, box exactly as many bricks as there were vacant boxes (zeroed),
leave every other value untouched, report TCM_ENOMEM and refuse later steps
with TCM_ESTATE.  Inside a batch, a simulation that boxes everything at
admission (and so claims nothing) keeps stepping correctly in the same
launch: its fields equal the oracle's bit for bit.
"""
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


SHAPE = (96, 96, 96)          # 12^3 bricks of 8^3
SHEET_Z = 5                   # brick layer holding the initial values
SHEET = 8                     # 8 x 8 bricks of that layer


def sheet_field(seed=3):
    """Non-zero values inside an 8 x 8 brick sheet (64 bricks), zero on its
    outer boundary layer: the update on the initial state boxes only the
    sheet (6 neighbours) or its 26-neighbourhood (26), and after the first
    step every outer face of what is boxed holds values."""
    rng = np.random.default_rng(seed)
    now = np.zeros(SHAPE, F32)
    z0 = SHEET_Z * 8
    n = 8 * SHEET
    now[z0 + 1:z0 + 7, 9:8 + n - 1, 9:8 + n - 1] = rng.uniform(0.5, 1.0, (6, n - 2, n - 2))
    prev = (now * F32(0.75)).astype(F32)
    return now, prev


M = SHAPE[2] // 8


def brick_id(cx, cy, cz):
    return (cz * M + cy) * M + cx


def primed_bricks(neighbours):
    """Bricks boxed before the first step: the sheet, or its 26-neighbourhood."""
    r = 0 if neighbours == 6 else 1
    return np.array(sorted(brick_id(1 + i, 1 + j, SHEET_Z + dz)
                           for dz in range(-r, r + 1) for j in range(-r, SHEET + r)
                           for i in range(-r, SHEET + r)), np.int64)


def brick_slice(bid):
    cz, cy, cx = bid // (M * M), (bid // M) % M, bid % M
    return (slice(cz * 8, cz * 8 + 8), slice(cy * 8, cy * 8 + 8), slice(cx * 8, cx * 8 + 8))


def oracle_steps(now, prev, neighbours, steps):
    o = oracle.OracleTCM(SHAPE, W.homogeneous(1.0), 1.0, 0.5, neighbours=neighbours)
    o.set_field(now, prev)
    o.step(steps)
    return o


@pytest.mark.parametrize("neighbours", [6, 26])
def test_claims_far_beyond_the_pool_solo(neighbours):
    now, prev = sheet_field()
    primed = primed_bricks(neighbours)
    free = 4
    boxes = len(primed) + free
    wl = W.Workload("sheet", SHAPE, W.homogeneous(1.0), 1.0, 0.5, [], 0, neighbours=neighbours)
    g = tcm.Sim.from_workload(wl, pool_bytes=boxes * tcm.tcm_slot_bytes())
    g.set_field(now, prev)
    assert np.array_equal(g.active_bricks(), primed)   # primed, nothing claimed yet
    # the values reach the outer faces of the sheet after one step; with the
    # 26-neighbour set they reach the primed neighbourhood's bricks after two
    steps = 1 if neighbours == 6 else 2
    o = oracle_steps(now, prev, neighbours, steps)
    # the oracle (unlimited pool) boxes far more than the vacant boxes left here
    assert o.active_count()[0] - len(primed) > 20 * free
    with pytest.raises(tcm.TCMError) as e:
        g.step(steps)
    assert e.value.status == tcm.TCM_ENOMEM
    act = g.active_bricks()
    assert len(act) == boxes                      # every box in use, none twice
    assert set(primed.tolist()) <= set(act.tolist())
    assert set(act.tolist()) <= set(o.active_bricks().tolist())
    # the primed bricks stepped exactly as the oracle's did; bricks that got
    # one of the vacant boxes hold zeros; nothing outside the boxes
    a, b = g.read_field(0), g.read_field(1)
    oa, ob = o.read_field(0), o.read_field(1)
    pset = set(primed.tolist())
    mask = np.zeros(SHAPE, bool)
    for bid in act.tolist():
        sl = brick_slice(bid)
        mask[sl] = True
        if bid in pset:
            assert np.array_equal(a[sl], oa[sl]) and np.array_equal(b[sl], ob[sl]), bid
        else:
            assert not a[sl].any() and not b[sl].any(), bid
    assert not a[~mask].any() and not b[~mask].any()
    with pytest.raises(tcm.TCMError) as e:
        g.step(1)
    assert e.value.status == tcm.TCM_ESTATE
    assert g.pool_info() == (boxes, 0)
    g.close()


def test_overcommitted_sim_beside_a_healthy_one_in_a_batch():
    now, prev = sheet_field(7)
    primed = primed_bricks(6)
    # healthy: boxes all of its 27 bricks at admission and never claims
    h_shape = (24, 24, 24)
    h_media = W.random_dense_media(h_shape, 11, 1.0, 1.8)
    h_dt = 0.5 / h_media.c_max()
    h_wl = W.Workload("healthy", h_shape, h_media, 1.0, h_dt, [(11, 12, 13, W.ricker(1 / 6, h_dt))], 0)
    free = 3
    boxes = 27 + len(primed) + free
    b = tcm.Batch(pool_bytes=boxes * tcm.tcm_slot_bytes(), max_bricks=4096, max_sims=4)
    hs = b.add(h_wl, dense=True)
    over = b.add(W.Workload("over", SHAPE, W.homogeneous(1.0), 1.0, 0.5, [], 0))
    over.set_field(now, prev)
    with pytest.raises(tcm.TCMError) as e:
        b.step(3)
    assert e.value.status == tcm.TCM_ENOMEM
    ho = oracle.OracleTCM(h_shape, h_media, 1.0, h_dt, dense=True)
    ho.add_source(11, 12, 13, W.ricker(1 / 6, h_dt).astype(F32))
    n = hs.step_index
    assert n >= 1
    ho.step(n)
    assert np.array_equal(hs.read_field(0), ho.read_field(0))
    assert np.array_equal(hs.read_field(1), ho.read_field(1))
    assert np.array_equal(hs.active_bricks(), np.arange(27))
    act = over.active_bricks()
    assert set(primed.tolist()) <= set(act.tolist())
    assert len(act) == len(primed) + free
    with pytest.raises(tcm.TCMError) as e:
        b.step(1)
    assert e.value.status == tcm.TCM_ESTATE
    assert np.array_equal(hs.read_field(0), ho.read_field(0))   # still readable, unchanged
    b.close()
