"""Degenerate input of the training step on the GPU, through the C ABI: a
camera turned away from the scene sees no block (the oracle's Level-1 set is
empty too), so the step renders the background only, its L2 loss is that of
the background against the target, and it trains nothing (parameters,
moments and step counters unchanged).  The table is left as a fresh one: its
next step, on a camera that sees the scene, gives a fresh table's first-step
loss, and the same parameters except for the few entries whose near-zero
gradient may change sign with the order of the atomic sums (the first Adam
step moves every touched entry by the learning rate times its sign)."""
import numpy as np
import pytest

import scenes
from parity_util import c1_inputs

pytestmark = pytest.mark.gpu

B = 1250


def _table(tgs, c):
    return tgs.TideTable(c["params"], block_size=B, max_batch=1, max_width=256, max_height=256, loss=1)


def test_camera_that_sees_nothing_trains_nothing(orc, tgs):
    c, perm, Pm, _ = c1_inputs(orc, block_size=B)
    cam = c["cams"][0]
    # at the first camera's centre, looking away from the cube
    R, t = scenes.look_at([0.0, 0.0, -3.0], [0.0, 0.0, -6.0])
    away = scenes.pinhole(256, 256, 60.0, R, t)
    sph = orc.block_spheres(Pm.astype(np.float64), B)
    _, vis = orc.visible_blocks(sph, [scenes.camera_array(away)])
    assert not vis.any()
    target = np.full((1, 256, 256, 3), 0.3, np.float32)

    table = _table(tgs, c)
    p0, m0, v0, s0 = table.state()
    loss = table.step([away], target)
    # background 0 against 0.3 everywhere: (0.3)^2
    assert abs(loss - 0.3 ** 2) < 1e-6
    sets = table.sets(1)
    assert not sets["k_visible"].any()
    assert len(sets["s_plus"]) == 0
    rec = table.camera_record(0, 256, 256)
    assert len(rec["ids"]) == 0 and len(rec["pair_vals"]) == 0
    assert not rec["image"].any()
    assert (rec["t_final"] == 1.0).all() and not rec["n_last"].any()
    p1, m1, v1, s1 = table.state()
    assert np.array_equal(p1, p0) and np.array_equal(m1, m0) and np.array_equal(v1, v0)
    assert np.array_equal(s1, s0) and not s1.any()

    # the next step sees the scene: as a fresh table's first step
    l_after = table.step([cam], target)
    fresh = _table(tgs, c)
    l_fresh = fresh.step([cam], target)
    assert abs(l_after - l_fresh) <= 1e-6 * l_fresh
    pa, _, _, sa = table.state()
    pb, _, _, sb = fresh.state()
    assert np.array_equal(sa, sb) and sa.any()
    moved = pb != p0
    assert moved.any()
    assert (np.abs(pa - pb) > 1e-6).mean() < 5e-4
    table.close()
    fresh.close()
