"""The learned prefetch gains over reactive streaming: a predictor trained on
the visibility logged along a camera orbit, attached to a table whose cache
holds less than the whole scene, leaves fewer blocks of each batch to be
fetched on demand than reactive streaming on the same orbit."""
import math

import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu


def _orbit(n=120):
    """A loop inside the cube at radius 0.6 looking along the direction of
    travel (50 degree field of view, far plane 1.2): about 38 of the 80
    blocks are visible and about 0.7 new blocks enter per step."""
    cams = []
    for i in range(n):
        a = 2 * math.pi * i / n
        pos = [0.6 * math.cos(a), 0.2 * math.sin(2 * a), 0.6 * math.sin(a)]
        tgt = [pos[0] - math.sin(a), pos[1] + 0.1, pos[2] + math.cos(a)]
        R, t = scenes.look_at(pos, tgt)
        cams.append(scenes.pinhole(128, 96, 50.0, R, t, zfar=1.2))
    return cams


def _run(tgs, params, cams, mode, predictor=None, cache=44, schedule=False):
    t = tgs.TideTable(params, block_size=250, max_batch=1, max_width=128, max_height=96, cache_blocks=cache,
                      spare_slots=8, prefetch_mode=mode, lr=0.0)
    if predictor is not None:
        t.set_predictor(predictor, threshold=0.3, horizon_mask=0b11)
    if schedule:
        t.set_schedule(cams, horizon=2)
    tgt = np.zeros((1, 96, 128, 3), np.float32)
    t.step([cams[0]], tgt, want_loss=False)
    t.sync()
    s0 = t.stats()  # the first batch loads everything it needs in both modes
    for c in cams[1:]:
        t.step([c], tgt, want_loss=False)
    t.sync()
    st = t.stats()
    t.close()
    return {k: st[k] - s0[k] for k in ("demand_blocks", "demand_hits", "predicted_blocks", "blocks_in")}


def test_learned_prefetch_reduces_demand_misses(tgs):
    import torch
    cfg = scenes.small_cube_config()
    P = cfg["params"]
    cams = _orbit()
    log_t = tgs.TideTable(P, block_size=250, max_batch=1, max_width=128, max_height=96)
    vis = np.concatenate([log_t.visible_blocks([c]) for c in cams])  # T x K
    sph = torch.tensor(log_t.spheres(), device="cuda")
    log_t.close()
    T, K = vis.shape
    assert 10 < vis.sum(1).mean() < K - 20
    pos = vis.mean()
    pred = tgs.Predictor(K, seed=5)
    for epoch in range(6):
        for t in np.random.default_rng(epoch).permutation(T):
            hist = [cams[max(t - 7 + s, 0)] for s in range(8)]
            lab = np.stack([vis[min(t + h, T - 1)] for h in range(1, 5)], 1).astype(np.float32)
            pred.train_step(sph, hist, torch.tensor(lab, device="cuda"), pos_weight=float((1 - pos) / pos),
                            lr=2e-3)
    react = _run(tgs, P, cams, 0)
    learn = _run(tgs, P, cams, 2, predictor=pred)
    miss_r = react["demand_blocks"] - react["demand_hits"]
    miss_l = learn["demand_blocks"] - learn["demand_hits"]
    assert react["demand_blocks"] == learn["demand_blocks"] > 0
    assert learn["predicted_blocks"] > 0
    assert miss_l < 0.5 * miss_r, (miss_l, miss_r)
    pred.close()


def test_exact_lookahead_prefetches_the_trajectory(tgs):
    """Prefetch mode 3 with the orbit as schedule: the next two cameras' exact
    visible sets stream ahead, so almost no block is fetched on demand."""
    cfg = scenes.small_cube_config()
    cams = _orbit()
    react = _run(tgs, cfg["params"], cams, 0)
    look = _run(tgs, cfg["params"], cams, 3, schedule=True)
    miss_r = react["demand_blocks"] - react["demand_hits"]
    miss_x = look["demand_blocks"] - look["demand_hits"]
    assert look["demand_blocks"] == react["demand_blocks"] > 0
    assert look["predicted_blocks"] > 0
    assert miss_x <= 0.1 * miss_r, (miss_x, miss_r)
