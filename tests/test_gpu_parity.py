"""GPU parity of the training step against the FP64 oracle, through the C ABI.

Small-cube workload: 20,000 Gaussians in 16 Morton blocks of 1,250, 256x256
cameras (16 x 16 tiles, several tiles per Gaussian, ragged last block when
n is not a multiple of B).  Tolerances: block order, visibility sets, deltas
and the tile/depth order bit-exact; projected centre and depth bit-exact (both
sides follow the FP32 key-path specification); images max-abs 1e-4 plus the
oracle's slack at pixels whose result depends on a borderline FP32 decision;
gradients rel-L2 1e-3 for every loss (the L1 sign decided on the GPU's image on both
sides); the block spheres after the update equal those of the updated
parameters."""
import numpy as np
import pytest

import scenes
from parity_util import c1_inputs, image_within, rel_l2, report

pytestmark = pytest.mark.gpu


def _setup(orc, tgs, loss=1, n=20000, block_size=1250, **cfg):
    c, perm, Pm, tp = c1_inputs(orc, block_size=block_size, n=n)
    cams = [scenes.camera_array(x) for x in c["cams"]]
    _, Pt = orc.create(tp, block_size)
    targets = [orc.render(Pt.astype(np.float64), cam)["img"].astype(np.float32) for cam in cams]
    table = tgs.TideTable(c["params"], block_size=block_size, max_batch=2, max_width=256, max_height=256, loss=loss,
                          **cfg)
    return c, perm, Pm, cams, targets, table


@pytest.mark.parametrize("B", [1250, 9000])
def test_create_block_order_and_spheres(orc, tgs, B):
    # B = 9000: blocks longer than one chunk of the bounds kernel (4,096 rows),
    # the last one ragged (2,000 rows)
    c, perm, Pm, cams, targets, table = _setup(orc, tgs, block_size=B)
    assert np.array_equal(table.block_order(), perm)
    sph_o = orc.block_spheres(Pm.astype(np.float64), B)
    sph_g = table.spheres()
    np.testing.assert_allclose(sph_g, sph_o, rtol=2e-6, atol=2e-6)
    table.close()


def _check_step(orc, tgs, params, B, camd, target, loss, W, H, **cfg):
    """One GPU training step vs the oracle's over the same render set R & K."""
    perm, Pm = orc.create(params, B)
    cam = scenes.camera_array(camd)
    K = (params.shape[0] + B - 1) // B
    table = tgs.TideTable(params, block_size=B, max_batch=1, max_width=W, max_height=H, loss=loss, **cfg)
    lval = table.step([camd], target[None])
    P = Pm.astype(np.float64).copy()
    M1, M2 = np.zeros_like(P), np.zeros_like(P)
    steps = np.zeros(K, np.int64)
    sph = orc.block_spheres(Pm.astype(np.float64), B)
    _, vis = orc.visible_blocks(sph, [cam])
    sets = table.sets(1)
    assert np.array_equal(sets["k_visible"], vis)
    render_blocks = np.nonzero(vis & sets["r_resident"])[0]
    o = orc.train_step(P, M1, M2, steps, B, render_blocks, [cam], target[None], lr=1e-3, loss_kind=loss)
    assert abs(lval - o["loss"]) <= 1e-4 * o["loss"]
    # ---- forward intermediates
    rec = table.camera_record(0, W, H)
    orec = o["records"][0]
    assert np.array_equal(rec["ids"], o["ids"])
    S = orec["S"]
    vg = rec["splat"][:, 11] != 0
    vo = S[:, orc.VISIBLE] != 0
    border = S[:, orc.BORDER] != 0
    assert np.array_equal(vg[~border], vo[~border])
    both = vg & vo
    for col, name in ((0, "u"), (1, "v"), (2, "depth")):
        assert np.array_equal(rec["splat"][both, col], S[both, col].astype(np.float32)), name
    nb = both & ~border
    assert np.array_equal(rec["splat"][nb, 10], S[nb, orc.RADIUS])
    assert np.array_equal(rec["rect"][nb], S[nb][:, [orc.X0, orc.Y0, orc.X1, orc.Y1]].astype(np.int32))
    for col in (3, 4, 5, 6, 7, 8, 9):
        np.testing.assert_allclose(rec["splat"][both, col], S[both, col], rtol=2e-4, atol=2e-5)
    # sort order: per tile, identical sequences unless a border Gaussian is involved
    bset = set(np.nonzero(border)[0].tolist())
    for t in range(rec["ranges"].shape[0]):
        a, b = rec["ranges"][t]
        oa, ob = orec["ranges"][t]
        sg, so = rec["pair_vals"][a:b], orec["vals"][oa:ob]
        if bset & (set(sg.tolist()) | set(so.tolist())):
            continue
        assert np.array_equal(sg, so), t
    err, frac = image_within(rec["image"], orec)
    assert err <= 1e-4 and frac < 0.05
    img_err = err
    clean = orec["slack"] == 0
    np.testing.assert_allclose(rec["t_final"][clean], orec["T"][clean], atol=1e-5)
    assert np.array_equal(rec["n_last"][clean], orec["nlast"][clean])
    # ---- gradients: 2D record and the 59-parameter gradient (from m = (1 - b1) g)
    # The reference is the oracle's analytic backward from dL/dimage with the
    # L1 sign decisions taken on the GPU's FP32 image: sign(C - C_target) is a
    # decision, and where |C - C_target| is within the image tolerance the two
    # sides may legitimately take opposite signs; both then take the kernel's.
    # The D-SSIM part is continuous and comes from the oracle's own image.
    img_o = orec["img"][None]
    tg = target[None].astype(np.float64)
    nval = img_o.size
    sg = np.sign(rec["image"][None].astype(np.float64) - tg)
    if loss == 1:
        dimg = 2.0 * (img_o - tg) / nval
    elif loss == 0:
        dimg = sg / nval
    else:
        from oracle import ssim as ossim
        dimg = 0.8 * sg / nval - 0.2 * ossim.ssim_grad(img_o, tg)
    ids = o["ids"]
    Ps = Pm[ids].astype(np.float64)
    g_ref, g2_ref = orc.render_grad(Ps, cam, orec, dimg[0])
    for q in range(9):
        assert rel_l2(rec["grad2d"][vo & vg, q], g2_ref[vo & vg, q]) < 1e-3, q
    p_g, m1, m2, st = table.state()
    touched = o["touched"].astype(bool)
    g_gpu = m1[ids] / 0.1
    assert rel_l2(g_gpu[touched], g_ref[touched]) < 1e-3
    for f in range(59):
        assert rel_l2(g_gpu[touched, f], g_ref[touched, f]) < 1e-3, f
    report(f"c1 cube {params.shape[0]} {W}x{H} loss {loss}", "fp32", image_maxabs=img_err, slack_frac=frac,
           grad2d_rel_l2=max(rel_l2(rec["grad2d"][vo & vg, q], g2_ref[vo & vg, q]) for q in range(9)),
           grad59_rel_l2=rel_l2(g_gpu[touched], g_ref[touched]))
    # ---- masked Adam: untouched rows bit-identical, touched rows moved by one
    # Adam step of the reference gradient (from zero moments, step 1)
    moved = np.zeros(len(p_g), bool)
    moved[ids[touched]] = True
    assert np.array_equal(p_g[~moved], Pm[~moved])
    assert np.array_equal(st, steps.astype(np.uint32))
    P1 = Ps.copy()
    orc.adam(P1, g_ref, np.zeros_like(P1), np.zeros_like(P1), touched.astype(np.uint8),
             np.ones(len(ids), np.int64), lr=1e-3)
    d_g = p_g[ids].astype(np.float64) - Ps
    d_o = P1 - Ps
    scale = np.abs(g_ref[touched]).max(0)
    amb = np.abs(g_ref) < 1e-4 * scale
    ok = np.abs(d_g - d_o) <= 1e-6 + 2.1e-3 * amb
    assert ok[touched].all()
    # ---- bound refresh (Sec. 3.3): the spheres after the update are those of
    # the updated parameters (blocks without a touched Gaussian kept theirs)
    np.testing.assert_allclose(table.spheres(), orc.block_spheres(p_g.astype(np.float64), B), rtol=2e-6, atol=2e-6)
    table.close()
    return len(render_blocks), K


@pytest.mark.parametrize("loss", [1, 0, 2])
def test_step_matches_oracle(orc, tgs, loss):
    c, perm, Pm, cams, targets, table = _setup(orc, tgs, loss=loss)
    table.close()
    _check_step(orc, tgs, c["params"], 1250, c["cams"][0], targets[0], loss, 256, 256)


def test_step_dssim_ragged_image(orc, tgs):
    """L1 + D-SSIM at 200 x 150: neither side is a multiple of the 16-pixel
    raster tiles or of the 32-pixel tiles of the SSIM filters, so the halo
    and the image edges cut through tiles."""
    cfg = scenes.small_cube_config()
    R, t = scenes.look_at([0.0, 0.0, -3.0], [0.7, 0.7, -0.7])
    camd = scenes.pinhole(200, 150, 22.0, R, t)
    tp = scenes.perturb(cfg["params"], seed=79)
    _, Pt = orc.create(tp, 250)
    target = orc.render(Pt.astype(np.float64), scenes.camera_array(camd))["img"].astype(np.float32)
    _check_step(orc, tgs, cfg["params"], 250, camd, target, 2, 200, 150)


def test_step_partial_render_list(orc, tgs):
    """A camera that sees about half of 80 blocks: the render list is a strict
    subset of the cache capacity (the layout of the per-step arrays differs
    from the full case)."""
    cfg = scenes.small_cube_config()
    R, t = scenes.look_at([0.0, 0.0, -3.0], [0.7, 0.7, -0.7])
    camd = scenes.pinhole(192, 160, 22.0, R, t)
    tp = scenes.perturb(cfg["params"], seed=78)
    _, Pt = orc.create(tp, 250)
    target = orc.render(Pt.astype(np.float64), scenes.camera_array(camd))["img"].astype(np.float32)
    nr, K = _check_step(orc, tgs, cfg["params"], 250, camd, target, 1, 192, 160)
    assert nr < K


def test_block_delta_two_cameras(orc, tgs):
    """Capacity 8 of 16 blocks, two close cameras: R, S+ and S- follow
    Algorithm 1 exactly (exact next-batch prefetch)."""
    cfg = scenes.small_cube_config()
    perm, Pm = orc.create(cfg["params"], 1250)
    camsd = []
    for pos, tgt in (([0.0, 0.0, -1.4], [0.5, 0.4, 0.0]), ([0.3, 0.1, -1.4], [0.9, 0.3, 0.2]),
                     ([0.7, 0.2, -1.2], [1.0, -0.2, 0.4])):
        R, t = scenes.look_at(pos, tgt)
        camsd.append(scenes.pinhole(256, 256, 50.0, R, t))
    cams = [scenes.camera_array(x) for x in camsd]
    table = tgs.TideTable(cfg["params"], block_size=1250, max_batch=1, max_width=256, max_height=256,
                          cache_blocks=8, spare_slots=2, prefetch_mode=1, lr=0.0)
    tgt = np.zeros((1, 256, 256, 3), np.float32)
    sph = orc.block_spheres(Pm.astype(np.float64), 1250)
    K = 16
    r = np.zeros(K, np.uint8)
    kacc = np.zeros(K, np.uint8)
    age = np.full(K, 126, np.uint32)
    for i in range(3):
        nxt = [camsd[i + 1]] if i + 1 < 3 else None
        table.step([camsd[i]], tgt, next_cams=nxt)
        vis, _ = orc.visible_blocks(sph, [cams[i]])
        out = orc.residency(kacc, vis[None] if vis.ndim == 1 else vis, r, age, 8, 0.75, 8 // 2)
        sets = table.sets(1)
        assert np.array_equal(sets["k_visible"], vis.reshape(-1)), i
        assert np.array_equal(sets["r_resident"], out["r_next"]), i
        assert sets["s_plus"].tolist() == out["s_plus"].tolist(), i
        assert sets["s_minus"].tolist() == out["s_minus"].tolist(), i
        kacc = (out["r_next"] & vis.reshape(-1)).astype(np.uint8)
        r, age = out["r_next"], out["age"]
    table.close()


def test_pair_overflow_skips_the_update_and_recovers(orc, tgs):
    """A pair capacity far below the render's pairs: the step's update is
    skipped (parameters and step counters unchanged), the capacity grows once
    the host reads the count, and the next step matches the oracle."""
    c, perm, Pm, tp = c1_inputs(orc)
    camd = c["cams"][0]
    cam = scenes.camera_array(camd)
    _, Pt = orc.create(tp, 1250)
    target = orc.render(Pt.astype(np.float64), cam)["img"].astype(np.float32)
    table = tgs.TideTable(c["params"], block_size=1250, max_batch=1, max_width=256, max_height=256, loss=1,
                          pair_capacity=100)
    table.step([camd], target[None])
    st = table.stats()
    assert st["pair_overflows"] == 1 and st["dropped_steps"] == 1
    p_g, m1, m2, steps = table.state()
    assert np.array_equal(p_g, Pm) and not m1.any() and not steps.any()
    lval = table.step([camd], target[None])
    st = table.stats()
    assert st["pair_overflows"] == 1 and st["dropped_steps"] == 1 and st["last_pairs"] > 1149
    K = 16
    sph = orc.block_spheres(Pm.astype(np.float64), 1250)
    _, vis = orc.visible_blocks(sph, [cam])
    P = Pm.astype(np.float64).copy()
    M1, M2 = np.zeros_like(P), np.zeros_like(P)
    o = orc.train_step(P, M1, M2, np.zeros(K, np.int64), 1250, np.nonzero(vis)[0], [cam], target[None], lr=1e-3,
                       loss_kind=1)
    assert abs(lval - o["loss"]) <= 1e-4 * o["loss"]
    p_g, m1, m2, steps = table.state()
    t = o["touched"].astype(bool)
    assert rel_l2(m1[o["ids"]][t] / 0.1, o["grad"][t]) < 1e-3
    table.close()


def test_render_after_pair_overflow_is_complete(orc, tgs):
    import torch
    c, perm, Pm, tp = c1_inputs(orc)
    camd = c["cams"][1]
    table = tgs.TideTable(c["params"], block_size=1250, max_batch=1, max_width=256, max_height=256,
                          pair_capacity=100)
    img = torch.zeros(256, 256, 3, device="cuda")
    table.render(camd, img)
    st = table.stats()
    assert st["pair_overflows"] == 1 and st["dropped_steps"] == 0
    orec = orc.render(Pm.astype(np.float64), scenes.camera_array(camd))
    err, frac = image_within(img.cpu().numpy(), orec)
    assert err <= 1e-4 and frac < 0.05
    table.close()


def test_grouped_learning_rates_follow_the_schedule(orc, tgs):
    """lr_schedule 1: from zero moments each touched parameter moves by its
    group's rate times the sign of its gradient (Adam's first step); with a
    one-step decay the second step's means move by the final rate."""
    c, perm, Pm, tp = c1_inputs(orc)
    camd = c["cams"][0]
    cam = scenes.camera_array(camd)
    _, Pt = orc.create(tp, 1250)
    target = orc.render(Pt.astype(np.float64), cam)["img"].astype(np.float32)
    rates = [1e-3, 2e-3, 3e-3, 4e-3, 5e-3, 6e-3]
    table = tgs.TideTable(c["params"], block_size=1250, max_batch=1, max_width=256, max_height=256, loss=1,
                          lr_schedule=1, lr_groups=rates, lr_means_final=1e-5, lr_decay_steps=1)
    table.step([camd], target[None])
    p1, m1, _, _ = table.state()
    d = p1.astype(np.float64) - Pm.astype(np.float64)
    g = m1.astype(np.float64) / 0.1
    lr_col = orc.group_lr(rates)
    big = np.abs(g) > 1e-6 * np.abs(g).max()
    expect = -np.sign(g) * lr_col[None, :]
    assert big.sum() > 1000
    np.testing.assert_allclose(d[big], expect[big], rtol=2e-3, atol=1e-9)
    # the second step: the means' rate is the final one
    table.step([camd], target[None])
    p2, _, _, _ = table.state()
    step2 = np.abs(p2[:, 0:3].astype(np.float64) - p1[:, 0:3])
    moved = step2 > 0
    assert moved.any() and step2[moved].max() <= 1e-5 * 1.5
    table.close()


def test_two_camera_batch_matches_oracle(orc, tgs):
    """A batch of two cameras (the fused chain rule sums both cameras'
    gradients per Gaussian): loss, touched set, step counters and the summed
    59-parameter gradient against the oracle."""
    c, perm, Pm, cams, targets, table = _setup(orc, tgs, loss=1)
    lval = table.step(c["cams"], np.stack(targets))
    p_g, m1, _, st = table.state()
    table.close()
    K = 16
    sph = orc.block_spheres(Pm.astype(np.float64), 1250)
    _, vis = orc.visible_blocks(sph, cams)
    P = Pm.astype(np.float64).copy()
    M1, M2 = np.zeros_like(P), np.zeros_like(P)
    steps = np.zeros(K, np.int64)
    o = orc.train_step(P, M1, M2, steps, 1250, np.nonzero(vis)[0], cams, np.stack(targets), lr=1e-3, loss_kind=1)
    assert abs(lval - o["loss"]) <= 1e-4 * o["loss"]
    assert np.array_equal(st, steps.astype(np.uint32))
    t = o["touched"].astype(bool)
    g_gpu = m1[o["ids"]].astype(np.float64) / 0.1
    assert rel_l2(g_gpu[t], o["grad"][t]) < 1e-3
    for f in range(59):
        assert rel_l2(g_gpu[t, f], o["grad"][t, f]) < 1e-3, f
