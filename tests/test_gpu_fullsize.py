"""Parity at full size: the 100M-Gaussian street table in the benchmark's
configuration (4,096-Gaussian blocks, 24 GB HBM cache, 1600x900, the
benchmark's L1 + D-SSIM loss), one render and one training step of camera 0
through the C ABI, against the FP64 oracle on the camera's neighbourhood:
every Gaussian whose mean lies within the ball through the far corners of the
frustum (plus 10 m for footprints), generated row-exactly on the CPU.
Gaussians outside that ball are culled by Level 2 in both, so
  - the images agree pixel by pixel (max-abs 1e-4 plus the oracle's slack for
    borderline FP32 decisions) and the losses to 1e-4 relative;
  - the 2D gradients of the step and the 59-parameter gradients of the
    touched Gaussians (read back as the first Adam moment, m = (1 - b1) g)
    agree to rel-L2 1e-3 with the oracle's backward (the L1 sign decided on
    the GPU's image on both sides);
  - the touched rows moved by one Adam step of that gradient, the others
    not at all, and the refreshed spheres of the rendered blocks are those of
    their updated rows;
  - a render of the same camera from the BF16 record matches the oracle on
    the same rows with their SH rest rounded to BF16."""
import math

import numpy as np
import pytest

import scenes
from parity_util import image_within, rel_l2, report
from test_gpu_bf16 import bf16_round

pytestmark = pytest.mark.gpu

N = 100_000_000


def test_street_100m_step_matches_oracle(orc, tgs):
    import torch
    from oracle import ssim as ossim
    dev = torch.device("cuda", 0)
    gt, _ = scenes.street_scene(N, device=dev)
    host = gt.cpu().numpy()
    del gt
    torch.cuda.empty_cache()
    cams = scenes.street_drive_cameras(2)
    cam = cams[0]
    W, H = cam["width"], cam["height"]
    cache = int(24e9 // (4096 * 708))
    table = tgs.TideTable(host, block_size=4096, max_batch=1, max_width=W, max_height=H, cache_blocks=cache,
                          spare_slots=512, prefetch_mode=0, loss=2)
    img = torch.zeros(H, W, 3, device=dev)
    table.render(cam, img)
    gpu_img = img.cpu().numpy()
    tgt = np.full((1, H, W, 3), 0.3, np.float32)
    lval = table.step([cam], tgt)
    rec = table.camera_record(0, W, H)
    perm = table.block_order()
    ids_g = rec["ids"]
    vis_g = rec["splat"][:, 11] != 0
    # rows of the rendered blocks after the update, and their spheres
    blocks = np.unique(ids_g // 4096)
    all_ids = np.concatenate([np.arange(b * 4096, min((b + 1) * 4096, N)) for b in blocks])
    p_after, m1_after, _ = table.state_rows(all_ids)
    sph_after = table.spheres()[blocks]
    table.close()
    # the BF16 record (SH rest and moments BF16 in the host tier and the
    # cache): a render of the same camera
    tb = tgs.TideTable(host, block_size=4096, max_batch=1, max_width=W, max_height=H, cache_blocks=cache,
                       spare_slots=512, prefetch_mode=0, loss=2, host_bf16=1, stochastic_round=1)
    tb.render(cam, img)
    gpu_img_bf16 = img.cpu().numpy()
    tb.close()
    del host

    # the oracle on the neighbourhood, in the table's (Morton) row order
    pos = -np.asarray(cam["R"]).T @ np.asarray(cam["t"])
    tx, ty = 0.5 * W / cam["fx"], 0.5 * H / cam["fy"]
    radius = cam["zfar"] * math.sqrt(1.0 + tx * tx + ty * ty) + 10.0
    rows, idx, _ = scenes.street_scene(N, device="cpu", chunk=1 << 22, near=(pos, radius))
    rank = np.empty(N, np.int64)
    rank[perm] = np.arange(N)
    rk = rank[idx.numpy()]
    order = np.argsort(rk, kind="stable")
    oid = rk[order]  # block-order ids of the oracle's rows
    P = rows.numpy()[order].astype(np.float64)
    ca = scenes.camera_array(cam)
    o = orc.render(P, ca, with_slack=True)
    err, frac = image_within(gpu_img, o)
    assert err <= 1e-4 and frac < 0.05
    err, frac = image_within(rec["image"], o)
    assert err <= 1e-4 and frac < 0.05
    img_err, img_frac = err, frac
    # BF16 form against the oracle on the same rows with their SH rest rounded
    Pbf = P.copy()
    Pbf[:, 14:] = bf16_round(P[:, 14:])
    ob = orc.render(Pbf, ca, with_slack=True)
    err_b, frac_b = image_within(gpu_img_bf16, ob)
    assert err_b <= 1e-4 and frac_b < 0.05
    report("c3 street-100M 1600x900 render", "bf16", image_maxabs=err_b, slack_frac=frac_b,
           image_maxabs_vs_fp32_table=float(np.abs(gpu_img_bf16.astype(np.float64) - o["img"]).max()))
    del ob, Pbf
    lo, _ = orc.loss(o["img"][None], tgt.astype(np.float64), 2)
    assert abs(lval - lo) <= 1e-4 * lo

    vis_o = o["S"][:, orc.VISIBLE] != 0
    border = o["S"][:, orc.BORDER] != 0
    # render-list position of each oracle row (ids_g ascends); rows of blocks
    # the GPU did not render must be invisible, and no visible GPU Gaussian
    # lies outside the neighbourhood
    at = np.minimum(np.searchsorted(ids_g, oid), len(ids_g) - 1)
    inset = ids_g[at] == oid
    assert not (vis_o & ~inset).any()
    vis_at = np.where(inset, vis_g[at], False)
    assert np.array_equal(vis_at[~border], vis_o[~border])
    assert vis_g.sum() == vis_at.sum()
    both = vis_o & vis_at

    tg = tgt.astype(np.float64)
    nval = tg.size
    sg = np.sign(rec["image"][None].astype(np.float64) - tg)
    dimg = 0.8 * sg / nval - 0.2 * ossim.ssim_grad(o["img"][None], tg)
    g_ref, g2_ref = orc.render_grad(P, ca, o, dimg[0])
    r2 = [rel_l2(rec["grad2d"][at[both], q], g2_ref[both, q]) for q in range(9)]
    for q in range(9):
        assert r2[q] < 1e-3, q
    # 59-parameter gradients of the touched rows from the first moment
    sel = np.searchsorted(all_ids, oid[both])  # all_ids ascends
    assert np.array_equal(all_ids[sel], oid[both])
    g_gpu = m1_after[sel].astype(np.float64) / 0.1
    assert rel_l2(g_gpu, g_ref[both]) < 1e-3
    report("c3 street-100M 1600x900 step", "fp32", image_maxabs=img_err, slack_frac=img_frac, grad2d_rel_l2=max(r2),
           grad59_rel_l2=rel_l2(g_gpu, g_ref[both]))
    for f in range(59):
        assert rel_l2(g_gpu[:, f], g_ref[both, f]) < 1e-3, f
    # one Adam step of the reference gradient (zero moments, step 1)
    P1 = P[both].copy()
    orc.adam(P1, g_ref[both], np.zeros_like(P1), np.zeros_like(P1), np.ones(len(P1), np.uint8),
             np.ones(len(P1), np.int64), lr=1e-3)
    d_g = p_after[sel].astype(np.float64) - P[both]
    d_o = P1 - P[both]
    scale = np.abs(g_ref[both]).max(0)
    amb = np.abs(g_ref[both]) < 1e-4 * scale
    # (FP32 parameters: half an ulp of rounding at the parameter's magnitude)
    assert (np.abs(d_g - d_o) <= 1e-6 + 2.4e-7 * np.abs(P[both]) + 2.1e-3 * amb).all()
    # neighbourhood rows that the camera did not touch are bit-identical
    idle = inset & ~vis_at
    sel_idle = np.searchsorted(all_ids, oid[idle])
    assert np.array_equal(p_after[sel_idle], rows.numpy()[order][idle])
    # bound refresh: each rendered block's sphere from its updated rows (the
    # kernel works in FP32 at street coordinates of up to 2 km: two ulps of
    # the block centre's magnitude)
    for j, b in enumerate(blocks):
        lo_, hi_ = b * 4096, min((b + 1) * 4096, N)
        rows_b = p_after[np.searchsorted(all_ids, lo_):np.searchsorted(all_ids, hi_)].astype(np.float64)
        want = orc.block_spheres(rows_b, 4096)[0]
        tol = 2e-6 + 2.4e-7 * np.abs(want[:3]).max()
        np.testing.assert_allclose(sph_after[j], want, rtol=2e-6, atol=tol)
