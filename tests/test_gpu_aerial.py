"""Parity of the fully resident aerial configuration: 2,000,000 Gaussians of
the synthetic 1 km x 1 km block scene (jittered ground grid plus box
buildings, 4,096-Gaussian blocks), one orbit camera at 150 m altitude,
1920 x 1080 (120 x 68 tiles, the last tile row ragged), through the
hand-written autograd rasteriser (tgs_raster_forward / tgs_raster_backward)
against the FP64 oracle:
  - image max-abs 1e-4 plus the oracle's slack at borderline FP32 decisions;
  - gradient of the linear functional <w, image> (w a seeded weight map)
    rel-L2 1e-3 over the visible Gaussians and per parameter group;
  - central finite differences of the oracle on a seeded 2,000-Gaussian
    visible subset: along random directions over those Gaussians' 59
    parameters, (L(P + h d) - L(P - h d)) / 2h matches <grad, d> of the
    oracle's analytic backward (to 1e-5, two step sizes agreeing) and of
    the GPU (to 2e-3); the finite differences use the oracle's FP64 key
    path, so a step moves centres and depths continuously."""
import numpy as np
import pytest

import scenes
from parity_util import image_within, rel_l2, report

pytestmark = pytest.mark.gpu

GROUPS = ((0, 3), (3, 6), (6, 10), (10, 11), (11, 14), (14, 59))


def test_aerial_2m_1080p_autograd_and_finite_differences(orc, tgs):
    import torch
    cfg = scenes.aerial_config()
    P = cfg["params"]
    n, B = P.shape[0], cfg["block_size"]
    cam = cfg["cams"][0]
    W, H = cam["width"], cam["height"]
    assert (W, H) == (1920, 1080) and n == 2_000_000
    bg = (0.0, 0.0, 0.0)
    blocks = tgs.to_block_layout(torch.tensor(P, device="cuda"), B).requires_grad_(True)
    r = tgs.Rasterizer(n, W, H)
    img = tgs.rasterize(blocks, n, cam, bg, r)
    w = np.random.default_rng(21).normal(size=(H, W, 3)).astype(np.float32)
    (img * torch.tensor(w, device="cuda")).sum().backward()
    g = tgs.from_block_layout(blocks.grad, n).detach().cpu().numpy().astype(np.float64)
    gpu_img = img.detach().cpu().numpy()
    r.close()
    del blocks, img
    torch.cuda.empty_cache()

    ca = scenes.camera_array(cam)
    P64 = P.astype(np.float64)
    o = orc.render(P64, ca, bg=bg, with_slack=True)
    err, frac = image_within(gpu_img, o)
    assert err <= 1e-4 and frac < 0.05
    go, _ = orc.render_grad(P64, ca, o, w.astype(np.float64), bg)
    vis = o["S"][:, orc.VISIBLE] != 0
    assert vis.sum() > 100_000  # the view sees a large part of the scene
    assert rel_l2(g[vis], go[vis]) < 1e-3
    for a, b in GROUPS:
        assert rel_l2(g[vis, a:b], go[vis, a:b]) < 1e-3, (a, b)
    assert not g[~vis].any()
    report("c2 aerial-2M 1920x1080 (autograd)", "fp32", image_maxabs=err, slack_frac=frac,
           grad59_rel_l2=rel_l2(g[vis], go[vis]))

    # ---- finite differences on a seeded 2,000-Gaussian visible subset
    rng = np.random.default_rng(22)
    sub = np.sort(rng.choice(np.nonzero(vis)[0], 2000, replace=False))
    w64 = w.astype(np.float64)
    o64 = orc.render(P64, ca, bg=bg, fp32key=False)
    g64, _ = orc.render_grad(P64, ca, o64, w64, bg)

    def L(Pq):
        return float((orc.render(Pq, ca, bg=bg, fp32key=False)["img"] * w64).sum())

    checked = 0
    for trial in range(4):
        d = np.zeros_like(P64)
        d[sub] = rng.normal(size=(len(sub), 59))
        fds = []
        for h in (1e-6, 5e-7):
            Pp, Pm = P64.copy(), P64.copy()
            Pp[sub] += h * d[sub]
            Pm[sub] -= h * d[sub]
            fds.append((L(Pp) - L(Pm)) / (2 * h))
        # a step that crossed a discontinuity (alpha = 1/255, the T stop, a
        # tile-rect edge) makes the two step sizes disagree: skip that direction
        if abs(fds[0] - fds[1]) > 1e-6 * abs(fds[1]):
            continue
        fd = fds[1]
        ana = float((g64[sub] * d[sub]).sum())
        assert abs(ana - fd) <= 1e-5 * abs(fd), (ana, fd)
        gpu = float((g[sub] * d[sub]).sum())
        assert abs(gpu - fd) <= 2e-3 * abs(fd), (gpu, fd)
        checked += 1
        if checked == 2:
            break
    assert checked == 2, "too many directions crossed a discontinuity"
