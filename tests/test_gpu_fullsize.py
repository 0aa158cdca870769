"""Parity at full size: the 100M-Gaussian street table in the benchmark's
configuration (4,096-Gaussian blocks, 24 GB HBM cache, 1600x900), one render
and one training step of camera 0 through the C ABI, against the FP64 oracle
on the camera's neighbourhood: every Gaussian whose mean lies within the ball
through the far corners of the frustum (plus 10 m for footprints), generated
row-exactly on the CPU.  Gaussians outside that ball are culled by Level 2 in
both, so the images agree pixel by pixel (max-abs 1e-4 plus the oracle's slack
for borderline FP32 decisions) and the losses to 1e-4 relative."""
import math

import numpy as np
import pytest

import scenes
from parity_util import image_within

pytestmark = pytest.mark.gpu

N = 100_000_000


def test_street_100m_render_and_loss_match_oracle(orc, tgs):
    import torch
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
                          spare_slots=512, prefetch_mode=0, loss=0)
    img = torch.zeros(H, W, 3, device=dev)
    table.render(cam, img)
    gpu_img = img.cpu().numpy()
    tgt = np.full((1, H, W, 3), 0.3, np.float32)
    lval = table.step([cam], tgt)
    perm = table.block_order()
    table.close()
    del host

    # the oracle on the neighbourhood, in the table's (Morton) row order
    pos = -np.asarray(cam["R"]).T @ np.asarray(cam["t"])
    tx, ty = 0.5 * W / cam["fx"], 0.5 * H / cam["fy"]
    radius = cam["zfar"] * math.sqrt(1.0 + tx * tx + ty * ty) + 10.0
    rows, idx, _ = scenes.street_scene(N, device="cpu", chunk=1 << 22, near=(pos, radius))
    rank = np.empty(N, np.int64)
    rank[perm] = np.arange(N)
    order = np.argsort(rank[idx.numpy()], kind="stable")
    P = rows.numpy()[order].astype(np.float64)
    ca = scenes.camera_array(cam)
    rec = orc.render(P, ca, with_slack=True)
    err, frac = image_within(gpu_img, rec)
    assert err <= 1e-4 and frac < 0.05
    lo, _ = orc.loss(rec["img"][None], tgt.astype(np.float64), 0)
    assert abs(lval - lo) <= 1e-4 * lo
