"""Resident rasteriser behind torch.autograd (tgs_raster_forward/backward)
against the FP64 oracle: image max-abs 1e-4 (+ oracle slack), gradient of a
linear functional <w, image> rel-L2 1e-3 per parameter group."""
import numpy as np
import pytest

import scenes
from parity_util import image_within, rel_l2

pytestmark = pytest.mark.gpu


# 256: long tile lists split into backward segments, all 256 tiles in one
# 1,024-tile chunk of the tile order; 200: ragged edge tiles; 640: 1,600
# tiles (two chunks of the order and of the backward units), 376 split
@pytest.mark.parametrize("n,B,size", [(20000, 1250, 256), (3001, 512, 200), (20000, 1250, 640)])
def test_autograd_matches_oracle(orc, tgs, n, B, size):
    import torch
    cfg = scenes.small_cube_config(n=n, size=size)
    P = cfg["params"]
    cam = cfg["cams"][1]
    bg = (0.05, 0.1, 0.15)
    blocks = tgs.to_block_layout(torch.tensor(P, device="cuda"), B).requires_grad_(True)
    r = tgs.Rasterizer(n, size, size)
    img = tgs.rasterize(blocks, n, cam, bg, r)
    w = np.random.default_rng(3).normal(size=(size, size, 3)).astype(np.float32)
    (img * torch.tensor(w, device="cuda")).sum().backward()
    g = tgs.from_block_layout(blocks.grad, n).detach().cpu().numpy()
    ca = scenes.camera_array(cam)
    o = orc.render(P.astype(np.float64), ca, bg=bg, with_slack=True)
    err, frac = image_within(img.detach().cpu().numpy(), o)
    assert err <= 1e-4 and frac < 0.05
    go, _ = orc.render_grad(P.astype(np.float64), ca, o, w.astype(np.float64), bg)
    vis = o["S"][:, orc.VISIBLE] != 0
    assert rel_l2(g[vis], go[vis]) < 1e-3
    for a, b in ((0, 3), (3, 6), (6, 10), (10, 11), (11, 14), (14, 59)):
        assert rel_l2(g[vis, a:b], go[vis, a:b]) < 1e-3, (a, b)
    assert not g[~vis].any()  # Gaussians without a tile rect get no gradient
    r.close()


def test_dense_adam_matches_oracle(orc, tgs):
    import torch
    rng = np.random.default_rng(4)
    n, B = 5000, 1024
    P = rng.normal(size=(n, 59)).astype(np.float32)
    G = rng.normal(size=(n, 59)).astype(np.float32)
    touched = (rng.random(n) < 0.5).astype(np.uint8)
    blocks = tgs.to_block_layout(torch.tensor(P, device="cuda"), B)
    gb = tgs.to_block_layout(torch.tensor(G, device="cuda"), B)
    m1, m2 = torch.zeros_like(blocks), torch.zeros_like(blocks)
    steps = torch.zeros((n + B - 1) // B, dtype=torch.int32, device="cuda")
    t = torch.tensor(touched, device="cuda")
    Po = P.astype(np.float64)
    M1, M2 = np.zeros_like(Po), np.zeros_like(Po)
    st = np.zeros((n + B - 1) // B, np.int64)
    for k in range(3):
        tgs.adam(blocks, gb, m1, m2, t, steps, n, lr=1e-3)
        blk = np.arange(n) // B
        for b in np.unique(blk[touched.astype(bool)]):
            st[b] += 1
        orc.adam(Po, G.astype(np.float64), M1, M2, touched, st[blk], lr=1e-3)
    torch.cuda.synchronize()
    Pg = tgs.from_block_layout(blocks, n).cpu().numpy()
    np.testing.assert_allclose(Pg, Po, rtol=0, atol=2e-6)
    assert np.array_equal(Pg[touched == 0], P[touched == 0])
