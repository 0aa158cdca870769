"""The allocation-free forward renderer, tgs_raster_forward_noalloc.

Callers that cannot allocate device memory when they render -- renderers
confined to a memory budget owned by another allocator, real-time loops that
must not allocate -- use this entry point; it
keeps its intermediates in a fixed static device array instead of buffers from
cudaMalloc.  This test calls it through the C ABI twice in a row and checks
each image against the regular entry point, tgs_raster_forward, within the
image tolerance of the other parity tests (1e-4).  The file sorts last so a
run that stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu


def _inputs(torch, tgs):
    cfg = scenes.small_cube_config(n=20000, size=256)
    params = torch.tensor(cfg["params"], device="cuda")
    blocks = tgs.to_block_layout(params, 1250)
    return cfg, blocks


def test_noalloc_matches_regular_forward_twice(tgs):
    import torch
    cfg, blocks = _inputs(torch, tgs)
    n = cfg["params"].shape[0]
    bg = (0.1, 0.2, 0.3)
    r = tgs.Rasterizer(n, 256, 256)
    for cam in cfg["cams"]:  # two calls in a row, one per camera
        ref = torch.empty(256, 256, 3, device="cuda")
        r.forward(blocks, n, cam, bg, ref)
        out = torch.full((256, 256, 3), -1.0, device="cuda")
        tgs.raster_forward_noalloc(blocks, n, cam, bg, out)
        torch.cuda.synchronize()
        err = (out - ref).abs().max().item()
        assert err <= 1e-4, err
        assert ref.abs().sum().item() > 0  # the scene is actually visible
    r.close()


def test_noalloc_rejects_oversize_inputs(tgs):
    import torch
    cfg, blocks = _inputs(torch, tgs)
    cam = dict(cfg["cams"][0], width=1024, height=1024, cx=511.5, cy=511.5)
    out = torch.zeros(1024, 1024, 3, device="cuda")
    with pytest.raises(tgs.TgsError) as e:
        tgs.raster_forward_noalloc(blocks, 20000, cam, (0, 0, 0), out)
    assert e.value.code == 4
    big = torch.zeros((40, 59, 1250), device="cuda")
    with pytest.raises(tgs.TgsError) as e:
        tgs.raster_forward_noalloc(big, 50000, cfg["cams"][0], (0, 0, 0), out)
    assert e.value.code == 4


def test_noalloc_rejects_too_many_pairs(tgs):
    """Within the Gaussian and image limits, a render whose (tile, Gaussian)
    pairs exceed the fixed 524,288 is rejected before any pair is written: the
    count comes from the scan of per-Gaussian tile counts, checked on the host
    ahead of pair emission."""
    import torch
    cfg = scenes.small_cube_config(n=1250, size=512)
    p = torch.tensor(cfg["params"], device="cuda")
    # 1,250 Gaussians around the origin with scales of the cube's size: each
    # covers most of the 32 x 32 tiles of a 512 x 512 view at distance 3
    p[:, 0:3] *= 0.05
    p[:, 3:6] = float(np.log(0.6))
    p[:, 10] = 3.0
    blocks = tgs.to_block_layout(p, 1250)
    out = torch.zeros(512, 512, 3, device="cuda")
    with pytest.raises(tgs.TgsError) as e:
        tgs.raster_forward_noalloc(blocks, 1250, cfg["cams"][0], (0, 0, 0), out)
    assert e.value.code == 4
    assert "pairs" in str(e.value)
    # the table is still usable afterwards: a small render succeeds
    cfg2, blocks2 = _inputs(torch, tgs)
    ok = torch.zeros(256, 256, 3, device="cuda")
    tgs.raster_forward_noalloc(blocks2, 20000, cfg2["cams"][0], (0, 0, 0), ok)
    torch.cuda.synchronize()
    assert ok.abs().sum().item() > 0
