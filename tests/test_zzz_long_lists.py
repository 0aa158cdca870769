"""Tile lists longer than the binning's shared-memory sort, through the C ABI:
32,000 small Gaussians piled along the view rays of two tiles of a 32x32
image (20,000 in one tile, 12,000 in another, depths U[2, 10]), so the
per-tile sort takes runs of 8,192 keys merged in global memory (two merge
levels for one tile, one for the other), and the backward takes each list
whole (a 32x32 image has 16 checkpoint slots, fewer than the 79 and 47
segments the lists would need), recomputing the transmittance in reverse
over up to 20,000 positions.  One L2 step is checked
against the oracle as in the small-cube parity test: visible set, splat
records, the per-tile pair sequences bit-exact, image, T_final, n_last, 2D
and 59-column gradients, the Adam update and the refreshed spheres."""
import numpy as np
import pytest

import scenes
from test_gpu_parity import _check_step

pytestmark = pytest.mark.gpu

W = H = 32
B = 4000


def _pile(cam, n, px, py, seed):
    """n means whose projections fall within 2.5 px of pixel (px, py), at
    depths U[2, 10]."""
    z = scenes.uniform(seed, 1, n, 2.0, 10.0)
    u = px + scenes.uniform(seed, 2, n, -2.5, 2.5)
    v = py + scenes.uniform(seed, 3, n, -2.5, 2.5)
    xc = np.stack([(u - cam["cx"]) / cam["fx"] * z, (v - cam["cy"]) / cam["fy"] * z, z], 1)
    return (xc - cam["t"]) @ cam["R"]  # world = R^T (x_c - t)


def _scene(cam):
    n0, n3 = 20000, 12000
    n = n0 + n3
    p = np.zeros((n, 59), np.float32)
    p[:, 0:3] = np.concatenate([_pile(cam, n0, 7.5, 7.5, 11), _pile(cam, n3, 23.5, 23.5, 12)])
    p[:, 3:6] = -6.0 + scenes.normal(13, 1, 3 * n, 0.0, 0.2).reshape(n, 3)
    q = scenes.normal(13, 2, 4 * n).reshape(n, 4)
    p[:, 6:10] = q / np.linalg.norm(q, axis=1, keepdims=True)
    p[:, 10] = scenes.normal(13, 3, n, 0.0, 1.0)
    p[:, 11:59] = scenes.normal(13, 4, 48 * n, 0.0, 0.2).reshape(n, 48)
    return p


def test_step_with_lists_above_the_shared_memory_sort(orc, tgs):
    R, t = scenes.look_at([0.0, 0.0, 0.0], [0.0, 0.0, 1.0])
    cam = scenes.pinhole(W, H, 60.0, R, t)
    params = _scene(cam)
    # the oracle's binning: the intended list lengths, no border Gaussian (so
    # that every tile's sequence is compared)
    _, Pm = orc.create(params, B)
    S = orc.preprocess(Pm.astype(np.float64), scenes.camera_array(cam))
    assert not (S[:, orc.BORDER] != 0).any()
    _, _, ranges = orc.bin_sort(S, W, H)
    assert list(ranges[:, 1].astype(np.int64) - ranges[:, 0]) == [20000, 0, 0, 12000]
    target = np.full((H, W, 3), 0.2, np.float32)
    _check_step(orc, tgs, params, B, cam, target, 1, W, H)
