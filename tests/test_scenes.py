"""Pins of the seeded input generators (CPU): SplitMix64 against its published
test vector, the counter-based streams' independence of the requested range,
the torch streams (used for scenes of 10^8 Gaussians) against the numpy ones,
the moments of the uniform and Box-Muller normal draws, the street scene's
neighbourhood rows against the same rows of the full table (the full-size
parity tests run the oracle on such neighbourhoods), and the camera paths
against their recipe (the street drive: 2 m per frame at 1.5 m on the road
centre lines, turns at 400 m marks; the aerial lawnmower: 150 m, 45 degrees
down, 8 m per frame, passes 400 m apart)."""
import numpy as np

import scenes


def test_splitmix64_published_sequence():
    # the first five outputs of SplitMix64 seeded with 1234567, the test
    # vector that accompanies the generator's public reference code
    want = np.array([6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
                     16408922859458223821], np.uint64)
    with np.errstate(over="ignore"):
        got = scenes._mix64(np.uint64(1234567) + np.arange(1, 6, dtype=np.uint64) * scenes.GAMMA)
    assert np.array_equal(got, want)


def test_streams_are_counter_based():
    full = scenes.u64(7, 3, 0, 1000)
    assert np.array_equal(scenes.u64(7, 3, 400, 100), full[400:500])
    assert not np.any(scenes.u64(7, 4, 0, 1000) == full)
    assert not np.any(scenes.u64(8, 3, 0, 1000) == full)
    z = scenes.normal(7, 3, 500)
    assert np.array_equal(scenes.normal(7, 3, 100, start=200), z[200:300])
    u = scenes.uniform(7, 3, 500, -2.0, 3.0)
    assert np.array_equal(scenes.uniform(7, 3, 50, -2.0, 3.0, start=450), u[450:])


def test_torch_streams_match_numpy():
    import torch
    a = scenes.u64(11, 5, 123, 4096).view(np.int64)
    b = scenes.t_u64(11, 5, 123, 4096, "cpu").numpy()
    assert np.array_equal(a, b)
    idx = torch.tensor([0, 1, 17, 4095, 10 ** 9], dtype=torch.int64)
    at = scenes.t_u64_at(11, 5, idx).numpy()
    ref = np.concatenate([scenes.u64(11, 5, int(i), 1) for i in idx]).view(np.int64)
    assert np.array_equal(at, ref)
    assert np.array_equal(scenes.t_uniform(11, 5, 4096, -1.0, 2.0, device="cpu").numpy(),
                          scenes.uniform(11, 5, 4096, -1.0, 2.0))
    np.testing.assert_allclose(scenes.t_normal(11, 5, 4096, 0.5, 2.0, device="cpu").numpy(),
                               scenes.normal(11, 5, 4096, 0.5, 2.0), rtol=0, atol=1e-13)


def test_uniform_and_normal_moments():
    m = 1_000_000
    u = scenes.uniform(1, 2, m)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * (1 / 12) ** 0.5 / m ** 0.5
    assert abs(u.var() - 1 / 12) < 1e-3
    z = scenes.normal(1, 2, m)
    assert abs(z.mean()) < 5 / m ** 0.5
    assert abs(z.std() - 1.0) < 5e-3
    assert abs(np.mean(z ** 4) - 3.0) < 0.05  # Gaussian kurtosis
    assert abs(np.mean(np.abs(z) < 1.0) - 0.682689492) < 3e-3


def test_street_neighbourhood_rows_equal_the_full_table():
    import torch
    n = 200_000
    full, sp = scenes.street_scene(n, device="cpu", chunk=1 << 16)
    c = np.array([10.0, -40.0, 1.5])
    r = 400.0
    rows, idx, sp2 = scenes.street_scene(n, device="cpu", chunk=50_000, near=(c, r))
    assert sp == sp2
    sel = ((full[:, :3].double() - torch.tensor(c)) ** 2).sum(1) < r * r
    want = torch.nonzero(sel).squeeze(1)
    assert len(want) > 1000
    assert torch.equal(idx, want)
    assert torch.equal(rows, full[want])
    # quaternions unit, opacity logits and log-scales finite
    q = full[:, 6:10].double()
    assert torch.allclose(q.norm(dim=1), torch.ones(n, dtype=torch.float64), atol=1e-6)
    assert torch.isfinite(full).all()


def _centre_and_view(cam):
    R = np.asarray(cam["R"], np.float64)
    t = np.asarray(cam["t"], np.float64)
    return -R.T @ t, R[2]  # camera centre, viewing direction (camera +z) in the world


def test_street_drive_follows_the_road_grid():
    cams = scenes.street_drive_cameras(500)
    assert len(cams) == 500
    c = np.array([_centre_and_view(k)[0] for k in cams])
    v = np.array([_centre_and_view(k)[1] for k in cams])
    for k in cams[:3]:
        R = np.asarray(k["R"])
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-12) and np.linalg.det(R) > 0
        assert (k["width"], k["height"], k["zfar"]) == (1600, 900, 200.0)
        assert abs(2 * np.degrees(np.arctan(0.5 * k["width"] / k["fx"])) - 90.0) < 1e-9
    assert np.allclose(c[:, 2], 1.5)                       # 1.5 m above the ground
    assert np.allclose(np.linalg.norm(np.diff(c[:, :2], axis=0), axis=1), 2.0)  # 2 m per frame
    assert np.all(np.abs(c[:, :2]) < 2000.0)               # inside the 4 km square
    assert np.allclose(v[:, 2], 0.0) and np.allclose(np.linalg.norm(v, axis=1), 1.0)
    # on a road centre line: the coordinate across the direction of travel is a
    # multiple of 100 m
    across = np.where(np.abs(v[:, 0]) > 0.5, c[:, 1], c[:, 0])
    r = np.mod(across + 2000.0, 100.0)
    assert np.all(np.minimum(r, 100.0 - r) < 1e-9)
    # the heading changes only at 400 m (200-frame) marks, by a quarter turn or a reversal
    turns = np.nonzero(np.any(np.abs(np.diff(v, axis=0)) > 1e-9, axis=1))[0] + 1
    assert len(turns) >= 2 and np.all(turns % 200 == 0)


def test_lawnmower_passes():
    cams = scenes.lawnmower_cameras(1000)
    c = np.array([_centre_and_view(k)[0] for k in cams])
    v = np.array([_centre_and_view(k)[1] for k in cams])
    assert np.allclose(c[:, 2], 150.0)
    assert np.allclose(np.degrees(np.arcsin(-v[:, 2])), 45.0)  # pitched 45 degrees down
    assert (cams[0]["width"], cams[0]["height"], cams[0]["zfar"]) == (1920, 1080, 600.0)
    step = np.linalg.norm(np.diff(c[:, :2], axis=0), axis=1)
    same_pass = np.isclose(np.diff(c[:, 1]), 0.0)
    assert same_pass.sum() > 900 and np.allclose(step[same_pass], 8.0)  # 8 m per frame along a pass
    ys = np.unique(np.round(c[:, 1], 6))
    assert len(ys) >= 2 and np.allclose(np.diff(ys), 400.0)    # passes 400 m apart
    assert np.all(np.abs(c[:, :2]) <= 2000.0)


def test_street_scene_recipe():
    n = 200_000
    full, spacing = scenes.street_scene(n, device="cpu", chunk=1 << 16)
    p = full.double().numpy()
    ng = n // 2
    assert np.all(p[:ng, 2] == 0.0)                        # the ground layer
    assert np.all(np.abs(p[:, :2]) <= 2000.0)              # inside the 4 km square
    z = p[ng:, 2]
    assert z.min() >= 0.0 and z.max() <= 60.0 and np.mean(z > 0) > 0.99  # facades up to 60 m
    ls = p[:, 3:6].ravel()
    assert abs(ls.mean() - np.log(0.5 * spacing)) < 0.005 and abs(ls.std() - 0.3) < 0.005
    assert abs(p[:, 10].mean() - 2.0) < 0.01 and abs(p[:, 10].std() - 0.5) < 0.01
    rest = p[:, 14:59].ravel()
    assert abs(rest.mean()) < 1e-3 and abs(rest.std() - 0.05) < 1e-3
