"""Pins of the oracle's geometry: SH basis, Morton blocking, bounding spheres,
Level-1 culling and the Level-2 projection (CPU only)."""
import math

import numpy as np
import pytest

import scenes


def test_sh_basis_matches_scipy(orc):
    """Real SH (l <= 3) = sqrt(2) Re/Im of scipy's Condon-Shortley harmonics."""
    from scipy.special import sph_harm_y
    rng = np.random.default_rng(7)
    d = rng.normal(size=(200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    ref = np.zeros((200, 16))
    k = 0
    for l in range(4):
        for m in range(-l, l + 1):
            if m == 0:
                ref[:, k] = sph_harm_y(l, 0, theta, phi).real
            elif m > 0:
                ref[:, k] = math.sqrt(2) * sph_harm_y(l, m, theta, phi).real
            else:
                ref[:, k] = math.sqrt(2) * sph_harm_y(l, -m, theta, phi).imag
            k += 1
    got = orc.sh_basis(d)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)


def test_sh_basis_orthonormal(orc):
    """Monte-Carlo check that the 16 functions are orthonormal on the sphere."""
    rng = np.random.default_rng(8)
    d = rng.normal(size=(400000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = orc.sh_basis(d)
    gram = 4 * math.pi * (Y.T @ Y) / d.shape[0]
    np.testing.assert_allclose(gram, np.eye(16), atol=0.02)


def _interleave(q):
    c = np.zeros(q.shape[0], np.uint64)
    for b in range(10):
        for a in range(3):
            c |= ((q[:, a].astype(np.uint64) >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + a)
    return c.astype(np.uint32)


def test_morton_codes_bruteforce(orc):
    """Codes equal an independent float32 numpy quantisation + bit interleave,
    and the block order equals a stable argsort of the codes."""
    p = scenes.cube_scene(5000, seed=3)
    m = p[:, 0:3].astype(np.float32)
    # include exact extremes and duplicates
    m[10] = m[11]
    lo, hi = m.min(0), m.max(0)
    f = ((m - lo) / (hi - lo)).astype(np.float32) * np.float32(1024.0)
    q = np.clip(np.floor(f), 0, 1023).astype(np.int64)
    ref = _interleave(q)
    got = orc.morton_codes(m)
    assert np.array_equal(got, ref)
    perm = orc.block_order(got)
    assert np.array_equal(perm, np.argsort(ref, kind="stable"))
    # the maximum coordinate maps to cell 1023, the minimum to 0
    assert q.max() == 1023 and q.min() == 0


def test_morton_locality(orc):
    """Morton blocks are spatially compact: mean block extent far below the scene's."""
    p = scenes.cube_scene(16384, seed=4)
    perm, P = orc.create(p, 1024)
    sph = orc.block_spheres(P.astype(np.float64), 1024)
    perm_rand = np.random.default_rng(0).permutation(16384)
    sph_rand = orc.block_spheres(p[perm_rand].astype(np.float64), 1024)
    assert sph[:, 3].mean() < 0.7 * sph_rand[:, 3].mean()
    assert np.array_equal(np.sort(perm), np.arange(16384))


def test_block_spheres_contain_and_are_tight(orc):
    """Each block sphere contains every member's 3-sigma ball and touches one;
    the last block is truncated at N (Eq. block_def)."""
    p = scenes.cube_scene(3000, seed=5).astype(np.float64)
    B = 700
    sph = orc.block_spheres(p, B)
    assert sph.shape[0] == math.ceil(3000 / B)
    for k in range(sph.shape[0]):
        rows = p[k * B:min(3000, (k + 1) * B)]
        c, r = sph[k, :3], sph[k, 3]
        reach = np.linalg.norm(rows[:, :3] - c, axis=1) + 3 * np.exp(rows[:, 3:6]).max(1)
        assert reach.max() <= r * (1 + 1e-14)
        assert reach.max() >= r * (1 - 1e-14)
        np.testing.assert_allclose(c, 0.5 * (rows[:, :3].min(0) + rows[:, :3].max(0)), atol=0)


def _axis_camera(W=64, H=48, f=50.0):
    # camera at the origin looking down +z of the world, x right, y down
    return scenes.camera_array(dict(width=W, height=H, fx=f, fy=f, cx=W / 2 - 0.5, cy=H / 2 - 0.5,
                                    znear=0.2, zfar=100.0, R=np.eye(3), t=np.zeros(3)))


def test_cull_hand_cases(orc):
    """Spheres placed by hand against an axis-aligned camera."""
    cam = _axis_camera()
    pl = orc.frustum_planes(cam, margin=0.0)
    # the left plane passes through the origin and the pixel column u = 0:
    # direction (x, z) with f x / z + cx = 0 -> x = -cx z / f
    cx, f = cam[4], cam[2]
    n_left = np.array([f, 0.0, cx]) / math.hypot(f, cx)
    z = 10.0
    x_edge = -cx * z / f
    tests = []
    for dist, expect in [(1.0 + 1e-6, 0), (1.0 - 1e-6, 1)]:
        # centre outside the left plane at signed distance -dist * r with r = 1
        c = np.array([x_edge, 0.0, z]) - dist * n_left
        tests.append((c, 1.0, expect))
    tests.append((np.array([0, 0, 0.0]), 0.5, 1))    # around the camera centre
    tests.append((np.array([0, 0, -5.0]), 1.0, 0))   # behind the camera
    tests.append((np.array([0, 0, 150.0]), 10.0, 0))  # beyond the far plane
    tests.append((np.array([0, 0, 105.0]), 10.0, 1))  # straddling the far plane
    sph = np.array([[*c, r] for c, r, _ in tests])
    vis, marg = orc.cull(sph, pl)
    assert list(vis) == [e for _, _, e in tests]
    # plane normals point inward and are unit length
    np.testing.assert_allclose(np.linalg.norm(pl[:, :3], axis=1), 1.0, atol=1e-15)


def test_cull_conservative_on_small_cube(orc):
    """Every Gaussian that Level 2 renders lies in a block that Level 1 keeps
    (Sec. 3.3: Level 1 is conservative), for cameras that see part of the scene."""
    cfg = scenes.small_cube_config()
    perm, P = orc.create(cfg["params"], 625)
    P = P.astype(np.float64)
    sph = orc.block_spheres(P, 625)
    blk = np.arange(P.shape[0]) // 625
    culled = 0
    for pos, tgt, fov in (([0.5, 0.5, 0.5], [2, 2, 2], 60.0), ([0, 0, -3.0], [0.8, 0.8, 0], 25.0),
                          ([-0.5, 0.2, 0.0], [-3, 0.5, 0.2], 90.0)):
        R, t = scenes.look_at(pos, tgt)
        cam = scenes.camera_array(scenes.pinhole(128, 96, fov, R, t))
        vis, _ = orc.cull(sph, orc.frustum_planes(cam))
        S = orc.preprocess(P, cam, fp32key=False)
        used = np.unique(blk[S[:, orc.VISIBLE] != 0])
        assert vis[used].all()
        culled += len(vis) - vis.sum()
    assert culled >= 10  # the test exercises actual culling


def test_cull_fp32_rule_matches_fp64(orc):
    """The FP32 specification of the test decides every seeded block like FP64."""
    cfg = scenes.small_cube_config()
    perm, P = orc.create(cfg["params"], 625)
    sph = orc.block_spheres(P.astype(np.float64), 625)
    sph32 = sph.astype(np.float32).astype(np.float64)
    for pos in ([0.0, 0.0, -1.6], [0.9, 0.2, -1.3], [1.5, 1.5, 1.5], [0, 0, -3.0]):
        R, t = scenes.look_at(pos, [0.3, 0.1, 0.0])
        cam = scenes.camera_array(scenes.pinhole(128, 96, 60.0, R, t))
        v64, m = orc.cull(sph32, orc.frustum_planes(cam, fp32=False))
        v32, _ = orc.cull(sph32, orc.frustum_planes(cam, fp32=True), fp32=True)
        assert np.array_equal(v32, v64)
        assert m.min() > 1e-6


def test_projection_hand_placed_camera(orc):
    """A small bright Gaussian at world (0, 0.5, 0) seen from (3, 0, 0) looking
    at the origin (y up) lands at (cx, cy - f * 0.5 / 3)."""
    W = H = 96
    f = 80.0
    # camera basis written out by hand: forward -x, right -z, down -y
    R = np.array([[0, 0, -1.0], [0, -1.0, 0], [-1.0, 0, 0]])
    pos = np.array([3.0, 0, 0])
    cam = scenes.camera_array(dict(width=W, height=H, fx=f, fy=f, cx=W / 2 - 0.5, cy=H / 2 - 0.5,
                                   znear=0.2, zfar=100.0, R=R, t=-R @ pos))
    p = np.zeros((1, 59))
    p[0, 0:3] = [0.0, 0.5, 0.0]
    p[0, 3:6] = math.log(0.02)
    p[0, 6] = 1.0
    p[0, 10] = 4.0
    S = orc.preprocess(p, cam, fp32key=False)
    assert S[0, orc.VISIBLE] == 1
    np.testing.assert_allclose(S[0, orc.U], W / 2 - 0.5, atol=1e-12)
    np.testing.assert_allclose(S[0, orc.V], H / 2 - 0.5 - f * 0.5 / 3.0, atol=1e-12)
    np.testing.assert_allclose(S[0, orc.DEPTH], 3.0, atol=1e-12)


@pytest.mark.parametrize("sigma,z0,opl", [(0.01, 2.0, 0.0), (0.03, 3.0, 2.0), (0.005, 1.0, -1.0)])
def test_single_gaussian_closed_form(orc, sigma, z0, opl):
    """Isotropic Gaussian on the optical axis: cov2D = ((f sigma/z0)^2 + 0.3) I;
    alpha(rho) = min(0.99, sigmoid(o) exp(-rho^2 / (2 s2))); C = alpha rgb + (1-alpha) bg
    with rgb = 0.5 + DC / (2 sqrt(pi)) (DC only)."""
    W, H, f = 64, 64, 60.0
    cam = scenes.camera_array(dict(width=W, height=H, fx=f, fy=f, cx=W / 2 - 0.5, cy=H / 2 - 0.5,
                                   znear=0.2, zfar=100.0, R=np.eye(3), t=np.zeros(3)))
    p = np.zeros((1, 59))
    p[0, 0:3] = [0, 0, z0]
    p[0, 3:6] = math.log(sigma)
    p[0, 6:10] = [0.3, -0.5, 0.2, 0.7]  # rotation is irrelevant for an isotropic Gaussian
    p[0, 10] = opl
    dc = np.array([0.4, -0.2, 0.9])
    p[0, 11:14] = dc
    bg = np.array([0.1, 0.2, 0.3])
    r = orc.render(p, cam, bg=bg, fp32key=False)
    s2 = (f * sigma / z0) ** 2 + 0.3
    rgb = np.maximum(0.5 + dc / (2 * math.sqrt(math.pi)), 0)
    op = 1 / (1 + math.exp(-opl))
    yy, xx = np.mgrid[0:H, 0:W]
    rho2 = (xx - (W / 2 - 0.5)) ** 2 + (yy - (H / 2 - 0.5)) ** 2
    a = np.minimum(0.99, op * np.exp(-rho2 / (2 * s2)))
    a = np.where(a >= 1 / 255, a, 0.0)
    # tile coverage: pixels outside the splat's tile rect are not evaluated
    S = r["S"]
    x0, y0, x1, y1 = (int(S[0, c]) for c in (orc.X0, orc.Y0, orc.X1, orc.Y1))
    inside = (xx // 16 >= x0) & (xx // 16 < x1) & (yy // 16 >= y0) & (yy // 16 < y1)
    a = np.where(inside, a, 0.0)
    expect = a[..., None] * rgb + (1 - a[..., None]) * bg
    np.testing.assert_allclose(r["img"], expect, atol=1e-12)
    rad = math.ceil(3 * math.sqrt(s2 + math.sqrt(0.1)))
    assert S[0, orc.RADIUS] == rad


def test_clamp_and_dilation_radius(orc):
    """lambda1 uses max(0.1, mid^2 - det): for an isotropic splat mid^2 = det, so
    lambda1 = s2 + sqrt(0.1) exactly."""
    cam = _axis_camera(64, 64, 60.0)
    p = np.zeros((1, 59))
    p[0, 2] = 2.0
    p[0, 3:6] = math.log(0.02)
    p[0, 6] = 1.0
    S = orc.preprocess(p, cam, fp32key=False)
    s2 = (60.0 * 0.02 / 2.0) ** 2 + 0.3
    np.testing.assert_allclose(S[0, 23], s2 + math.sqrt(0.1), rtol=1e-14)
    np.testing.assert_allclose(S[0, orc.CA], 1 / s2, rtol=1e-14)
    np.testing.assert_allclose(S[0, orc.CB], 0.0, atol=1e-18)
