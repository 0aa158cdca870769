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


# ----------------------------------------------------------------------------
# Anisotropic, rotated and off-axis projection (standard EWA splatting, the
# Level-2 preprocess of Sec. 3.3): pinned against scipy's rotations and a
# finite-difference linearisation of the pinhole map, so that a transposed
# rotation, a conjugated quaternion or a swapped off-diagonal term fails.
# ----------------------------------------------------------------------------
def _conic_to_cov(S, i):
    """2D covariance (dilated) of splat i from the oracle's conic (A, B, C):
    the conic is its inverse, [[A, B], [B, C]] = cov^-1."""
    A, B, C = S[i, 3], S[i, 4], S[i, 5]
    return np.linalg.inv(np.array([[A, B], [B, C]]))


def _sigma_scipy(quat_wxyz, scales):
    """World covariance R diag(s^2) R^T with R from scipy (scalar-last order)."""
    from scipy.spatial.transform import Rotation
    w, x, y, z = quat_wxyz
    Rq = Rotation.from_quat([x, y, z, w]).as_matrix()
    return Rq @ np.diag(np.asarray(scales) ** 2) @ Rq.T


def test_quarter_turn_about_z_swaps_the_2d_variances(orc):
    """q = (cos 45, 0, 0, sin 45) maps x to y: an on-axis Gaussian with scales
    (s1, s2, s3) projects to diag((f s2/z)^2 + 0.3, (f s1/z)^2 + 0.3) exactly
    (the camera looks down +z, no skew term)."""
    f, z0 = 70.0, 2.5
    cam = _axis_camera(64, 64, f)
    s1, s2, s3 = 0.011, 0.047, 0.02
    p = np.zeros((1, 59))
    p[0, 2] = z0
    p[0, 3:6] = np.log([s1, s2, s3])
    p[0, 6:10] = [math.cos(math.pi / 4), 0.0, 0.0, math.sin(math.pi / 4)]
    S = orc.preprocess(p, cam, fp32key=False)
    assert S[0, orc.VISIBLE] == 1
    a = (f * s2 / z0) ** 2 + 0.3
    c = (f * s1 / z0) ** 2 + 0.3
    np.testing.assert_allclose(S[0, orc.CA], 1.0 / a, rtol=1e-12)
    np.testing.assert_allclose(S[0, orc.CC], 1.0 / c, rtol=1e-12)
    assert abs(S[0, orc.CB]) < 1e-12 * S[0, orc.CA]
    # lambda1 = the larger variance (mid^2 - det = ((a - c)/2)^2 > 0.1 here)
    np.testing.assert_allclose(S[0, 23], max(a, c), rtol=1e-12)


def test_rotation_matches_scipy_on_axis(orc):
    """On the optical axis of an identity camera the Jacobian is diag(f/z, f/z)
    in its first two columns and zero in the third, so the 2D covariance is
    (f/z)^2 times the top-left 2x2 block of the world covariance plus 0.3 I;
    the world covariance comes from scipy's rotation of random (unnormalised)
    quaternions with anisotropic scales."""
    rng = np.random.default_rng(31)
    f, z0 = 90.0, 3.0
    cam = _axis_camera(96, 96, f)
    n = 64
    p = np.zeros((n, 59))
    p[:, 2] = z0
    scales = np.exp(rng.uniform(np.log(0.005), np.log(0.05), size=(n, 3)))
    p[:, 3:6] = np.log(scales)
    p[:, 6:10] = rng.normal(size=(n, 4)) * 2.7
    S = orc.preprocess(p, cam, fp32key=False)
    for i in range(n):
        Sig = _sigma_scipy(p[i, 6:10], scales[i])
        expect = (f / z0) ** 2 * Sig[:2, :2] + 0.3 * np.eye(2)
        np.testing.assert_allclose(_conic_to_cov(S, i), expect, rtol=1e-10, atol=1e-12)


def test_off_axis_projection_matches_finite_difference_linearisation(orc):
    """EWA projects the world covariance through the linearisation of the
    pinhole map at the mean: cov2D = J Sigma J^T + 0.3 I with J = d(u, v)/d(mu).
    Here J is taken by central differences of the projection itself (not the
    analytic formula), for random camera poses, rotations and anisotropic
    scales with the mean well inside the Jacobian's clamp limits."""
    rng = np.random.default_rng(32)
    W = H = 128
    for trial in range(24):
        pos = rng.normal(size=3) * 2.0
        tgt = rng.normal(size=3) * 0.3
        R, t = scenes.look_at(pos, tgt, up=tuple(rng.normal(size=3)))
        camd = scenes.pinhole(W, H, 65.0, R, t)
        cam = scenes.camera_array(camd)
        fx, fy, cx, cy = camd["fx"], camd["fy"], camd["cx"], camd["cy"]
        # a mean in view: camera coordinates (x, y, z) with |x/z|, |y/z| < 0.5
        zc = rng.uniform(1.0, 4.0)
        xc, yc = rng.uniform(-0.5, 0.5, size=2) * zc
        mu = R.T @ (np.array([xc, yc, zc]) - t)
        scales = np.exp(rng.uniform(np.log(0.004), np.log(0.04), size=3))
        q = rng.normal(size=4)
        p = np.zeros((1, 59))
        p[0, 0:3] = mu
        p[0, 3:6] = np.log(scales)
        p[0, 6:10] = q
        S = orc.preprocess(p, cam, fp32key=False)
        assert S[0, orc.VISIBLE] == 1

        def proj(m):
            c = R @ m + t
            return np.array([fx * c[0] / c[2] + cx, fy * c[1] / c[2] + cy])

        h = 1e-5
        Jfd = np.stack([(proj(mu + h * e) - proj(mu - h * e)) / (2 * h) for e in np.eye(3)], axis=1)
        expect = Jfd @ _sigma_scipy(q, scales) @ Jfd.T + 0.3 * np.eye(2)
        np.testing.assert_allclose(_conic_to_cov(S, 0), expect, rtol=1e-7, atol=1e-9)
        # the projected centre is the pinhole map of the mean
        np.testing.assert_allclose([S[0, orc.U], S[0, orc.V]], proj(mu), rtol=0, atol=1e-9)
