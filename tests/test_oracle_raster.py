"""Pins of the oracle's tile binning, compositing and analytic backward (CPU only)."""
import math

import numpy as np
import pytest

import scenes


def _tiny_scene(n=30, seed=11, W=48, H=40, big=False):
    rng = np.random.default_rng(seed)
    p = np.zeros((n, 59))
    p[:, 0] = rng.uniform(-0.6, 0.6, n)
    p[:, 1] = rng.uniform(-0.5, 0.5, n)
    p[:, 2] = rng.uniform(1.5, 3.0, n)
    p[:, 3:6] = rng.normal(math.log(0.08 if big else 0.04), 0.4, (n, 3))
    q = rng.normal(size=(n, 4))
    p[:, 6:10] = q / np.linalg.norm(q, axis=1, keepdims=True) * rng.uniform(0.5, 2.0, (n, 1))
    p[:, 10] = rng.normal(0.5, 1.0, n)
    p[:, 11:59] = rng.normal(0, 0.3, (n, 48))
    cam = scenes.camera_array(dict(width=W, height=H, fx=40.0, fy=42.0, cx=W / 2 - 0.5, cy=H / 2 - 0.5,
                                   znear=0.2, zfar=100.0, R=scenes.rot_y(4.0), t=np.array([0.05, -0.02, 0.1])))
    return p, cam


def _brute_render(orc, S, W, H, bg):
    """Untiled reference: for every pixel, every visible Gaussian whose tile
    rect contains the pixel's tile, ordered by (float32 depth, id), composited
    front to back with the stated rules."""
    img = np.zeros((H, W, 3))
    Tf = np.ones((H, W))
    vis = np.nonzero(S[:, orc.VISIBLE])[0]
    d32 = S[:, orc.DEPTH].astype(np.float32)
    order = sorted(vis, key=lambda i: (d32[i], i))
    for py in range(H):
        for px in range(W):
            tx, ty = px // 16, py // 16
            T, C = 1.0, np.zeros(3)
            for i in order:
                s = S[i]
                if not (s[orc.X0] <= tx < s[orc.X1] and s[orc.Y0] <= ty < s[orc.Y1]):
                    continue
                dx, dy = px - s[orc.U], py - s[orc.V]
                power = -0.5 * (s[orc.CA] * dx * dx + s[orc.CC] * dy * dy) - s[orc.CB] * dx * dy
                if power > 0:
                    continue
                a = min(0.99, s[orc.OPAC] * math.exp(power))
                if a < 1 / 255:
                    continue
                Tn = T * (1 - a)
                if Tn < 1e-4:
                    break
                C += s[orc.R:orc.B + 1] * a * T
                T = Tn
            img[py, px] = C + T * np.asarray(bg)
            Tf[py, px] = T
    return img, Tf


@pytest.mark.parametrize("seed", [11, 12])
def test_tiled_render_equals_untiled_bruteforce(orc, seed):
    p, cam = _tiny_scene(seed=seed, big=True)
    bg = np.array([0.2, 0.1, 0.05])
    r = orc.render(p, cam, bg=bg, fp32key=True)
    ref, Tref = _brute_render(orc, r["S"], 48, 40, bg)
    np.testing.assert_allclose(r["img"], ref, atol=1e-13)
    np.testing.assert_allclose(r["T"], Tref, atol=1e-13)
    assert r["S"][:, orc.VISIBLE].sum() >= 20


def test_sort_keys_and_ranges(orc):
    """Pairs are sorted by (tile, depth bits) with ties by id; ranges cover each tile."""
    p, cam = _tiny_scene(seed=13, big=True)
    r = orc.render(p, cam)
    keys, vals, ranges = r["keys"], r["vals"], r["ranges"]
    assert np.all(np.diff(keys.astype(np.float64)) >= 0) or np.all(keys[1:] >= keys[:-1])
    same = keys[1:] == keys[:-1]
    assert np.all(vals[1:][same] > vals[:-1][same])
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    for t in range(ranges.shape[0]):
        a, b = ranges[t]
        assert np.all(tiles[a:b] == t)
    assert sum(b - a for a, b in ranges) == len(keys)
    # every pair count equals the rect area
    S = r["S"]
    area = ((S[:, orc.X1] - S[:, orc.X0]) * (S[:, orc.Y1] - S[:, orc.Y0]) * S[:, orc.VISIBLE]).sum()
    assert area == len(keys)


def test_compositing_invariants(orc):
    """rgb = 1 and bg = 0 give image = 1 - T_final; T_final in [1e-4, 1];
    the order of the input rows does not change the image."""
    p, cam = _tiny_scene(n=60, seed=14, big=True)
    p[:, 11:59] = 0.0
    p[:, 11:14] = math.sqrt(math.pi)  # DC such that rgb = 0.5 + DC / (2 sqrt(pi)) = 1
    p[:, 10] = 3.0                    # opaque enough to trigger the T < 1e-4 stop
    r = orc.render(p, cam)
    np.testing.assert_allclose(r["img"][..., 0], 1.0 - r["T"], atol=1e-14)
    assert r["T"].min() >= 1e-4 and r["T"].max() <= 1.0
    assert (r["T"] < 2e-3).any()  # the stop rule was exercised
    perm = np.random.default_rng(0).permutation(p.shape[0])
    r2 = orc.render(p[perm], cam)
    np.testing.assert_allclose(r2["img"], r["img"], atol=1e-14)


def _fd_check(orc, p, cam, bg, w, cols, fp_h=1e-6):
    r = orc.render(p, cam, bg=bg, fp32key=False)
    g, _ = orc.render_grad(p, cam, r, w, bg)

    def f(pp):
        return float((orc.render(pp, cam, bg=bg, fp32key=False)["img"] * w).sum())

    checked = skipped = 0
    scale = np.abs(g).max()
    for i in range(p.shape[0]):
        for j in cols:
            h = fp_h * max(1.0, abs(p[i, j]))
            e = np.zeros_like(p)
            e[i, j] = h
            fd1 = (f(p + e) - f(p - e)) / (2 * h)
            fd2 = (f(p + e / 2) - f(p - e / 2)) / h
            if abs(fd1 - fd2) > 1e-6 * (abs(fd1) + 1e-3 * scale):
                skipped += 1  # a discontinuity (threshold, stop, tile edge) inside the stencil
                continue
            checked += 1
            assert abs(g[i, j] - fd1) <= 2e-6 * abs(fd1) + 1e-7 * scale, (i, j, g[i, j], fd1)
    return checked, skipped


def test_backward_matches_finite_differences(orc):
    """Central differences of <w, render(P)> w.r.t. all 59 columns (FP64 path)."""
    p, cam = _tiny_scene(n=12, seed=21, big=True)
    bg = np.array([0.3, 0.2, 0.1])
    w = np.random.default_rng(5).normal(size=(40, 48, 3))
    checked, skipped = _fd_check(orc, p, cam, bg, w, range(59))
    assert checked >= 0.9 * 12 * 59, (checked, skipped)


def test_backward_jacobian_clamp_branch(orc):
    """A large Gaussian whose centre lies beyond 1.3x the half field of view
    (so the Jacobian is taken at the clamped point) still gets exact gradients."""
    W, H = 48, 40
    cam = scenes.camera_array(dict(width=W, height=H, fx=40.0, fy=40.0, cx=W / 2 - 0.5, cy=H / 2 - 0.5,
                                   znear=0.2, zfar=100.0, R=np.eye(3), t=np.zeros(3)))
    p = np.zeros((2, 59))
    p[0, 0:3] = [1.85, 0.1, 2.0]   # tx/tz = 0.925 > 1.3 * 24/40 = 0.78
    p[0, 3:6] = [math.log(0.6), math.log(0.3), math.log(0.4)]
    p[1, 0:3] = [0.1, -1.3, 2.2]   # ty/tz beyond 1.3 * 20/40 = 0.65
    p[1, 3:6] = [math.log(0.3), math.log(0.5), math.log(0.2)]
    p[:, 6:10] = [[0.9, 0.2, -0.3, 0.1], [0.7, -0.1, 0.4, 0.3]]
    p[:, 10] = [1.0, 0.5]
    p[:, 11:59] = np.random.default_rng(3).normal(0, 0.3, (2, 48))
    S = orc.preprocess(p, cam, fp32key=False)
    assert S[:, orc.VISIBLE].all()
    w = np.random.default_rng(6).normal(size=(H, W, 3))
    checked, _ = _fd_check(orc, p, cam, np.zeros(3), w, range(10))
    assert checked >= 16


def test_backward_two_forms_agree(orc):
    """The reverse recurrence (T_i = T_{i+1} / (1 - alpha_i)) equals the
    stored-list form to rounding."""
    cfg = scenes.small_cube_config(n=4000, size=128)
    perm, P = orc.create(cfg["params"], 250)
    cam = scenes.camera_array(cfg["cams"][0])
    r = orc.render(P.astype(np.float64), cam, bg=(0.1, 0.2, 0.3))
    w = np.random.default_rng(1).normal(size=r["img"].shape)
    g0, g20 = orc.render_grad(P.astype(np.float64), cam, r, w, (0.1, 0.2, 0.3), mode=0)
    g1, g21 = orc.render_grad(P.astype(np.float64), cam, r, w, (0.1, 0.2, 0.3), mode=1)
    np.testing.assert_allclose(g20, g21, atol=1e-10 * np.abs(g21).max())
    np.testing.assert_allclose(g0, g1, atol=1e-10 * np.abs(g1).max())


def test_loss_values(orc):
    rng = np.random.default_rng(2)
    a, b = rng.random((2, 5, 7, 3)), rng.random((2, 5, 7, 3))
    l1, g1 = orc.loss(a, b, 0)
    l2, g2 = orc.loss(a, b, 1)
    assert abs(l1 - np.abs(a - b).mean()) < 1e-15
    assert abs(l2 - ((a - b) ** 2).mean()) < 1e-15
    np.testing.assert_allclose(g1, np.sign(a - b) / a.size)
    np.testing.assert_allclose(g2, 2 * (a - b) / a.size)


def _record(orc, u, v, depth, conic, opac, rgb=(0.5, 0.5, 0.5)):
    s = np.zeros(orc.NS)
    s[orc.U], s[orc.V], s[orc.DEPTH] = u, v, depth
    s[orc.CA], s[orc.CB], s[orc.CC] = conic
    s[orc.OPAC] = opac
    s[orc.R:orc.B + 1] = rgb
    s[orc.RADIUS] = 16
    s[orc.X0], s[orc.Y0], s[orc.X1], s[orc.Y1] = 0, 0, 1, 1
    s[orc.VISIBLE] = 1
    return s


def _composite(orc, S, W=16, H=16):
    _, vals, ranges = orc.bin_sort(S, W, H)
    return orc.composite_fwd(S, W, H, vals, ranges)


def test_slack_alpha_threshold_window_grows_with_power(orc):
    """An entry whose alpha lies within the FP32 error of the 1/255 skip gets
    slack; the window is about 1e-5 |power| relative (the power is a quadratic
    form of FP32 values), wider than tol_a: at |power| = 4.9 an alpha 2e-5
    above the threshold is borderline, one 1e-3 above is not."""
    o, px = 0.5, 10
    for delta, borderline in ((2e-5, True), (1e-3, False)):
        power = math.log((1.0 + delta) / (255.0 * o))
        a = -2.0 * power / (px * px)
        S = np.stack([_record(orc, 0.0, 0.0, 1.0, (a, 0.0, a), o)])
        img, T, nl, sl = _composite(orc, S)
        assert (sl[0, px] > 0) == borderline, (delta, sl[0, px])
        # the pixel's result includes the entry either way (alpha >= 1/255)
        assert abs(T[0, px] - (1.0 - o * math.exp(power))) < 1e-12
        # pixels one step nearer or farther are far from the threshold
        assert sl[0, px - 1] == 0 and sl[0, px + 1] == 0


def test_slack_stop_window_follows_the_transmittance_product(orc):
    """Three entries at the pixel centre (alpha = opacity): 0.9, 0.99
    (clamped) and 0.9 - 0.1 delta, so the third leaves T' = 1e-4 (1 + delta).
    The FP32 product of the factors carries a relative error of about
    sum alpha / (1 - alpha) times the alphas' errors, ~1e-4 here: delta = 5e-5
    is a borderline stop and gets slack of at least the transmittance left;
    delta = 1e-2 is not."""
    for delta, borderline in ((5e-5, True), (1e-2, False)):
        S = np.stack([_record(orc, 0.0, 0.0, 1.0, (1.0, 0.0, 1.0), 0.9),
                      _record(orc, 0.0, 0.0, 2.0, (1.0, 0.0, 1.0), 0.995),
                      _record(orc, 0.0, 0.0, 3.0, (1.0, 0.0, 1.0), 0.9 - 0.1 * delta)])
        img, T, nl, sl = _composite(orc, S)
        assert (sl[0, 0] > 0) == borderline, (delta, sl[0, 0])
        assert nl[0, 0] == 3  # T' >= 1e-4: the third entry is included
        if borderline:
            assert sl[0, 0] >= 2 * 1e-3 * 0.5  # 2 T max(rgb, bg) before the third entry
