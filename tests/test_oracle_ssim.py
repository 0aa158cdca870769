"""Pins of the D-SSIM loss oracle (CPU): identities of SSIM, a brute-force
per-pixel window sum written from the definition, and central finite
differences of the loss gradient."""
import numpy as np


def _imgs(rng, H=13, W=11):
    x = rng.uniform(0.0, 1.0, (H, W, 3))
    y = np.clip(x + rng.normal(0.0, 0.15, x.shape), 0.0, 1.0)
    return x, y


def test_ssim_identities():
    from oracle import ssim
    rng = np.random.default_rng(0)
    x, y = _imgs(rng)
    assert abs(ssim.ssim(x, x) - 1.0) < 1e-12
    assert abs(ssim.ssim(x, y) - ssim.ssim(y, x)) < 1e-14
    assert ssim.ssim(x, y) < 0.99
    w = ssim.window_1d()
    assert abs(w.sum() - 1.0) < 1e-15 and np.allclose(w, w[::-1])


def test_ssim_matches_brute_force_window_sums():
    from oracle import ssim
    rng = np.random.default_rng(1)
    x, y = _imgs(rng, 9, 12)
    H, W, _ = x.shape
    w = ssim.window_1d()
    r = len(w) // 2
    S = np.zeros(x.shape)
    for i in range(H):
        for j in range(W):
            for c in range(3):
                mx = my = exx = eyy = exy = 0.0
                for a in range(-r, r + 1):
                    for b in range(-r, r + 1):
                        ii, jj = i + a, j + b
                        if 0 <= ii < H and 0 <= jj < W:
                            g = w[a + r] * w[b + r]
                            xv, yv = x[ii, jj, c], y[ii, jj, c]
                            mx += g * xv
                            my += g * yv
                            exx += g * xv * xv
                            eyy += g * yv * yv
                            exy += g * xv * yv
                num = (2 * mx * my + ssim.C1) * (2 * (exy - mx * my) + ssim.C2)
                den = (mx * mx + my * my + ssim.C1) * ((exx - mx * mx) + (eyy - my * my) + ssim.C2)
                S[i, j, c] = num / den
    np.testing.assert_allclose(ssim.ssim_terms(x, y)["S"], S, rtol=1e-12, atol=1e-14)


def test_loss_gradient_matches_finite_differences():
    from oracle import ssim
    rng = np.random.default_rng(2)
    x, y = _imgs(rng)
    g = ssim.loss_grad(x, y)
    gs = ssim.ssim_grad(x, y)
    h = 1e-6
    for idx in [tuple(rng.integers(0, s) for s in x.shape) for _ in range(40)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (ssim.ssim(xp, y) - ssim.ssim(xm, y)) / (2 * h)
        assert abs(gs[idx] - fd) <= 1e-8 + 1e-5 * abs(fd), idx
        fdl = (ssim.loss(xp, y) - ssim.loss(xm, y)) / (2 * h)
        assert abs(g[idx] - fdl) <= 1e-8 + 1e-5 * abs(fdl), idx


def test_window_matches_scipy_gaussian_filter():
    """The 11 x 11 window with zero padding is scipy's Gaussian filter with
    sigma 1.5 truncated at radius 5 (its kernel renormalised over the
    truncated support) and constant-zero boundary mode."""
    from scipy.ndimage import gaussian_filter
    from oracle import ssim
    rng = np.random.default_rng(3)
    a = rng.uniform(0.0, 1.0, (17, 14, 3))
    ref = np.stack([gaussian_filter(a[..., c], sigma=1.5, truncate=5.0 / 1.5, mode="constant", cval=0.0)
                    for c in range(3)], axis=-1)
    np.testing.assert_allclose(ssim.blur(a), ref, rtol=1e-12, atol=1e-14)


def test_constant_images_closed_form():
    """Away from the border (every window inside the image) two constant
    images a and b have zero variances and covariance, so
    SSIM = (2ab + C1) / (a^2 + b^2 + C1) with C1 = (0.01 x 1)^2."""
    from oracle import ssim
    H, W = 16, 15
    for a, b in ((0.3, 0.7), (0.0, 0.5), (0.9, 0.9), (0.02, 0.01)):
        x = np.full((H, W, 3), a)
        y = np.full((H, W, 3), b)
        S = ssim.ssim_terms(x, y)["S"][5:H - 5, 5:W - 5]
        want = (2 * a * b + 1e-4) / (a * a + b * b + 1e-4)
        np.testing.assert_allclose(S, want, rtol=1e-12)


def test_structure_term_closed_form():
    """Away from the border, x = a + d and y = a + k d for a zero-mean
    checkerboard d of amplitude s: the window means of x and y are a + e and
    a + k e, and variances / covariance follow from E[d^2] and e; the SSIM
    then has the closed form below, which involves C2 = (0.03 x 1)^2."""
    from oracle import ssim
    H, W = 24, 23
    ii, jj = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    d = np.where((ii + jj) % 2 == 0, 1.0, -1.0)[..., None] * np.ones(3)
    a, s, k = 0.5, 0.1, -0.6
    x, y = a + s * d, a + k * s * d
    t = ssim.ssim_terms(x, y)
    w = ssim.window_1d()
    # window mean of the checkerboard at (i, j): (sum_even w - sum_odd w)^2 times the sign of d
    alt = (w[0::2].sum() - w[1::2].sum()) ** 2
    for i, j in ((8, 9), (12, 11), (10, 10)):
        e = s * d[i, j, 0] * alt
        mx, my = a + e, a + k * e
        vx = s * s - e * e          # E[(s d)^2] - e^2
        vy = k * k * vx
        cxy = k * vx
        want = (2 * mx * my + 1e-4) * (2 * cxy + 9e-4) / ((mx * mx + my * my + 1e-4) * (vx + vy + 9e-4))
        np.testing.assert_allclose(t["S"][i, j], want, rtol=1e-10)


def test_batch_is_the_mean_of_its_images():
    """A batch of J same-size images: the loss is the mean of the per-image
    losses and each image's gradient is its own gradient divided by J (no
    window crosses from one image into the next)."""
    from oracle import ssim
    rng = np.random.default_rng(5)
    xs, ys = zip(*[_imgs(rng, 10, 12) for _ in range(3)])
    X, Y = np.stack(xs), np.stack(ys)
    per = [ssim.loss(x, y) for x, y in zip(xs, ys)]
    assert abs(ssim.loss(X, Y) - np.mean(per)) < 1e-14
    G = ssim.loss_grad(X, Y)
    for j, (x, y) in enumerate(zip(xs, ys)):
        np.testing.assert_allclose(G[j], ssim.loss_grad(x, y) / 3.0, rtol=1e-12, atol=1e-18)
