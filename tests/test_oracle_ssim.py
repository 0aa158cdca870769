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
