"""FP64 oracle of the 3DGS photometric loss with the D-SSIM term.

TEST INFRASTRUCTURE ONLY (imported by tests and the benchmark's CPU leg).

The paper trains with the standard 3DGS recipe (Sec. 4, implementation
details); its loss f_i (App. A.1) is then (1 - lam) L1 + lam (1 - SSIM), lam =
0.2, with SSIM (Wang et al., 2004) computed per colour channel over an 11 x 11
Gaussian window (sigma 1.5, normalised), zero padding outside the image,
C1 = 0.01^2, C2 = 0.03^2, and averaged over every pixel and channel:

  m_x = G * x, m_y = G * y, s_xx = G * x^2 - m_x^2, s_yy = G * y^2 - m_y^2,
  s_xy = G * (x y) - m_x m_y,
  S = (2 m_x m_y + C1)(2 s_xy + C2) / ((m_x^2 + m_y^2 + C1)(s_xx + s_yy + C2)).

Its gradient with respect to the rendered image x: with e_xx = G * x^2 and
e_xy = G * (x y) the per-pixel partials of S are
  dS/dm_x  = 2 m_y (A2 - A1) / (B1 B2) - 2 m_x S (1/B1 - 1/B2),
  dS/de_xx = -S / B2,      dS/de_xy = 2 A1 / (B1 B2)
(A1, A2, B1, B2 the four factors above), and the adjoint of the zero-padded
correlation with the symmetric window is the same correlation, so
  d mean(S) / dx = (G * dS/dm_x + 2 x G * dS/de_xx + y G * dS/de_xy) / N.

Images are (..., H, W, 3) arrays; the window runs over H and W.
Pinned by tests/test_oracle_ssim.py: SSIM(x, x) = 1, symmetry, a brute-force
per-pixel window sum, and central finite differences of the loss.
"""
from __future__ import annotations

import numpy as np

WIN = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2
LAMBDA = 0.2


def window_1d(size=WIN, sigma=SIGMA):
    x = np.arange(size, dtype=np.float64) - (size // 2)
    g = np.exp(-(x * x) / (2.0 * sigma * sigma))
    return g / g.sum()


def blur(a, w=None):
    """Zero-padded 'same' correlation of the H and W axes with the separable
    window (outer product of the 1D window with itself)."""
    w = window_1d() if w is None else w
    r = len(w) // 2
    a = np.asarray(a, np.float64)
    H, W = a.shape[-3], a.shape[-2]
    pad = [(0, 0)] * a.ndim
    pad[-3] = (r, r)
    pad[-2] = (r, r)
    p = np.pad(a, pad)
    # along W
    t = np.zeros(a.shape[:-3] + (H + 2 * r, W, a.shape[-1]))
    for k in range(len(w)):
        t += w[k] * p[..., :, k:k + W, :]
    out = np.zeros(a.shape)
    for k in range(len(w)):
        out += w[k] * t[..., k:k + H, :, :]
    return out


def ssim_terms(x, y):
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    mx, my = blur(x), blur(y)
    exx, eyy, exy = blur(x * x), blur(y * y), blur(x * y)
    sxx, syy, sxy = exx - mx * mx, eyy - my * my, exy - mx * my
    A1 = 2 * mx * my + C1
    A2 = 2 * sxy + C2
    B1 = mx * mx + my * my + C1
    B2 = sxx + syy + C2
    S = A1 * A2 / (B1 * B2)
    return dict(mx=mx, my=my, A1=A1, A2=A2, B1=B1, B2=B2, S=S)


def ssim(x, y):
    """Mean SSIM over every pixel and channel."""
    return float(ssim_terms(x, y)["S"].mean())


def ssim_grad(x, y):
    """d mean(SSIM) / dx."""
    t = ssim_terms(x, y)
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    n = x.size
    B12 = t["B1"] * t["B2"]
    d_m = 2 * t["my"] * (t["A2"] - t["A1"]) / B12 - 2 * t["mx"] * t["S"] * (1 / t["B1"] - 1 / t["B2"])
    d_xx = -t["S"] / t["B2"]
    d_xy = 2 * t["A1"] / B12
    return (blur(d_m) + 2 * x * blur(d_xx) + y * blur(d_xy)) / n


def loss(x, y, lam=LAMBDA):
    """(1 - lam) mean |x - y| + lam (1 - mean SSIM)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    return float((1 - lam) * np.abs(x - y).mean() + lam * (1.0 - ssim(x, y)))


def loss_grad(x, y, lam=LAMBDA):
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    return (1 - lam) * np.sign(x - y) / x.size - lam * ssim_grad(x, y)
