"""FP64 reference of the SSIM term of the image loss -- TEST INFRASTRUCTURE ONLY.

Eq. 3 of the paper: L_image = (1 - lambda_s) |I - I_gt|_1 + lambda_s (1 - SSIM(I, I_gt)).
The paper does not define SSIM further; the reading used here is the one of
the 3DGS method it builds on: an 11 x 11 Gaussian window (sigma 1.5, weights
normalised to sum 1), C1 = 0.01^2, C2 = 0.03^2 (images in [0, 1]), windowed
means taken as a same-size correlation with zero padding outside the image,

    SSIM(p) = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_x^2 + s_y^2 + C2)),
    s_x^2 = w*(x^2) - mu_x^2,  s_xy = w*(x y) - mu_x mu_y,

and SSIM(I, I_gt) the mean of SSIM(p) over the pixels and the three channels.
The gradient is the chain rule written out: SSIM(p) depends on I only through
mu_x = w*x, w*(x^2) and w*(x y), so dL/dx = w*g_mu + 2 x (w*g_xx) + y (w*g_xy)
with the per-pixel partial derivatives g (the window is symmetric, so the
adjoint of the correlation is the same correlation).
"""
from __future__ import annotations

import numpy as np
from scipy.signal import correlate2d

SIGMA, RADIUS = 1.5, 5
C1, C2 = 0.01 ** 2, 0.03 ** 2


def window() -> np.ndarray:
    k = np.arange(-RADIUS, RADIUS + 1, dtype=np.float64)
    g = np.exp(-k * k / (2.0 * SIGMA * SIGMA))
    g /= g.sum()
    return np.outer(g, g)


def _corr(a, w):
    return correlate2d(a, w, mode="same", boundary="fill", fillvalue=0.0)


def ssim_map(x, y):
    """Per-pixel SSIM of two [H, W] images."""
    w = window()
    mx, my = _corr(x, w), _corr(y, w)
    vx = _corr(x * x, w) - mx * mx
    vy = _corr(y * y, w) - my * my
    cxy = _corr(x * y, w) - mx * my
    return ((2 * mx * my + C1) * (2 * cxy + C2)) / ((mx * mx + my * my + C1) * (vx + vy + C2))


def ssim_term(rgb, tgt, lam_s):
    """lam_s (1 - SSIM) for one view ([3, H, W] arrays) and its gradient with respect to rgb."""
    rgb = np.asarray(rgb, np.float64)
    tgt = np.asarray(tgt, np.float64)
    w = window()
    C, H, W = rgb.shape
    coef = -lam_s / (C * H * W)  # d loss / d SSIM(p)
    total = 0.0
    grad = np.zeros_like(rgb)
    for c in range(C):
        x, y = rgb[c], tgt[c]
        mx, my = _corr(x, w), _corr(y, w)
        vx = _corr(x * x, w) - mx * mx
        vy = _corr(y * y, w) - my * my
        cxy = _corr(x * y, w) - mx * my
        A1, A2 = 2 * mx * my + C1, 2 * cxy + C2
        B1, B2 = mx * mx + my * my + C1, vx + vy + C2
        S = A1 * A2 / (B1 * B2)
        total += S.sum()
        g_mu = coef * S * (2 * my / A1 - 2 * my / A2 - 2 * mx / B1 + 2 * mx / B2)
        g_xx = coef * S * (-1.0 / B2)
        g_xy = coef * S * (2.0 / A2)
        grad[c] = _corr(g_mu, w) + 2 * x * _corr(g_xx, w) + y * _corr(g_xy, w)
    return lam_s * (1.0 - total / (C * H * W)), grad
