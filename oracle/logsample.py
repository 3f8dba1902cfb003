"""Reference of the LoG penalty sampling of Eq. 1 -- TEST INFRASTRUCTURE ONLY.

Sec. III-B ("Sampling"): the probability that a pixel spawns a Gaussian is
P_s = max(P_L - P~, 0), P_L the norm of the Laplacian-of-Gaussian (LoG)
response of the input image and P~ that of the image rendered from the
current map (Eq. 1).  The paper leaves the operator's scale, the norm, the
border and the sampling rule open; the readings used here:
  * LoG with sigma = 1 on a 7 x 7 support, written as the sum of two
    separable terms K(dx, dy) = g2(dx) g(dy) + g(dx) g2(dy), with
    g(d) = exp(-d^2 / 2) normalised to sum 1 and g2(d) = (d^2 - 1) g(d)
    shifted to sum 0 (so a constant image responds with 0);
  * the norm is the Euclidean norm of the three channel responses;
  * pixels outside the image repeat the nearest edge pixel;
  * pixel p is sampled iff u(p) < min(1, kappa P_s(p)) for caller-supplied
    uniform numbers u.
"""
from __future__ import annotations

import numpy as np
from scipy.ndimage import correlate

RADIUS = 3


def taps():
    d = np.arange(-RADIUS, RADIUS + 1, dtype=np.float64)
    g = np.exp(-0.5 * d * d)
    g /= g.sum()
    g2 = (d * d - 1.0) * g
    g2 -= g2.mean()
    return g, g2


def kernel2d():
    g, g2 = taps()
    return np.outer(g, g2) + np.outer(g2, g)  # [dy, dx]


def log_norm(img):
    """|LoG| of a [3, H, W] image (FP64)."""
    K = kernel2d()
    r = np.stack([correlate(np.asarray(img[c], np.float64), K, mode="nearest") for c in range(img.shape[0])])
    return np.sqrt((r * r).sum(0))


def penalty(image, rendered):
    return np.maximum(log_norm(image) - log_norm(rendered), 0.0)


def sample(ps, u, kappa):
    """Indices (y W + x, ascending) with u < min(1, kappa P_s), the decision in FP32."""
    p = np.minimum(np.float32(1.0), np.float32(kappa) * np.asarray(ps, np.float32).reshape(-1))
    return np.nonzero(np.asarray(u, np.float32).reshape(-1) < p)[0]


Y00 = 0.28209479177387814


def backproject(idx, depth, image, cam, logit, F):
    """New Gaussians at the sampled pixels (rows [n, F], FP64): centre at the pixel's depth on its ray,
    log-scale log(depth / fx), identity rotation, the given opacity logit, SH DC from the colour."""
    idx = np.asarray(idx, np.int64)
    W = cam.W
    x, y = (idx % W).astype(np.float64), (idx // W).astype(np.float64)
    d = np.asarray(depth, np.float64).reshape(-1)[idx]
    T = np.asarray(cam.Tcw, np.float32).astype(np.float64)
    Xc = np.stack([d * (x - np.float32(cam.cx)) / np.float32(cam.fx), d * (y - np.float32(cam.cy)) / np.float32(cam.fy), d])
    Xw = T[:3, :3].T @ (Xc - T[:3, 3:4])
    out = np.zeros((idx.size, F))
    out[:, 0:3] = Xw.T
    out[:, 3:6] = np.log(d / np.float32(cam.fx))[:, None]
    out[:, 6] = 1.0
    out[:, 10] = logit
    img = np.asarray(image, np.float64).reshape(3, -1)
    out[:, 11:14] = ((img[:, idx] - 0.5) / Y00).T
    return out
