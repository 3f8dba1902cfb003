"""FP64 reference of the optimizer step over the active set -- TEST INFRASTRUCTURE ONLY.

The paper optimises the Gaussian parameters of the chunks in VRAM against the
loss of Eq. 2-4 (Sec. III-E "Optimization") and keeps optimizer state per
Gaussian (after a loop closure, Sec. III-F clears that state, and lowers the
opacity, where separately built parts of the map meet).  The optimizer is Adam (Kingma & Ba,
"Adam: A Method for Stochastic Optimization", Algorithm 1) with its bias
correction written in the equivalent form

    m <- b1 m + (1 - b1) g
    v <- b2 v + (1 - b2) g^2
    p <- p - (lr / (1 - b1^t)) * m / (sqrt(v) / sqrt(1 - b2^t) + eps)

with one learning rate per parameter component (row of the planar layout).
"""
from __future__ import annotations

import numpy as np


def adam_step(p, g, m, v, lr, beta1, beta2, eps, t):
    """One step on planar [F, n] arrays (FP64); lr has F entries; t >= 1.
    Returns new (p, m, v)."""
    p = np.asarray(p, np.float64)
    g = np.asarray(g, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    bc1 = 1.0 - beta1 ** t
    bc2 = 1.0 - beta2 ** t
    step = (np.asarray(lr, np.float64) / bc1).reshape(-1, 1)
    p = p - step * m / (np.sqrt(v) / np.sqrt(bc2) + eps)
    return p, m, v
