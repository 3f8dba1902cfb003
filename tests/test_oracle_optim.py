"""Pins of the FP64 Adam reference (CPU only)."""
import numpy as np
import pytest

from oracle import optim


def test_constant_gradient_moves_by_lr_each_step():
    # with a constant gradient the bias-corrected moments are exactly g and g^2,
    # so every step moves a parameter by lr g / (|g| + eps)
    rng = np.random.default_rng(0)
    F, n = 5, 7
    p0 = rng.normal(size=(F, n))
    g = rng.normal(size=(F, n))
    lr = rng.uniform(1e-4, 1e-2, F)
    eps = 1e-8
    p, m, v = p0, np.zeros_like(p0), np.zeros_like(p0)
    for t in range(1, 6):
        p, m, v = optim.adam_step(p, g, m, v, lr, 0.9, 0.999, eps, t)
        want = p0 - t * lr[:, None] * g / (np.abs(g) + eps)
        assert np.allclose(p, want, rtol=0, atol=1e-12)
    assert np.allclose(m, g * (1 - 0.9 ** 5), rtol=1e-13)
    assert np.allclose(v, g * g * (1 - 0.999 ** 5), rtol=1e-12)


def test_zero_gradient_only_decays_the_moments():
    rng = np.random.default_rng(1)
    p0 = rng.normal(size=(3, 4))
    m0 = rng.normal(size=(3, 4))
    v0 = rng.uniform(0.1, 1.0, size=(3, 4))
    p, m, v = optim.adam_step(p0, np.zeros_like(p0), m0, v0, [1e-3] * 3, 0.9, 0.99, 1e-8, 3)
    assert np.allclose(m, 0.9 * m0) and np.allclose(v, 0.99 * v0)
    # the step still uses the decayed moments
    bc1, bc2 = 1 - 0.9 ** 3, 1 - 0.99 ** 3
    assert np.allclose(p, p0 - 1e-3 / bc1 * (0.9 * m0) / (np.sqrt(0.99 * v0) / np.sqrt(bc2) + 1e-8))


def test_matches_an_independent_library_adam():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    F, n = 4, 9
    p0 = rng.normal(size=(F, n))
    lr = [1e-3, 5e-3, 2e-2, 1e-4]
    rows = [torch.tensor(p0[c].copy(), dtype=torch.float64, requires_grad=True) for c in range(F)]
    opt = torch.optim.Adam([{"params": [rows[c]], "lr": lr[c]} for c in range(F)], betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0, np.zeros_like(p0), np.zeros_like(p0)
    for t in range(1, 8):
        g = rng.normal(size=(F, n))
        for c in range(F):
            rows[c].grad = torch.tensor(g[c], dtype=torch.float64)
        opt.step()
        p, m, v = optim.adam_step(p, g, m, v, lr, 0.9, 0.999, 1e-8, t)
        got = np.stack([r.detach().numpy() for r in rows])
        assert np.allclose(p, got, rtol=1e-12, atol=1e-14), t
