"""Pins of the FP64 prefetch-MLP reference: central finite differences of its
analytic gradient, GELU and BCE against independent library forms, the
SE(3) logarithm against its exponential, and Adam's first step."""
import math

import numpy as np
import pytest

from paper_2511_23030_b300 import synth


def test_gelu_and_bce_against_library_forms():
    from scipy.special import log_expit, ndtr

    from oracle import mlp

    x = np.linspace(-6, 6, 101)
    assert np.allclose(mlp.gelu(x), x * ndtr(x), atol=1e-14)  # x Phi(x)
    h = 1e-6
    assert np.allclose(mlp.gelu_grad(x), (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h), atol=1e-8)
    assert mlp.gelu_grad(np.array([0.0]))[0] == 0.5
    # BCE with logits equals -y log sigma(z) - (1-y) log(1 - sigma(z))
    z = np.array([-30.0, -2.0, 0.0, 1.5, 40.0])
    for y in (0.0, 1.0):
        ours = np.maximum(z, 0) - z * y + np.log1p(np.exp(-np.abs(z)))
        ref = -(y * log_expit(z) + (1 - y) * log_expit(-z))
        assert np.allclose(ours, ref, atol=1e-12)


def test_mlp_gradient_finite_differences():
    from oracle import mlp

    rng = np.random.default_rng(0)
    P = synth.mlp_init_params(1).astype(np.float64)
    P += rng.normal(0, 0.01, P.shape)  # non-zero biases too
    x = rng.normal(0, 1, (8, mlp.N_IN))
    y = (rng.uniform(size=8) < 0.5).astype(np.float64)
    L, g = mlp.loss_and_grads(P, x, y, bf16_storage=False)
    idx = np.concatenate([rng.choice(mlp.N_PARAMS, 40, replace=False), [mlp.N_PARAMS - 1, mlp.N_PARAMS - 2]])
    for i in idx:
        h = 1e-6
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (mlp.loss_and_grads(Pp, x, y, False)[0] - mlp.loss_and_grads(Pm, x, y, False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_bf16_rounding():
    from oracle import mlp

    # 1 + 2^-8 is exactly halfway between bf16 neighbours 1 and 1 + 2^-7: ties to even -> 1
    assert mlp.bf16(np.array([1.0 + 2 ** -8]))[0] == 1.0
    assert mlp.bf16(np.array([1.0 + 3 * 2 ** -9]))[0] == 1.0 + 2 ** -7
    assert mlp.bf16(np.array([-2.5]))[0] == -2.5


def test_se3_log_inverts_exponential():
    from scipy.linalg import expm

    from oracle import mlp

    rng = np.random.default_rng(3)
    for _ in range(20):
        xi = np.concatenate([rng.normal(0, 2, 3), rng.normal(0, 0.5, 3)])
        X = np.zeros((4, 4))
        w = xi[3:]
        X[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
        X[:3, 3] = xi[:3]
        assert np.allclose(mlp.se3_log(expm(X)), xi, atol=1e-9)


def test_adam_first_step_moves_by_lr():
    from oracle import mlp

    p = np.zeros(5)
    g = np.array([1.0, -2.0, 0.5, 1e-3, -1e3])
    p1, m1, m2 = mlp.adam_step(p, g, np.zeros(5), np.zeros(5), 1, 1e-2)
    # bias-corrected first step is lr * sign(g) (up to eps)
    assert np.allclose(p1, -1e-2 * np.sign(g), rtol=1e-4)
