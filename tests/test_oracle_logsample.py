"""Pins of the LoG penalty reference (CPU only)."""
import numpy as np

from oracle import logsample as ls


def test_kernel_is_zero_sum_and_symmetric():
    K = ls.kernel2d()
    assert K.shape == (7, 7) and abs(K.sum()) < 1e-15
    assert np.allclose(K, K.T) and np.allclose(K, K[::-1, ::-1])
    assert K[3, 3] < 0  # a bright dot gives a negative centre response


def test_constant_and_linear_images_give_no_response():
    H, W = 20, 24
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    const = np.full((3, H, W), 0.4)
    ramp = np.stack([0.01 * x + 0.02 * y, 0.03 * x, 0.5 - 0.01 * y])
    assert np.abs(ls.log_norm(const)).max() < 1e-14
    # the Laplacian of a linear function vanishes (away from the replicated border)
    assert np.abs(ls.log_norm(ramp)[3:-3, 3:-3]).max() < 1e-14


def test_quadratic_image_gives_the_continuous_laplacian_up_to_sampling():
    # the LoG of a(x^2 + y^2) is the constant 4a in the continuum; the sampled
    # 7-tap kernel reproduces it to within a few per cent
    H, W = 30, 30
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    a = 1e-3
    img = np.stack([a * ((x - 15) ** 2 + (y - 15) ** 2)] + [np.zeros((H, W))] * 2)
    r = ls.log_norm(img)[4:-4, 4:-4]
    assert np.ptp(r) < 1e-12
    assert abs(r.mean() / (4 * a) - 1.0) < 0.05


def test_penalty_and_sampling_rules():
    rng = np.random.default_rng(0)
    img = rng.uniform(0, 1, (3, 17, 19))
    assert np.abs(ls.penalty(img, img)).max() == 0.0
    assert np.allclose(ls.penalty(img, np.zeros_like(img)), ls.log_norm(img))
    ps = ls.penalty(img, 0.5 * img)
    assert (ps >= 0).all() and ps.max() > 0
    u = rng.uniform(0, 1, ps.size)
    idx = ls.sample(ps, u, 2.0)
    brute = [p for p in range(ps.size) if np.float32(u[p]) < min(np.float32(1), np.float32(2.0) * np.float32(ps.flat[p]))]
    assert list(idx) == brute
