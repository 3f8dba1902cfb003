"""Pins of the FP64 SSIM reference (CPU only)."""
import numpy as np

from oracle import ssim


def test_window_is_a_normalised_separable_gaussian():
    w = ssim.window()
    assert w.shape == (11, 11) and abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(w, w.T) and np.allclose(w, w[::-1, ::-1])
    # ratio of neighbouring taps of exp(-k^2 / (2 sigma^2))
    assert np.isclose(w[5, 6] / w[5, 5], np.exp(-1 / (2 * 1.5 ** 2)))


def test_identical_images_give_zero_loss_and_gradient():
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, (3, 23, 31))
    L, g = ssim.ssim_term(x, x, 0.2)
    assert abs(L) < 1e-14 and np.abs(g).max() < 1e-13


def test_constant_images_interior_closed_form():
    # away from the zero-padded border every window sees the constants a and b:
    # the variances vanish and SSIM = (2ab + C1) / (a^2 + b^2 + C1)
    a, b = 0.3, 0.7
    S = ssim.ssim_map(np.full((30, 30), a), np.full((30, 30), b))
    want = (2 * a * b + ssim.C1) / (a * a + b * b + ssim.C1)
    assert np.allclose(S[5:-5, 5:-5], want, rtol=1e-13)
    assert not np.allclose(S[0, 0], want)  # the border sees the zero padding


def test_symmetry_and_bounds():
    rng = np.random.default_rng(1)
    x, y = rng.uniform(0, 1, (2, 19, 17))
    S1, S2 = ssim.ssim_map(x, y), ssim.ssim_map(y, x)
    assert np.allclose(S1, S2, rtol=1e-14)
    assert (S1 <= 1 + 1e-12).all() and (S1 >= -1 - 1e-12).all()


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    x = rng.uniform(0.1, 0.9, (3, 14, 13))
    y = rng.uniform(0.1, 0.9, (3, 14, 13))
    _, g = ssim.ssim_term(x, y, 0.3)
    h = 1e-6
    for (c, i, j) in [(0, 0, 0), (1, 7, 6), (2, 13, 12), (0, 3, 11), (2, 10, 1)]:
        xp, xm = x.copy(), x.copy()
        xp[c, i, j] += h
        xm[c, i, j] -= h
        fd = (ssim.ssim_term(xp, y, 0.3)[0] - ssim.ssim_term(xm, y, 0.3)[0]) / (2 * h)
        assert abs(fd - g[c, i, j]) <= 1e-7 * max(1.0, abs(fd)) + 1e-9, (c, i, j, fd, g[c, i, j])
