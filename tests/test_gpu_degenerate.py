"""Degenerate Gaussians and image shapes against the oracle at every pixel,
forward and backward, through the product launch (16x16 tiles, half-warp
blends):

* a Gaussian whose 3-sigma rectangle spans more than 1024 tiles, which the
  binning emits whole (every tile of the rectangle) instead of by row spans;
* needle-thin covariances across and along the viewing ray (the 0.3 px^2
  dilation of the 2D covariance keeps them invertible);
* an opacity so small that alpha never reaches 1/255 (never composited) and
  one that saturates at the 0.99 alpha clamp;
* a Gaussian just in front of the near plane, one behind the camera and one
  whose centre projects outside the image while its support reaches in;
* a ragged view (650 x 470: neither side a multiple of the tile), and 1 x 1
  and 17 x 33 views of a random room.

Near-singular 2D covariances are ill-conditioned in FP32 whatever the
kernel: along a needle the three terms of q = A dx^2 + 2 B dx dy + C dy^2
cancel (their absolute sum S reaches 10^4 where q ~ 2), and the determinant
of the covariance cancels by kappa_det = (|a c| + b^2) / (a c - b^2) (4500
for the first needle).  With u = 2^-24, q carries an error of about
6 u S + 3 u q kappa_det (a few roundings of each coefficient, and the
determinant's relative error scaling every coefficient), and a pixel's
colour and transmittance move by at most alpha / 2 per unit of q of each
Gaussian; the image check allows that sum per pixel on top of the usual
1e-5 (for a well-conditioned Gaussian S = q and the extra is below 1e-6).
Their gradients are worse conditioned still (the inverse covariance enters
twice): an FP32 evaluation of the oracle's own formulas deviates from the
FP64 one by 1.5 % on the first needle.  So the needles' gradients are only
required finite, the colour part within its derived bound, and every other
Gaussian's gradient within the usual 1e-4; the same scene without the two
needles is then checked in full, pose included."""
import math

import numpy as np
import pytest

from paper_2511_23030_b300 import dcg, synth

from gpu_util import GRAD_TOL, GROUPS, RGB_TOL, T_TOL, backward, check_image, make_ctx, rel_l2, render

pytestmark = pytest.mark.gpu

W, H = 650, 470
NEEDLES = (1, 2)
U32 = 2.0 ** -24
F0 = 14  # SH degree 0: mean 3, log-scale 3, quaternion 4, opacity logit 1, colour 3


def _g(pos, log_s, quat=(1.0, 0.0, 0.0, 0.0), logit=0.0, rgb=(0.5, 0.5, 0.5)):
    p = np.zeros(F0, np.float32)
    p[0:3], p[3:6], p[6:10], p[10] = pos, log_s, quat, logit
    p[11:14] = (np.asarray(rgb, np.float64) - 0.5) / synth.Y00
    return p


def _scene():
    c15, s15 = math.cos(math.radians(15)), math.sin(math.radians(15))
    L = math.log
    special = [
        _g((0.1, -0.05, 3.0), (L(3.0), L(2.0), L(1.0)), logit=-1.0, rgb=(0.2, 0.4, 0.9)),  # > 1024 tiles: whole
        _g((-0.4, 0.3, 4.0), (L(0.8), L(1e-4), L(1e-4)), (c15, 0.0, 0.0, s15), 2.0, (0.9, 0.1, 0.1)),  # needle across
        _g((0.6, -0.4, 3.5), (L(1e-4), L(1e-4), L(1.5)), logit=2.0, rgb=(0.1, 0.9, 0.2)),  # needle along the ray
        _g((0.0, 0.2, 2.0), (L(0.2), L(0.2), L(0.2)), logit=-12.0, rgb=(1.0, 1.0, 1.0)),  # alpha < 1/255 everywhere
        _g((0.5, 0.2, 2.5), (L(0.05), L(0.08), L(0.05)), logit=12.0, rgb=(0.9, 0.8, 0.1)),  # alpha clamped at 0.99
        _g((0.01, -0.02, 0.202), (L(0.002), L(0.003), L(0.002)), logit=1.0, rgb=(0.3, 0.3, 0.8)),  # just past znear
        _g((0.0, 0.0, -1.0), (L(2.0), L(2.0), L(2.0)), logit=3.0, rgb=(1.0, 0.0, 0.0)),  # behind the camera
        _g((3.6, 0.1, 3.0), (L(0.6), L(0.3), L(0.3)), logit=1.5, rgb=(0.6, 0.2, 0.7)),  # centre off screen
    ]
    rng = np.random.default_rng(42)
    n = 48
    means = np.stack([rng.uniform(-1.5, 1.5, n), rng.uniform(-1.2, 1.2, n), rng.uniform(1.5, 6.0, n)], 1)
    rnd = synth._gaussians(rng, means.astype(np.float32), 0, (0.02, 0.3), dc_rgb=rng.uniform(0, 1, (n, 3)))
    return np.concatenate([np.stack(special), rnd]).astype(np.float32)


def _cam(w, h, f):
    return synth.Camera(f, f, w / 2.0, h / 2.0, w, h, np.eye(4, dtype=np.float32), 0.2, 100.0)


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx(deg=0, n_max=8192, views=1, pixels=W * H)
    yield c
    dcg.dcg_destroy(c)


def _conic_error_bound(pr, cam):
    """Per-pixel bound of the FP32 error of colour and transmittance (first) and of the relative
    depth (second) from the evaluation of the conic form, from the oracle's FP64 projection:
    sum over Gaussians of alpha / 2 (6 u S + 3 u q kappa_det), the depth term scaled by the
    Gaussian's depth over max(1, pixel depth) once the depth is known."""
    ys, xs = np.mgrid[0:cam.H, 0:cam.W]
    xs, ys = xs.ravel().astype(np.float64), ys.ravel().astype(np.float64)
    b_c = np.zeros(xs.size)
    b_z = np.zeros(xs.size)
    for g in np.nonzero(pr["vis"] > 0)[0]:
        a, b, c = pr["a"][g], pr["b2"][g], pr["c"][g]
        kd = (abs(a * c) + b * b) / (a * c - b * b)
        dx, dy = xs - pr["u"][g], ys - pr["v"][g]
        q = pr["A"][g] * dx * dx + 2.0 * pr["B"][g] * dx * dy + pr["C"][g] * dy * dy
        S = abs(pr["A"][g]) * dx * dx + 2.0 * np.abs(pr["B"][g] * dx * dy) + abs(pr["C"][g]) * dy * dy
        al = np.minimum(0.99, pr["o"][g] * np.exp(-0.5 * q))
        al[(q > 9.0) | (al < 1.0 / 255.0)] = 0.0
        e = 0.5 * al * (6.0 * U32 * S + 3.0 * U32 * q * kd)
        b_c += e
        b_z += e * max(1.0, pr["z"][g])
    return b_c, b_z


def _check_bounded(o, rgb, depth, T, bounds, tag):
    b_c, b_z = bounds
    ok = o["flags"] == 0
    assert ok.mean() >= 0.99, tag
    e_rgb = np.abs(rgb - o["rgb"]).max(1)
    e_T = np.abs(T - o["T"])
    e_z = np.abs(depth - o["depth"])
    tol_z = RGB_TOL + b_z / np.maximum(1.0, np.abs(o["depth"]))
    assert (e_rgb[ok] <= RGB_TOL + b_c[ok]).all(), (tag, e_rgb[ok].max())
    assert (e_T[ok] <= T_TOL + b_c[ok]).all(), (tag, e_T[ok].max())
    assert (e_z[ok] / np.maximum(1.0, np.abs(o["depth"][ok])) <= tol_z[ok]).all(), tag


def _full(orc, ctx, P, cam, seed, bounds=None):
    import torch

    n = P.shape[0]
    g_t, _, rgb, depth = render(ctx, P, 0, [cam])
    st = dcg.dcg_state_read(ctx, None, 1, n, cam.W * cam.H)
    o = orc.render(P, 0, cam)
    r = rgb.view(3, -1).T.cpu().numpy().astype(np.float64)
    d = depth.cpu().numpy().astype(np.float64)
    T = st["T"].astype(np.float64)
    if bounds is None:
        check_image(o, r, d, T, f"{cam.W}x{cam.H}", max_flag=0.01)
    else:
        _check_bounded(o, r, d, T, bounds, f"{cam.W}x{cam.H}")
    rng = np.random.default_rng(seed)
    Pn = cam.W * cam.H
    gr = rng.normal(size=(Pn, 3))
    gd = rng.normal(size=Pn) * 0.1
    gr[o["flags"] != 0] = 0
    gd[o["flags"] != 0] = 0
    dr = torch.from_numpy(np.ascontiguousarray(gr.T.reshape(-1)).astype(np.float32)).cuda()
    dd = torch.from_numpy(gd.astype(np.float32)).cuda()
    grad, pose = backward(ctx, g_t, 0, n, dr, dd, 1)
    og, opose = orc.render_bwd(P, 0, cam, gr.astype(np.float32).astype(np.float64),
                               gd.astype(np.float32).astype(np.float64))
    return o, st, grad, og, pose[0], opose


def test_degenerate_gaussians_on_a_ragged_view(ctx, orc):
    P = _scene()
    cam = _cam(W, H, 300.0)
    pr = orc.project(P, 0, cam)
    bounds = _conic_error_bound(pr, cam)
    o, st, grad, og, pose, opose = _full(orc, ctx, P, cam, 3, bounds)
    # the cases are what they claim to be
    rect = st["rect"]
    ntiles = (rect[:, 2] - rect[:, 0] + 1) * (rect[:, 3] - rect[:, 1] + 1)
    assert ntiles[0] > 1024  # emitted whole
    assert rect[6, 2] < rect[6, 0] and pr["vis"][6] == 0  # behind the camera: culled
    assert pr["vis"][5] > 0 and pr["z"][5] < 0.21  # just past the near plane, kept
    assert not (0 <= pr["u"][7] < W) and rect[7, 2] >= rect[7, 0]  # off-screen centre, reaches in
    with np.errstate(invalid="ignore", divide="ignore"):  # the culled Gaussian has no covariance
        kd = (np.abs(pr["a"] * pr["c"]) + pr["b2"] ** 2) / (pr["a"] * pr["c"] - pr["b2"] ** 2)
    assert kd[1] > 1000 and kd[2] > 500  # the needles are near-singular
    assert (o["n"] > 0).mean() > 0.9  # the whole-image Gaussian reaches (almost) every pixel
    assert bounds[0].max() > 1e-4  # ... and the needles make the FP32 bound matter
    # the transparent Gaussian composites nowhere: its gradient is zero on both sides
    assert not og[3].any() and not grad[3].any()
    assert np.isfinite(grad).all() and np.isfinite(pose).all()
    well = np.array([k for k in range(P.shape[0]) if k not in NEEDLES])
    for name, sl in GROUPS.items():
        e = rel_l2(grad[well, sl], og[well, sl])
        assert e <= GRAD_TOL, (name, e)
    for k in (0, 4, 5, 7):
        assert rel_l2(grad[k], og[k]) <= GRAD_TOL, (k, grad[k], og[k])
    # needles: the colour gradient sum_p T alpha g moves with alpha, relatively by at most half the
    # largest q error over the pixels they reach
    ys, xs = np.mgrid[0:H, 0:W]
    for k in NEEDLES:
        dx, dy = xs.ravel() - pr["u"][k], ys.ravel() - pr["v"][k]
        q = pr["A"][k] * dx * dx + 2.0 * pr["B"][k] * dx * dy + pr["C"][k] * dy * dy
        S = abs(pr["A"][k]) * dx * dx + 2.0 * np.abs(pr["B"][k] * dx * dy) + abs(pr["C"][k]) * dy * dy
        reach = q <= 9.0
        dq = (6.0 * U32 * S[reach] + 3.0 * U32 * q[reach] * kd[k]).max()
        assert rel_l2(grad[k, 11:14], og[k, 11:14]) <= 0.5 * dq + GRAD_TOL, (k, grad[k], og[k])


def test_degenerate_gaussians_without_needles(ctx, orc):
    """The same view without the two needles: images at 1e-5, every gradient and the pose at 1e-4."""
    P = _scene()
    P = P[[k for k in range(P.shape[0]) if k not in NEEDLES]]
    cam = _cam(W, H, 300.0)
    o, st, grad, og, pose, opose = _full(orc, ctx, P, cam, 4)
    for name, sl in GROUPS.items():
        e = rel_l2(grad[:, sl], og[:, sl])
        assert e <= GRAD_TOL, (name, e)
    assert rel_l2(pose, opose) <= GRAD_TOL, (pose, opose)


@pytest.mark.parametrize("w,h", [(1, 1), (17, 33)])
def test_tiny_views_match_oracle(ctx, orc, w, h):
    sc = synth.room_small(0)
    P = sc["params"]
    cam = _cam(w, h, 100.0)
    o, _, grad, og, pose, opose = _full(orc, ctx, P, cam, w + h)
    if o["n"].max() > 0:
        for name, sl in GROUPS.items():
            assert rel_l2(grad[:, sl], og[:, sl]) <= GRAD_TOL, name
        assert rel_l2(pose, opose) <= GRAD_TOL


def test_clamped_jacobian_gaussians_match_oracle(orc):
    """Gaussians whose centres project beyond the image extended by 15 % per
    side, so that the perspective Jacobian takes x/z, y/z or both at the limit
    (the clamped branch of the forward and of its gradient), but whose ellipses
    reach into the image: every pixel and every gradient, pose included."""
    P, cam = synth.clamp_scene()
    P = P.astype(np.float32)
    fl = orc.clamp_flags(P, 3, cam)
    assert (fl & 1).sum() >= 4 and (fl & 2).sum() >= 4 and (fl == 3).sum() >= 2
    c = make_ctx(deg=3, n_max=64, views=1, pixels=cam.W * cam.H)
    try:
        import torch

        n = P.shape[0]
        g_t, _, rgb, depth = render(c, P, 3, [cam])
        st = dcg.dcg_state_read(c, None, 1, n, cam.W * cam.H)
        o = orc.render(P, 3, cam)
        check_image(o, rgb.view(3, -1).T.cpu().numpy().astype(np.float64), depth.cpu().numpy().astype(np.float64),
                    st["T"].astype(np.float64), "clamped", max_flag=0.01)
        rng = np.random.default_rng(5)
        Pn = cam.W * cam.H
        gr = rng.normal(size=(Pn, 3))
        gd = rng.normal(size=Pn) * 0.1
        gr[o["flags"] != 0] = 0
        gd[o["flags"] != 0] = 0
        dr = torch.from_numpy(np.ascontiguousarray(gr.T.reshape(-1)).astype(np.float32)).cuda()
        dd = torch.from_numpy(gd.astype(np.float32)).cuda()
        grad, pose = backward(c, g_t, 3, n, dr, dd, 1)
        og, opose = orc.render_bwd(P, 3, cam, gr.astype(np.float32).astype(np.float64),
                                   gd.astype(np.float32).astype(np.float64))
        clamped = np.nonzero(fl)[0]
        assert np.abs(og[clamped]).max(1).min() > 1e-6  # every clamped Gaussian reaches the image
        for name, sl in GROUPS.items():
            assert rel_l2(grad[:, sl], og[:, sl]) <= GRAD_TOL, name
            assert rel_l2(grad[clamped, sl], og[clamped, sl]) <= GRAD_TOL, name
        assert rel_l2(pose[0], opose) <= GRAD_TOL, (pose[0], opose)
    finally:
        dcg.dcg_destroy(c)
