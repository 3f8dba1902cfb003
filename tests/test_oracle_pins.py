"""Pins of the FP64 oracle to things other than itself: hand-worked ids of
Eq. 5/6, point-sampled frustum membership, textbook/scipy spherical
harmonics, closed-form single- and two-Gaussian pixels, back-to-front
compositing, and central finite differences of the oracle's own forward."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2511_23030_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ Eq. 5 / 6
def test_chunk_ids_golden(orc):
    n = 0
    for line in open(os.path.join(GOLDEN, "chunk_ids.txt")):
        if line.startswith("#") or not line.strip():
            continue
        a, c, i = line.split("|")
        s, px, py, pz = map(float, a.split())
        coords, keys, bad = orc.chunk_keys(np.array([[px, py, pz]], np.float32), s)
        assert bad[0] == 0
        assert list(coords[0]) == list(map(int, c.split()))
        assert int(keys[0]) == int(i)
        assert orc.decode_key(int(keys[0])) == tuple(map(int, c.split()))
        n += 1
    assert n == 7


def test_chunk_coord_interval_property(orc):
    """Exact rational check: chunk c of p satisfies c*s - s/2 <= p < c*s + s/2,
    unless p is within float32 rounding of a boundary."""
    rng = np.random.default_rng(1)
    for s in (4.0, 8.0, 10.0, 0.37):
        p = rng.uniform(-5000, 5000, (4000, 3)).astype(np.float32)
        # plant exact boundaries
        p[:200, 0] = (rng.integers(-100, 100, 200) * s + s / 2).astype(np.float32)
        coords, keys, bad = orc.chunk_keys(p, s)
        assert not bad.any()
        S = Fraction(float(np.float32(s)))
        for k in range(0, 4000, 7):
            for a in range(3):
                P = Fraction(float(p[k, a]))
                c = int(coords[k, a])
                lo, hi = c * S - S / 2, c * S + S / 2
                ulp = Fraction(float(np.spacing(np.float32(abs(p[k, a]) + s))))
                assert lo - 2 * ulp <= P < hi + 2 * ulp


def test_chunk_key_range_and_nan(orc):
    p = np.array([[1048576.0, 0, 0], [-1048577.0, 0, 0], [np.nan, 0, 0], [0, np.inf, 0], [3.0, 3.0, 3.0]], np.float32)
    _, keys, bad = orc.chunk_keys(p, 1.0)
    assert list(bad) == [1, 1, 1, 1, 0]


def test_chunk_key_order_is_lexicographic(orc):
    rng = np.random.default_rng(2)
    p = rng.uniform(-1e5, 1e5, (5000, 3)).astype(np.float32)
    coords, keys, _ = orc.chunk_keys(p, 8.0)
    a = np.lexsort((coords[:, 2], coords[:, 1], coords[:, 0]))
    b = np.argsort(keys, kind="stable")
    assert (coords[a] == coords[b]).all()


# ------------------------------------------------------------------ cull
def _rand_cam(rng, W=320, H=240):
    eye = rng.uniform(-20, 20, 3)
    T = synth.look_at(eye, eye + rng.normal(0, 1, 3), up=(0, 0, 1))
    f = rng.uniform(0.4, 1.2) * W
    return synth.Camera(f, f * rng.uniform(0.9, 1.1), W * rng.uniform(0.4, 0.6), H * rng.uniform(0.4, 0.6),
                        W, H, T, 0.2, float(rng.uniform(20, 60)))


def _inside(cam, X):
    T = np.asarray(cam.Tcw, np.float64)
    t = X @ T[:3, :3].T + T[:3, 3]
    Z = t[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        u = cam.fx * t[:, 0] / Z + cam.cx
        v = cam.fy * t[:, 1] / Z + cam.cy
    return (Z >= cam.znear) & (Z <= cam.zfar) & (u >= 0) & (u <= cam.W) & (v >= 0) & (v <= cam.H)


def test_frustum_planes_classify_points(orc):
    """Planes from the view-projection matrix agree with direct projection of points."""
    rng = np.random.default_rng(3)
    for _ in range(10):
        cam = _rand_cam(rng)
        planes, C = orc.frustum_planes(cam)
        T = np.asarray(cam.Tcw, np.float64)
        assert np.allclose(C, -T[:3, :3].T @ T[:3, 3], atol=1e-5)
        X = C + rng.normal(0, 1, (20000, 3)) * rng.uniform(1, 40, (20000, 1))
        val = X @ planes[:, :3].T + planes[:, 3]
        inside_planes = (val >= 0).all(1)
        direct = _inside(cam, X)
        scale = np.linalg.norm(planes[:, :3], axis=1)
        margin = (np.abs(val) / scale).min(1) > 1e-6
        assert (inside_planes[margin] == direct[margin]).all()
        assert direct.sum() > 0


def test_cull_conservative_vs_point_samples(orc):
    rng = np.random.default_rng(4)
    s = 4.0
    coords = np.array(np.meshgrid(*[np.arange(-8, 8)] * 3, indexing="ij")).reshape(3, -1).T.astype(np.int32)
    for _ in range(6):
        cam = _rand_cam(rng)
        cam.Tcw = synth.look_at(rng.uniform(-10, 10, 3), rng.uniform(-5, 5, 3))
        dfar = 35.0
        mask = orc.cull(coords, s, cam, dfar)
        T = np.asarray(cam.Tcw, np.float64)
        C = -T[:3, :3].T @ T[:3, 3]
        # any sample point of a chunk inside the frustum and within dfar => the chunk is kept
        for k in rng.choice(len(coords), 600, replace=False):
            X = coords[k] * s + rng.uniform(-s / 2, s / 2, (64, 3))
            ok = _inside(cam, X) & (np.linalg.norm(X - C, axis=1) <= dfar)
            if ok.any():
                assert mask[k] == 1
        # a chunk whose 8 corners are all outside one plane is dropped
        planes, _ = orc.frustum_planes(cam)
        corners = np.array([[i, j, l] for i in (-1, 1) for j in (-1, 1) for l in (-1, 1)]) * s / 2
        for k in range(len(coords)):
            X = coords[k] * s + corners
            val = X @ planes[:, :3].T + planes[:, 3]
            if ((val < -1e-9).all(0)).any():
                assert mask[k] == 0


def test_cull_hierarchical_equals_flat(orc):
    rng = np.random.default_rng(5)
    for trial in range(12):
        n = int(rng.integers(1, 3000))
        coords = rng.integers(-60, 60, (n, 3)).astype(np.int32)
        coords = np.unique(coords, axis=0)
        cam = _rand_cam(rng)
        s = float(rng.choice([4.0, 8.0, 10.0]))
        dfar = float(rng.uniform(10, 200))
        a = orc.cull(coords, s, cam, dfar, hierarchical=False)
        b = orc.cull(coords, s, cam, dfar, hierarchical=True)
        assert (a == b).all()


def test_cull_distance_filter(orc):
    cam = synth.Camera(100, 100, 64, 48, 128, 96, np.eye(4, dtype=np.float32), 0.2, 1000.0)
    coords = np.array([[0, 0, z] for z in range(1, 40)], np.int32)
    mask = orc.cull(coords, 1.0, cam, 10.0)
    # chunk (0,0,z) spans z in [z-0.5, z+0.5): nearest point at distance z - 0.5
    assert list(np.nonzero(mask)[0] + 1) == list(range(1, 11))


# ------------------------------------------------------------------ LRU (Sec. III-E)
def test_lru_minimal_oldest_first(orc):
    rng = np.random.default_rng(6)
    for _ in range(200):
        n = int(rng.integers(1, 12))
        resident = rng.uniform(size=n) < 0.8
        visible = rng.uniform(size=n) < 0.3
        last = rng.integers(0, 5, n)
        keys = rng.permutation(n)
        counts = rng.integers(1, 10, n)
        deficit = int(rng.integers(0, 40))
        sel = orc.lru_select(resident, visible, last, keys, counts, deficit)
        evictable = [k for k in range(n) if resident[k] and not visible[k]]
        if sel is None:
            assert sum(counts[k] for k in evictable) < deficit
            continue
        assert set(sel) <= set(evictable)
        assert sum(counts[k] for k in sel) >= deficit
        # minimality: dropping the most recently used chosen chunk no longer covers the deficit
        if sel:
            assert sum(counts[k] for k in sel[:-1]) < deficit
        # oldest first: no unchosen evictable chunk is older than a chosen one
        rest = [k for k in evictable if k not in sel]
        for k in rest:
            for j in sel:
                assert (last[k], keys[k]) > (last[j], keys[j])


def test_gather_order(orc):
    keys = np.array([50, 10, 30, 20], np.uint64)
    counts = np.array([5, 2, 7, 1])
    vis = np.array([1, 1, 0, 1], bool)
    order, n = orc.gather_order(keys, counts, vis)
    assert order == [(1, 0), (3, 2), (0, 3)] and n == 8


# ------------------------------------------------------------------ spherical harmonics
def _dirs(rng, n):
    d = rng.normal(size=(n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def test_sh_matches_scipy_complex_harmonics(orc):
    """Real SH with Condon-Shortley phase: Y_lm = sqrt2 Re Y_l^m (m>0),
    sqrt2 Im Y_l^|m| (m<0), Y_l^0 (m=0), from scipy's complex harmonics."""
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(7)
    d = _dirs(rng, 300)
    Y = orc.sh_basis(3, d)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    for l in range(4):
        for m in range(-l, l + 1):
            am = abs(m)
            if hasattr(sp, "sph_harm_y"):
                Yc = sp.sph_harm_y(l, am, theta, phi)
            else:  # older scipy: sph_harm(m, l, azimuth, polar)
                Yc = sp.sph_harm(am, l, phi, theta)
            ref = Yc.real if m == 0 else (math.sqrt(2) * (Yc.real if m > 0 else Yc.imag))
            assert np.allclose(Y[:, l * l + l + m], ref, atol=1e-12), (l, m)


def test_sh_textbook_low_orders(orc):
    rng = np.random.default_rng(8)
    d = _dirs(rng, 50)
    Y = orc.sh_basis(2, d)
    x, y, z = d.T
    c0 = 0.5 / math.sqrt(math.pi)
    c1 = math.sqrt(3 / (4 * math.pi))
    assert np.allclose(Y[:, 0], c0)
    assert np.allclose(Y[:, 1], -c1 * y) and np.allclose(Y[:, 2], c1 * z) and np.allclose(Y[:, 3], -c1 * x)
    assert np.allclose(Y[:, 4], 0.5 * math.sqrt(15 / math.pi) * x * y)
    assert np.allclose(Y[:, 6], 0.25 * math.sqrt(5 / math.pi) * (3 * z * z - 1))


def test_sh_orthonormal_quadrature(orc):
    nt, npf = 40, 80
    xg, wg = np.polynomial.legendre.leggauss(nt)
    phi = (np.arange(npf) + 0.5) * 2 * math.pi / npf
    ct, ph = np.meshgrid(xg, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    d = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    w = (np.repeat(wg, npf) * 2 * math.pi / npf)
    Y = orc.sh_basis(3, d)
    G = (Y * w[:, None]).T @ Y
    assert np.allclose(G, np.eye(16), atol=1e-12)


# ------------------------------------------------------------------ projection / rendering
def _one(mean, log_s, quat, logit, rgb, deg=0):
    F = synth.n_fields(deg)
    p = np.zeros((1, F), np.float64)
    p[0, 0:3] = mean
    p[0, 3:6] = log_s
    p[0, 6:10] = quat
    p[0, 10] = logit
    p[0, 11:14] = (np.asarray(rgb) - 0.5) / synth.Y00
    return p


def _cam_id(W=64, H=48, f=50.0):
    return synth.Camera(f, f, W / 2.0, H / 2.0, W, H, np.eye(4, dtype=np.float32), 0.2, 100.0)


def test_single_gaussian_closed_form(orc):
    """Isotropic Gaussian on the optical axis: Sigma' = diag(f^2 s^2/z^2 + 0.3) and
    pixel = c * min(0.99, o exp(-q/2)) where the support and cut-off tests pass."""
    cam = _cam_id()
    z, sig, o_logit = 3.0, 0.08, 0.7
    rgb = np.array([0.9, 0.4, 0.2])
    p = _one([0, 0, z], [math.log(sig)] * 3, [1, 0, 0, 0], o_logit, rgb)
    out = orc.render(p, 0, cam)
    var = (cam.fx * sig / z) ** 2 + 0.3
    o = 1 / (1 + math.exp(-o_logit))
    pix = out["pix"].astype(np.float64)
    q = ((pix[:, 0] - cam.cx) ** 2 + (pix[:, 1] - cam.cy) ** 2) / var
    a = np.minimum(0.99, o * np.exp(-0.5 * q))
    keep = (q <= 9) & (a >= 1 / 255)
    exp_rgb = np.where(keep[:, None], a[:, None] * rgb[None], 0)
    assert np.allclose(out["rgb"], exp_rgb, atol=1e-14)
    assert np.allclose(out["depth"], np.where(keep, a * z, 0), atol=1e-13)
    assert keep.sum() > 50
    proj = orc.project(p, 0, cam)
    assert math.isclose(proj["a"][0], var, rel_tol=1e-13) and abs(proj["b2"][0]) < 1e-15


def test_two_gaussians_over_operator(orc):
    cam = _cam_id()
    c1, c2 = np.array([1.0, 0.1, 0.2]), np.array([0.1, 0.8, 0.3])
    p = np.concatenate([_one([0, 0, 4.0], [math.log(0.2)] * 3, [1, 0, 0, 0], 0.3, c2),
                        _one([0, 0, 2.0], [math.log(0.1)] * 3, [1, 0, 0, 0], -0.2, c1)])
    out = orc.render(p, 0, cam, pix=np.array([[32, 24]], np.int32))
    a1 = 1 / (1 + math.exp(0.2))
    a2 = 1 / (1 + math.exp(-0.3))
    assert np.allclose(out["rgb"][0], c1 * a1 + (1 - a1) * a2 * c2, atol=1e-14)
    assert math.isclose(out["depth"][0], 2.0 * a1 + (1 - a1) * a2 * 4.0, rel_tol=1e-13)
    assert math.isclose(out["T"][0], (1 - a1) * (1 - a2), rel_tol=1e-13)


def _tiny_scene(seed, n=48, deg=3, W=32, H=32):
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(2, 4, n)], 1)
    P = np.zeros((n, synth.n_fields(deg)))
    P[:, 0:3] = means
    P[:, 3:6] = rng.uniform(math.log(0.05), math.log(0.3), (n, 3))
    P[:, 6:10] = synth.random_quats(rng, n)
    P[:, 10] = rng.normal(0, 1.5, n)
    P[:, 11:] = rng.normal(0, 0.3, (n, P.shape[1] - 11))
    T = synth.look_at([0.3, -0.2, -0.5], [0.0, 0.1, 3.0], up=(0, -1, 0))
    cam = synth.Camera(28.0, 30.0, 15.5, 16.5, W, H, T, 0.2, 50.0)
    return P, cam


def test_back_to_front_painter_equals_oracle(orc):
    """Brute force on tiny inputs: composite back to front (painter's
    algorithm, C <- a c + (1-a) C from the farthest Gaussian forward) over the
    same per-pixel candidate set; equals the front-to-back oracle wherever the
    1e-4 termination does not trigger."""
    P, cam = _tiny_scene(9)
    proj = orc.project(P, 3, cam)
    out = orc.render(P, 3, cam)
    vis = np.nonzero(proj["vis"] > 0)[0]
    z32 = orc.depth_f32(P[:, :3].astype(np.float32), cam)
    order = vis[np.lexsort((vis, z32[vis]))]
    n_checked = 0
    for k, (x, y) in enumerate(out["pix"]):
        dx = x - proj["u"][order]
        dy = y - proj["v"][order]
        q = proj["A"][order] * dx * dx + 2 * proj["B"][order] * dx * dy + proj["C"][order] * dy * dy
        a = np.minimum(0.99, proj["o"][order] * np.exp(-0.5 * q))
        keep = (q <= 9) & (a >= 1 / 255)
        if np.prod(1 - a[keep]) < 2e-4:
            continue
        C = np.zeros(3)
        D = 0.0
        for j in order[keep][::-1]:
            al = a[keep][list(order[keep]).index(j)]
            C = al * np.array([proj["r"][j], proj["g"][j], proj["b"][j]]) + (1 - al) * C
            D = al * proj["z"][j] + (1 - al) * D
        assert np.allclose(out["rgb"][k], C, atol=1e-13)
        assert math.isclose(out["depth"][k], D, rel_tol=1e-12, abs_tol=1e-13)
        n_checked += 1
    assert n_checked > 500


def test_transmittance_monotone_and_bounded(orc):
    P, cam = _tiny_scene(10, n=200)
    P[:, 10] += 3.0  # opaque enough to terminate
    out = orc.render(P, 3, cam)
    assert (out["T"] >= 1e-4).all() and (out["T"] <= 1).all()
    # more contributors never increases transmittance: T <= 0.99^0 and T < 1 when n > 0
    assert (out["T"][out["n"] > 0] < 1).all() and (out["T"][out["n"] == 0] == 1).all()
    assert (out["n"] > 0).sum() > 100


def test_finite_differences_of_oracle(orc):
    """Central differences of the oracle's own FP64 forward (h = 1e-6 relative)
    against its analytic gradient, for every parameter kind and the pose twist."""
    from scipy.linalg import expm

    P, cam = _tiny_scene(11, n=24)
    rng = np.random.default_rng(12)
    pix = orc.all_pixels(cam.W, cam.H)
    gr = rng.normal(size=(len(pix), 3))
    gd = rng.normal(size=len(pix)) * 0.1

    def loss(Pv, T=None):
        c = cam if T is None else synth.Camera(cam.fx, cam.fy, cam.cx, cam.cy, cam.W, cam.H, T, cam.znear, cam.zfar)
        out = orc.render(Pv, 3, c, pix=pix)
        return float((out["rgb"] * gr).sum() + (out["depth"] * gd).sum())

    grad, gpose = orc.render_bwd(P, 3, cam, gr, gd, pix=pix)
    cols = list(range(0, 11)) + [11, 12, 13, 14, 20, 30, 40, 50, 58]
    checked = 0
    for i in range(P.shape[0]):
        if np.abs(grad[i]).max() < 1e-6:
            continue
        for c in cols:
            h = 1e-6 * max(1.0, abs(P[i, c]))
            Pp, Pm = P.copy(), P.copy()
            Pp[i, c] += h
            Pm[i, c] -= h
            fd = (loss(Pp) - loss(Pm)) / (2 * h)
            assert abs(fd - grad[i, c]) <= 1e-6 * max(1.0, abs(grad[i, c])) + 1e-7, (i, c, fd, grad[i, c])
            checked += 1
        if checked > 150:
            break
    assert checked > 100
    # pose: Tcw <- exp(xi^) Tcw, xi = (v, w)
    T0 = np.asarray(cam.Tcw, np.float64)
    for k in range(6):
        xi = np.zeros(6)
        h = 1e-6
        mats = []
        for sgn in (1, -1):
            xi[:] = 0
            xi[k] = sgn * h
            Xh = np.zeros((4, 4))
            w = xi[3:]
            Xh[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
            Xh[:3, 3] = xi[:3]
            mats.append(expm(Xh) @ T0)
        # the camera takes float32 poses; evaluate the FD with double poses through the oracle directly
        fd = (_loss_T(orc, P, cam, mats[0], pix, gr, gd) - _loss_T(orc, P, cam, mats[1], pix, gr, gd)) / (2 * h)
        assert abs(fd - gpose[k]) <= 1e-6 * max(1.0, abs(gpose[k])), (k, fd, gpose[k])


def test_finite_differences_in_the_clamped_jacobian_branch(orc):
    """The perspective Jacobian evaluated at x/z and y/z clamped to the image
    extended by 15 % per side (the 3DGS lineage's frustum clamp): central
    differences of the oracle's forward against its analytic gradient on
    Gaussians that take that branch, for every parameter kind and the pose."""
    from scipy.linalg import expm

    P, cam = synth.clamp_scene()
    fl = orc.clamp_flags(P, 3, cam)
    pix = orc.all_pixels(cam.W, cam.H)
    out = orc.render(P, 3, cam, pix=pix)
    rng = np.random.default_rng(22)
    gr = rng.normal(size=(len(pix), 3))
    gd = rng.normal(size=len(pix)) * 0.1
    grad, gpose = orc.render_bwd(P, 3, cam, gr, gd, pix=pix)
    reach = np.abs(grad).max(1) > 1e-6  # composited somewhere in the image
    clamped = np.nonzero((fl != 0) & reach)[0]
    # every side of the clamp is exercised, by Gaussians that reach the image
    assert len(clamped) >= 8 and ((fl[clamped] & 1) != 0).sum() >= 4 and ((fl[clamped] & 2) != 0).sum() >= 4
    assert (fl[clamped] == 3).sum() >= 2
    assert not fl[10:].any() and (out["n"] > 0).mean() > 0.5

    def loss(Pv):
        o = orc.render(Pv, 3, cam, pix=pix)
        return float((o["rgb"] * gr).sum() + (o["depth"] * gd).sum())

    cols = list(range(0, 11)) + [11, 12, 13, 14, 20, 30, 40, 50, 58]
    for i in clamped:
        for c in cols:
            h = 1e-6 * max(1.0, abs(P[i, c]))
            Pp, Pm = P.copy(), P.copy()
            Pp[i, c] += h
            Pm[i, c] -= h
            fd = (loss(Pp) - loss(Pm)) / (2 * h)
            assert abs(fd - grad[i, c]) <= 1e-6 * max(1.0, abs(grad[i, c])) + 1e-7, (i, c, fd, grad[i, c])
    # the pose twist, with the clamped Gaussians carrying most of the image
    T0 = np.asarray(cam.Tcw, np.float64)
    for k in range(6):
        mats = []
        for sgn in (1, -1):
            xi = np.zeros(6)
            xi[k] = sgn * 1e-6
            Xh = np.zeros((4, 4))
            w = xi[3:]
            Xh[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
            Xh[:3, 3] = xi[:3]
            mats.append(expm(Xh) @ T0)
        fd = (_loss_T(orc, P, cam, mats[0], pix, gr, gd) - _loss_T(orc, P, cam, mats[1], pix, gr, gd)) / 2e-6
        assert abs(fd - gpose[k]) <= 1e-6 * max(1.0, abs(gpose[k])), (k, fd, gpose[k])
    # the clamp matters here: without it the same Gaussians would have other covariances
    pr = orc.project(P, 3, cam)
    assert np.isfinite(pr["A"][clamped]).all()


def test_clamped_covariance_closed_form(orc):
    """For an isotropic Gaussian (variance s^2) and an identity pose, the dilated
    2D covariance is s^2 J J^T + 0.3 I with the perspective Jacobian
    J = [[f/z, 0, -f x'/z^2], [0, f/z, -f y'/z^2]], where x' / z and y' / z are the
    centre's x / z and y / z limited to the image extended by 15 % of its size
    on each side: a = s^2 f^2 (1/z^2 + x'^2/z^4) + 0.3, b = s^2 f^2 x' y' / z^4,
    c = s^2 f^2 (1/z^2 + y'^2/z^4) + 0.3 (written out in scalars here; the oracle
    forms J W Sigma W^T J^T as matrix products)."""
    W, H, f = 48, 40, 30.0
    cam = synth.Camera(f, f, 23.5, 19.5, W, H, np.eye(4, dtype=np.float32), 0.2, 50.0)
    xlo, xhi = (-0.15 * W - 23.5) / f, (1.15 * W - 23.5) / f
    ylo, yhi = (-0.15 * H - 19.5) / f, (1.15 * H - 19.5) / f
    cases = [(1.30, 0.05), (-1.25, 0.10), (0.10, 1.05), (-0.20, -0.98), (1.20, 1.00), (-1.15, -0.95), (0.3, -0.2)]
    P = np.zeros((len(cases), synth.n_fields(0)))
    z, s = 3.0, 0.5
    for i, (rx, ry) in enumerate(cases):
        P[i, 0:3] = (rx * z, ry * z, z)
    P[:, 3:6] = math.log(s)
    P[:, 6] = 1.0
    pr = orc.project(P, 0, cam)
    fl = orc.clamp_flags(P, 0, cam)
    assert list(fl) == [1, 1, 2, 2, 3, 3, 0]
    for i, (rx, ry) in enumerate(cases):
        xc = min(max(rx, xlo), xhi) * z
        yc = min(max(ry, ylo), yhi) * z
        a = s * s * f * f * (1 / z ** 2 + xc * xc / z ** 4) + 0.3
        b = s * s * f * f * xc * yc / z ** 4
        c = s * s * f * f * (1 / z ** 2 + yc * yc / z ** 4) + 0.3
        assert math.isclose(pr["a"][i], a, rel_tol=1e-13)
        assert math.isclose(pr["b2"][i], b, rel_tol=1e-13, abs_tol=1e-15)
        assert math.isclose(pr["c"][i], c, rel_tol=1e-13)
        # the centre itself is not clamped
        assert math.isclose(pr["u"][i], f * rx + 23.5, rel_tol=1e-14)


def _loss_T(orc, P, cam, T, pix, gr, gd):
    """Render with a float64 pose (bypasses the float32 camera widening)."""
    import ctypes

    oc = orc._cam(cam)
    for k in range(16):
        oc.Tcw[k] = float(T.reshape(16)[k])
    m = pix.shape[0]
    rgb = np.zeros((m, 3))
    depth = np.zeros(m)
    Tf = np.zeros(m)
    n = np.zeros(m, np.int32)
    fl = np.zeros(m, np.int32)
    e = np.zeros(4)
    Pd = np.ascontiguousarray(P, np.float64)
    orc.lib().orc_render(orc._p(Pd), ctypes.c_int64(P.shape[0]), ctypes.c_int(3), ctypes.byref(oc), orc._p(pix),
                         ctypes.c_int64(m), orc._p(e), ctypes.c_int(0), orc._p(rgb), orc._p(depth), orc._p(Tf),
                         orc._p(n), orc._p(fl))
    return float((rgb * gr).sum() + (depth * gd).sum())


def test_depth_f32_matches_float32_dot(orc):
    rng = np.random.default_rng(13)
    m = rng.uniform(-50, 50, (1000, 3)).astype(np.float32)
    cam = _rand_cam(rng)
    z = orc.depth_f32(m, cam)
    proj = orc.project(np.concatenate([m.astype(np.float64), np.zeros((1000, 11))], 1), 0, cam)
    assert np.allclose(z, proj["z"], rtol=1e-6, atol=1e-5)
