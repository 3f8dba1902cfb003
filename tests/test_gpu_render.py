"""Parity of the CUDA renderer (forward and backward) with the FP64 oracle.

Tolerances (fixed by the FP32/FP64 comparison): RGB within 1e-5 absolute per
channel, depth within 1e-5 * max(1, depth) (depth is un-normalised metres),
final transmittance within 1e-5 absolute, at every pixel the oracle does not
flag as near a discrete boundary (support q = 9, alpha = 1/255, T = 1e-4,
depth ties); flagged pixels stay below 0.5 %.  Gradients: relative L2 error
<= 1e-4 per parameter group and for the pose twist.  Sort keys (FP32 depth)
bit-exact; per-tile lists are the unique (depth bits, index) order of the
Gaussians whose rectangle covers the tile."""
import math

import numpy as np
import pytest

from paper_2511_23030_b300 import dcg, synth

from gpu_util import (GRAD_TOL, GROUPS, RGB_TOL, backward, check_image, make_ctx, out_buffers, planar, rel_l2, render,
                      split_views)

pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module")
def ctx():
    c = make_ctx(deg=3, n_max=600_000, views=8)
    yield c
    dcg.dcg_destroy(c)


@pytest.fixture(scope="module")
def ctx0():
    c = make_ctx(deg=0, n_max=100_000, views=8)
    yield c
    dcg.dcg_destroy(c)


# blend kernels: block per tile (warp reductions or lane slots), warp per block,
# half-warp per half block with Gaussians on the lanes in the backward (the
# product launch) or with pixels on the lanes (one Gaussian per half per step)
BWD_VARIANTS = {"warp": dict(flags=0, stage=128), "slots": dict(flags=1, stage=128),
                "warp_per_block": dict(flags=0, stage=32), "half_warp": dict(flags=0, stage=16),
                "half_warp_pixel_lanes": dict(flags=2, stage=16)}


@pytest.fixture(scope="module", params=list(BWD_VARIANTS))
def ctx0b(request):
    # every blend variant: block per tile with warp reductions or lane slots, warp per block
    c = make_ctx(deg=0, n_max=100_000, views=8, **BWD_VARIANTS[request.param])
    yield c
    dcg.dcg_destroy(c)


@pytest.fixture(scope="module", params=list(BWD_VARIANTS))
def ctxb(request):
    c = make_ctx(deg=3, n_max=600_000, views=8, **BWD_VARIANTS[request.param])
    yield c
    dcg.dcg_destroy(c)


def _pix_arrays(rgb_v, depth_v):
    H, W = depth_v.shape
    return rgb_v.reshape(3, -1).T.astype(np.float64), depth_v.reshape(-1).astype(np.float64)


def test_small_view_forward_matches_oracle(ctx0, orc):
    sc = synth.room_small(0)
    P, cam = sc["params"], sc["cams"][0]
    _, _, rgb, depth = render(ctx0, P, 0, [cam])
    (rv, dv), = split_views(rgb, depth, [cam])
    st = dcg.dcg_state_read(ctx0, None, 1, P.shape[0], cam.W * cam.H)
    o = orc.render(P, 0, cam)
    r, d = _pix_arrays(rv, dv)
    check_image(o, r, d, st["T"].astype(np.float64), "room_small")
    assert (o["n"] > 0).mean() > 0.5


def test_sort_keys_bit_exact_and_tile_lists_valid(ctx0, orc):
    sc = synth.room_small(0)
    P, cam = sc["params"], sc["cams"][0]
    n = P.shape[0]
    render(ctx0, P, 0, [cam])
    st = dcg.dcg_state_read(ctx0, None, 1, n, cam.W * cam.H)
    z32 = orc.depth_f32(P[:, :3], cam)
    assert np.array_equal(st["depth"].view(np.uint32), z32.view(np.uint32))
    # per tile: the Gaussians whose rectangle covers it, in (depth bits, index) order, less those
    # whose support ellipse misses the tile.  What is left out must miss it: q > 9 at every pixel of
    # the tile by the oracle's FP64 conic.  Half-block masks likewise: a cleared bit 2 b + h means
    # q > 9 at every pixel of the 4 x 4 half h of the 8 x 4 block b.
    pr = orc.project(P, 0, cam)
    rect = st["rect"]
    vis = rect[:, 2] >= rect[:, 0]
    ntx = (cam.W + 15) // 16
    ranges, ids, masks = st["ranges"], st["ids"], st["masks"]
    zb = st["depth"].view(np.uint32)
    by, bx = np.mgrid[0:4, 0:4]

    def q_at(g, xs, ys):
        dx, dy = xs - pr["u"][g], ys - pr["v"][g]
        return pr["A"][g] * dx * dx + 2.0 * pr["B"][g] * dx * dy + pr["C"][g] * dy * dy

    dropped = kept = 0
    for t in range(ranges.shape[0]):
        ty, tx = divmod(t, ntx)
        lst = ids[ranges[t, 0]:ranges[t, 1]]
        msk = masks[ranges[t, 0]:ranges[t, 1]]
        want = np.nonzero(vis & (rect[:, 0] <= tx) & (rect[:, 2] >= tx) & (rect[:, 1] <= ty) & (rect[:, 3] >= ty))[0]
        want = want[np.lexsort((want, zb[want]))]
        assert np.array_equal(lst, want[np.isin(want, lst)]), t  # an ordered subsequence
        for g in want[~np.isin(want, lst)]:
            ys, xs = np.mgrid[16 * ty:16 * ty + 16, 16 * tx:16 * tx + 16]
            assert q_at(g, xs, ys).min() > 9.0, (t, g)
            dropped += 1
        for g, m in zip(lst, msk):
            assert m != 0, (t, g)
            for hb in range(16):
                if not (int(m) >> hb) & 1:
                    b, h = divmod(hb, 2)
                    xs = 16 * tx + 8 * (b % 2) + 4 * h + bx
                    ys = 16 * ty + 4 * (b // 2) + by
                    assert q_at(g, xs, ys).min() > 9.0, (t, g, hb)
            kept += 1
    assert kept > 0 and dropped > 0
    # rectangles agree with the oracle's FP64 extents except within rounding of a pixel boundary
    x0 = np.floor(pr["u"] - pr["ex"])
    x1 = np.ceil(pr["u"] + pr["ex"])
    near = (np.abs(pr["u"] - pr["ex"] - np.round(pr["u"] - pr["ex"])) < 1e-4) | (
        np.abs(pr["u"] + pr["ex"] - np.round(pr["u"] + pr["ex"])) < 1e-4)
    inside = (pr["vis"] > 0) & (x1 >= 0) & (x0 <= cam.W - 1)
    tx0 = (np.clip(x0, 0, cam.W - 1) // 16).astype(int)
    good = inside & ~near & vis
    assert np.array_equal(rect[good, 0], tx0[good])


def test_small_view_backward_matches_oracle(ctx0b, orc):
    ctx0 = ctx0b
    sc = synth.room_small(0)
    P, cam = sc["params"], sc["cams"][0]
    n = P.shape[0]
    g_t, g, rgb, depth = render(ctx0, P, 0, [cam])
    o = orc.render(P, 0, cam)
    rng = np.random.default_rng(5)
    Pn = cam.W * cam.H
    gr = rng.normal(size=(Pn, 3))
    gd = rng.normal(size=Pn) * 0.1
    gr[o["flags"] != 0] = 0
    gd[o["flags"] != 0] = 0
    import torch

    dr = torch.from_numpy(np.ascontiguousarray(gr.T.reshape(-1)).astype(np.float32)).cuda()
    dd = torch.from_numpy(gd.astype(np.float32)).cuda()
    grad, pose = backward(ctx0, g_t, 0, n, dr, dd, 1)
    og, opose = orc.render_bwd(P, 0, cam, gr, gd)
    for name, sl in GROUPS.items():
        e = rel_l2(grad[:, sl], og[:, sl])
        assert e <= GRAD_TOL, (name, e)
    assert rel_l2(pose[0], opose) <= GRAD_TOL, (pose[0], opose)


def _room_views(n=120_000, n_views=3, seed=1):
    sc = synth.room_indoor(seed, n=n, n_steps=n_views)
    return sc["params"], sc["cams"]


def test_room_sh3_sampled_pixels_and_sparse_seed_gradients(ctxb, orc):
    ctx = ctxb
    P, cams = _room_views(n=60_000, n_views=1, seed=1)
    cam = cams[0]
    n = P.shape[0]
    g_t, g, rgb, depth = render(ctx, P, 3, [cam])
    (rv, dv), = split_views(rgb, depth, [cam])
    rng = np.random.default_rng(3)
    # a dense 40x32 window plus scattered pixels
    ys, xs = np.mgrid[200:232, 300:340]
    win = np.stack([xs.ravel(), ys.ravel()], 1).astype(np.int32)
    pix = np.concatenate([win, synth.pixel_sample(rng, cam.W, cam.H, 1500)])
    pix = np.unique(pix, axis=0)
    o = orc.render(P, 3, cam, pix=pix)
    r = rv[:, pix[:, 1], pix[:, 0]].T.astype(np.float64)
    d = dv[pix[:, 1], pix[:, 0]].astype(np.float64)
    st = dcg.dcg_state_read(ctx, None, 1, n, cam.W * cam.H)
    T = st["T"].reshape(cam.H, cam.W)[pix[:, 1], pix[:, 0]].astype(np.float64)
    check_image(o, r, d, T, "room_indoor")
    # gradient of a loss seeded only on these pixels
    gr = rng.normal(size=(len(pix), 3))
    gd = rng.normal(size=len(pix)) * 0.1
    gr[o["flags"] != 0] = 0
    gd[o["flags"] != 0] = 0
    import torch

    full_r = np.zeros((3, cam.H, cam.W), np.float32)
    full_d = np.zeros((cam.H, cam.W), np.float32)
    full_r[:, pix[:, 1], pix[:, 0]] = gr.T
    full_d[pix[:, 1], pix[:, 0]] = gd
    dr = torch.from_numpy(full_r.reshape(-1)).cuda()
    dd = torch.from_numpy(full_d.reshape(-1)).cuda()
    grad, pose = backward(ctx, g_t, 3, n, dr, dd, 1)
    og, opose = orc.render_bwd(P, 3, cam, gr, gd, pix=pix)
    for name, sl in GROUPS.items():
        e = rel_l2(grad[:, sl], og[:, sl])
        assert e <= GRAD_TOL, (name, e)
    assert rel_l2(pose[0], opose) <= GRAD_TOL


def test_batched_views_equal_single_views(ctx):
    P, cams = _room_views(n=60_000, n_views=3, seed=2)
    sizes = [(640, 480), (320, 240), (200, 150)]
    for c, (W, H) in zip(cams, sizes):
        c.W, c.H, c.cx, c.cy = W, H, W / 2, H / 2
        c.fx = c.fy = 0.8 * W
    _, _, rgb_b, depth_b = render(ctx, P, 3, cams)
    batched = split_views(rgb_b, depth_b, cams)
    for v, c in enumerate(cams):
        _, _, rgb_s, depth_s = render(ctx, P, 3, [c])
        (rs, ds), = split_views(rgb_s, depth_s, [c])
        assert np.array_equal(rs, batched[v][0]) and np.array_equal(ds, batched[v][1])


@pytest.mark.parametrize("tile,stage", [((16, 16), 64), ((32, 16), 128), ((32, 32), 256), ((16, 16), 192),
                                        ((32, 32), 96), ((16, 16), 32), ((32, 16), 32),
                                        ((32, 32), 32), ((16, 16), 16), ((32, 16), 16), ((32, 32), 16)])
def test_launch_shapes_agree(ctx, tile, stage):
    P, cams = _room_views(n=60_000, n_views=1, seed=4)
    dcg.dcg_set_launch(ctx, 16, 16, 128)
    _, _, r0, d0 = render(ctx, P, 3, cams)
    dcg.dcg_set_launch(ctx, tile[0], tile[1], stage)
    try:
        _, _, r1, d1 = render(ctx, P, 3, cams)
    finally:
        dcg.dcg_set_launch(ctx, 16, 16, 128)
    # only the rounding of tile-local coordinates differs between launch shapes
    assert (r0 - r1).abs().max().item() <= RGB_TOL
    assert ((d0 - d1).abs() / d0.abs().clamp(min=1)).max().item() <= RGB_TOL


def test_edge_cases(ctx0):
    import torch

    sc = synth.room_small(0)
    cam = sc["cams"][0]
    # no Gaussians
    P = sc["params"][:0]
    _, _, rgb, depth = render(ctx0, P, 0, [cam])
    assert rgb.abs().max().item() == 0 and depth.abs().max().item() == 0
    # everything behind the camera
    P = sc["params"].copy()
    P[:, 2] = -3.0
    _, _, rgb, depth = render(ctx0, P, 0, [cam])
    assert rgb.abs().max().item() == 0
    # ragged 1x1 and 17x33 images
    for W, H in ((1, 1), (17, 33)):
        c = synth.Camera(100.0, 100.0, W / 2, H / 2, W, H, cam.Tcw, 0.2, 100.0)
        _, _, rgb, depth = render(ctx0, sc["params"], 0, [c])
        assert torch.isfinite(rgb).all()
    # backward with zero seed gives zero gradients
    g_t, g, rgb, depth = render(ctx0, sc["params"], 0, [cam])
    grad, pose = backward(ctx0, g_t, 0, sc["params"].shape[0], torch.zeros_like(rgb), torch.zeros_like(depth), 1)
    assert np.abs(grad).max() == 0 and np.abs(pose).max() == 0


def test_loss_l1_matches_definition(ctx0, orc):
    import torch

    sc = synth.room_small(0)
    cams = sc["cams"] * 2
    P = sum(c.W * c.H for c in cams)
    rng = np.random.default_rng(0)
    rgb = torch.from_numpy(rng.uniform(0, 1, 3 * P).astype(np.float32)).cuda()
    dep = torch.from_numpy(rng.uniform(0, 5, P).astype(np.float32)).cuda()
    trgb = torch.from_numpy(rng.uniform(0, 1, 3 * P).astype(np.float32)).cuda()
    tdep = torch.from_numpy(rng.uniform(0, 5, P).astype(np.float32)).cuda()
    dr, dd, loss = torch.zeros_like(rgb), torch.zeros_like(dep), torch.zeros(1, device="cuda")
    dcg.dcg_loss_l1(ctx0, rgb, dep, trgb, tdep, cams, 0.1, dr, dd, loss)
    dcg.dcg_sync(ctx0)
    L = 0.0
    for v in range(2):
        Pv = cams[v].W * cams[v].H
        sl3 = slice(3 * v * Pv, 3 * (v + 1) * Pv)
        sl = slice(v * Pv, (v + 1) * Pv)
        Lv, gr, gd = orc.l1_loss(rgb[sl3].cpu().numpy(), dep[sl].cpu().numpy(), trgb[sl3].cpu().numpy(),
                                 tdep[sl].cpu().numpy(), 0.1)
        L += Lv
        assert np.allclose(dr[sl3].cpu().numpy(), gr, rtol=1e-6, atol=0)
        assert np.allclose(dd[sl].cpu().numpy(), gd, rtol=1e-6, atol=0)
    assert math.isclose(loss.item(), L, rel_tol=1e-5)


def test_second_backward_of_one_forward_gives_the_same_gradients(ctx0b):
    """The per-pair 2D gradient slots are consumed (and zeroed) by each
    backward, so a second backward of the same forward does not accumulate
    on top of the first."""
    import torch

    sc = synth.room_small(0)
    P, cam = sc["params"], sc["cams"][0]
    n = P.shape[0]
    g_t, _, rgb, depth = render(ctx0b, P, 0, [cam])
    rng = np.random.default_rng(7)
    dr = torch.from_numpy(rng.normal(size=rgb.numel()).astype(np.float32)).cuda()
    dd = torch.from_numpy((0.1 * rng.normal(size=depth.numel())).astype(np.float32)).cuda()
    g1, p1 = backward(ctx0b, g_t, 0, n, dr, dd, 1)
    g2, p2 = backward(ctx0b, g_t, 0, n, dr, dd, 1)
    assert np.abs(g1).max() > 0
    assert rel_l2(g2, g1) <= 1e-6 and rel_l2(p2, p1) <= 1e-6


def test_capacity_errors_leave_the_context_usable():
    """More instances than configured: the forward clamps its lists (no
    access past the capacity) and the next dcg_sync reports
    DCG_ERR_CAPACITY; the context then renders a scene that fits.  More
    pixels than configured is a capacity error and more views an argument
    error, both returned at once."""
    sc = synth.room_small(0)
    P, cam = sc["params"], sc["cams"][0]
    n = P.shape[0]
    ctx = make_ctx(deg=0, n_max=n, views=1, pixels=cam.W * cam.H, inst=2000)
    try:
        g_t = planar(P)
        g = dcg.gaussians(g_t, 0)
        rgb, depth = out_buffers([cam])
        dcg.dcg_render_fwd(ctx, g, n, [cam], rgb, depth)
        with pytest.raises(dcg.DcgError) as e:
            dcg.dcg_sync(ctx)
        assert e.value.status == 6
        small = P[:50].copy()
        _, _, rgb_s, _ = render(ctx, small, 0, [cam])  # syncs: no error left over
        assert float(rgb_s.abs().sum()) > 0
        big = synth.Camera(cam.fx, cam.fy, cam.cx, cam.cy, 2 * cam.W, cam.H, cam.Tcw, cam.znear, cam.zfar)
        rgb2, depth2 = out_buffers([big])
        with pytest.raises(dcg.DcgError) as e:
            dcg.dcg_render_fwd(ctx, g, n, [big], rgb2, depth2)
        assert e.value.status == 6
        with pytest.raises(dcg.DcgError) as e:
            dcg.dcg_render_fwd(ctx, g, n, [cam, cam], rgb2, depth2)
        assert e.value.status == 1
    finally:
        dcg.dcg_destroy(ctx)


@pytest.mark.parametrize("deg", [1, 2])
def test_sixteen_views_batched_equal_single_and_oracle(deg, orc):
    """The largest batch the ABI takes (16 views of uneven sizes) in the
    default half-warp launch: every view equals its single-view render bit for
    bit, and sampled pixels of the last view and the gradients of a loss
    seeded on them match the oracle (SH degrees 1 and 2, which the other
    tests do not render)."""
    P3, cams = _room_views(n=20_000, n_views=16, seed=3)
    F = 11 + 3 * (deg + 1) ** 2
    P = np.ascontiguousarray(P3[:, :F])
    rng = np.random.default_rng(deg)
    for c in cams:
        W = int(rng.integers(40, 200))
        H = int(rng.integers(30, 150))
        c.W, c.H, c.cx, c.cy = W, H, W / 2, H / 2
        c.fx = c.fy = 0.8 * W
    ctx = make_ctx(deg=deg, n_max=P.shape[0], views=16, pixels=sum(c.W * c.H for c in cams), stage=16)
    try:
        _, _, rgb_b, depth_b = render(ctx, P, deg, cams)
        batched = split_views(rgb_b, depth_b, cams)
        for v, c in enumerate(cams):
            _, _, rgb_s, depth_s = render(ctx, P, deg, [c])
            (rs, ds), = split_views(rgb_s, depth_s, [c])
            assert np.array_equal(rs, batched[v][0]) and np.array_equal(ds, batched[v][1]), v
        c = cams[-1]
        pix = synth.pixel_sample(rng, c.W, c.H, 200)
        o = orc.render(P, deg, c, pix=pix)
        rv, dv = batched[-1]
        st = dcg.dcg_state_read(ctx, None, 1, P.shape[0], c.W * c.H)
        T = st["T"].reshape(c.H, c.W)
        check_image(o, rv[:, pix[:, 1], pix[:, 0]].T.astype(np.float64), dv[pix[:, 1], pix[:, 0]].astype(np.float64),
                    T[pix[:, 1], pix[:, 0]].astype(np.float64), f"16 views deg {deg}")
        # gradients at this degree, seeded on the sampled pixels of the last view
        import torch

        g_t, _, _, _ = render(ctx, P, deg, [c])
        gr = rng.normal(size=(len(pix), 3))
        gd = rng.normal(size=len(pix)) * 0.1
        gr[o["flags"] != 0] = 0
        gd[o["flags"] != 0] = 0
        full_r = np.zeros((3, c.H, c.W), np.float32)
        full_d = np.zeros((c.H, c.W), np.float32)
        full_r[:, pix[:, 1], pix[:, 0]] = gr.T
        full_d[pix[:, 1], pix[:, 0]] = gd
        grad, pose = backward(ctx, g_t, deg, P.shape[0], torch.from_numpy(full_r.reshape(-1)).cuda(),
                              torch.from_numpy(full_d.reshape(-1)).cuda(), 1)
        og, opose = orc.render_bwd(P, deg, c, gr.astype(np.float32).astype(np.float64),
                                   gd.astype(np.float32).astype(np.float64), pix=pix)
        for name, sl in GROUPS.items():
            assert rel_l2(grad[:, sl], og[:, sl]) <= GRAD_TOL, (name, deg)
        assert rel_l2(pose[0], opose) <= GRAD_TOL
    finally:
        dcg.dcg_destroy(ctx)


def test_phase_timers_report_a_full_pool(ctx0):
    # the timers hold 4096 intervals between reads (three a forward call); a read after more
    # returns the recorded figures and reports DCG_ERR_CAPACITY, and the next read is clean
    sc = synth.room_small(0)
    P, cam = sc["params"], sc["cams"][0]
    g_t = planar(P)
    g = dcg.gaussians(g_t, 0)
    rgb, depth = out_buffers([cam])
    dcg.dcg_profile(ctx0, True)
    try:
        dcg.dcg_profile_read(ctx0)
        for _ in range(1000):
            dcg.dcg_render_fwd(ctx0, g, P.shape[0], [cam], rgb, depth)
        prof = dcg.dcg_profile_read(ctx0)  # 3000 intervals: within the pool
        assert prof["blend_fwd"][1] == 1000
        for _ in range(1500):
            dcg.dcg_render_fwd(ctx0, g, P.shape[0], [cam], rgb, depth)
        with pytest.raises(dcg.DcgError) as err:
            dcg.dcg_profile_read(ctx0)
        assert dcg.STATUS[err.value.status] == "DCG_ERR_CAPACITY"
        dcg.dcg_render_fwd(ctx0, g, P.shape[0], [cam], rgb, depth)
        prof = dcg.dcg_profile_read(ctx0)
        assert prof["blend_fwd"][1] == 1
    finally:
        dcg.dcg_profile(ctx0, False)
        dcg.dcg_sync(ctx0)
