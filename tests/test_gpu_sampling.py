"""LoG penalty sampling of Eq. 1 and back-projection against the references;
sampled Gaussians enter the chunk table."""
import numpy as np
import pytest

from oracle import logsample as ls
from paper_2511_23030_b300 import dcg, synth

from gpu_util import make_ctx, render, planar

pytestmark = pytest.mark.gpu


def _images(W, H, seed):
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    base = np.stack([0.5 + 0.4 * np.sin(0.3 * x + 0.2 * y), 0.5 + 0.4 * np.cos(0.25 * y), 0.3 + 0.002 * x])
    img = base + (rng.uniform(0, 1, (3, H, W)) < 0.05) * 0.5  # sparse bright details
    ren = base + 0.1 * rng.normal(size=(3, H, W))
    return np.clip(img, 0, 1).astype(np.float32), np.clip(ren, 0, 1).astype(np.float32)


@pytest.mark.parametrize("W,H", [(100, 70), (37, 23), (16, 16)])
def test_penalty_and_samples_match_reference(W, H):
    import torch

    img, ren = _images(W, H, W)
    u = np.random.default_rng(1).uniform(0, 1, W * H).astype(np.float32)
    ctx = make_ctx(deg=0, n_max=1000, views=1, pixels=W * H)
    try:
        ti, tr, tu = (torch.from_numpy(a.reshape(-1)).cuda() for a in (img, ren, u))
        ps = torch.zeros(W * H, device="cuda")
        idx = torch.zeros(W * H, dtype=torch.int32, device="cuda")
        dcg.dcg_profile(ctx, True)
        n = dcg.dcg_log_sample(ctx, ti, tr, W, H, 3.0, tu, idx, ps_out=ps)
        prof = dcg.dcg_profile_read(ctx)
        dcg.dcg_profile(ctx, False)
        assert prof["log_sample"][1] == 1 and prof["log_sample"][0] > 0  # one timed interval
        assert all(v[1] == 0 for k, v in prof.items() if k != "log_sample")
        want = ls.penalty(img, ren).reshape(-1)
        got = ps.cpu().numpy().astype(np.float64)
        assert np.abs(got - want).max() <= 1e-5 * want.max() + 1e-6
        got_idx = set(idx[:n].cpu().numpy().tolist())
        assert list(idx[:n].cpu().numpy()) == sorted(got_idx)  # ascending
        ref_idx = set(ls.sample(want, u, 3.0).tolist())
        # decisions may differ only where u is within rounding of the threshold
        amb = set(np.nonzero(np.abs(u - np.minimum(1.0, 3.0 * want)) <= 1e-5)[0].tolist())
        assert (got_idx ^ ref_idx) <= amb and len(got_idx) > 0
        # capacity: fewer slots than samples
        small = torch.zeros(max(1, n // 2), dtype=torch.int32, device="cuda")
        with pytest.raises(dcg.DcgError) as e:
            dcg.dcg_log_sample(ctx, ti, tr, W, H, 3.0, tu, small)
        assert e.value.status == 6
    finally:
        dcg.dcg_destroy(ctx)


def test_backprojection_and_insertion_into_chunks():
    import torch

    sc = synth.room_small(0)
    P, cam = sc["params"], sc["cams"][0]
    W, H = cam.W, cam.H
    ctx = make_ctx(deg=0, n_max=20_000, views=1, pixels=W * H, chunk=1.0, host=40_000)
    try:
        # the input image is the full scene, the current map holds half of it
        _, _, img, dep = render(ctx, P, 0, [cam])
        _, _, ren, _ = render(ctx, P[::2].copy(), 0, [cam])
        u = torch.from_numpy(np.random.default_rng(2).uniform(0, 1, W * H).astype(np.float32)).cuda()
        idx = torch.zeros(W * H, dtype=torch.int32, device="cuda")
        n = dcg.dcg_log_sample(ctx, img, ren, W, H, 20.0, u, idx)
        assert n > 10
        # depths where the full scene rendered something
        d = dep.clone()
        d[d <= 0.05] = 1.0
        F = 11 + 3
        out = torch.zeros((F, n), device="cuda")
        dcg.dcg_backproject(ctx, idx, n, d, img, cam, 0.0, out)
        dcg.dcg_sync(ctx)
        want = ls.backproject(idx[:n].cpu().numpy(), d.cpu().numpy(), img.cpu().numpy().reshape(3, H, W), cam, 0.0, F)
        got = out.T.cpu().numpy().astype(np.float64)
        assert np.allclose(got, want, rtol=2e-6, atol=2e-6)
        # into the chunk table: the map grows by the sampled Gaussians
        dcg.dcg_chunk_table_update(ctx, planar(P), P.shape[0])
        dcg.dcg_chunk_table_update(ctx, out, n)
        info = dcg.dcg_chunk_info(ctx)
        assert int(info["counts"].sum()) == P.shape[0] + n
    finally:
        dcg.dcg_destroy(ctx)


def _posed_cam(W, H, f, yaw, t):
    c, s = np.cos(yaw), np.sin(yaw)
    T = np.eye(4, dtype=np.float32)
    T[:3, :3] = [[c, 0, s], [0, 1, 0], [-s, 0, c]]
    T[:3, 3] = t
    return synth.Camera(f, f * 1.05, W / 2.0 + 0.3, H / 2.0 - 0.2, W, H, T, 0.2, 100.0)


WINDOWS = {
    "three_views": [(100, 70), (37, 23), (16, 16)],
    # the most views a call takes, uneven and mostly below one 32 x 32 tile
    "sixteen_views": [(1, 1), (5, 3), (33, 31), (64, 8), (2, 40), (17, 17), (31, 33), (3, 1),
                      (40, 40), (7, 9), (1, 64), (32, 32), (9, 2), (65, 33), (4, 4), (12, 30)],
}


@pytest.mark.parametrize("window", list(WINDOWS))
def test_window_of_views_in_one_call_matches_reference_and_single_calls(window):
    """A window of views of uneven sizes through dcg_log_sample_views / dcg_backproject_views: per
    view the same P_s and samples as the one-view call (bit-identical) and as the reference; window
    indices ascending; per-view counts; back-projection with each view's own pose."""
    import torch

    sizes = WINDOWS[window]
    cams = [_posed_cam(W, H, 80.0 + 10 * k, 0.1 * k, (0.2 * k, -0.1, 0.05 * k)) for k, (W, H) in enumerate(sizes)]
    offs = np.cumsum([0] + [W * H for W, H in sizes])
    N = int(offs[-1])
    imgs, rens = zip(*[_images(W, H, 7 + k) for k, (W, H) in enumerate(sizes)])
    u = np.random.default_rng(3).uniform(0, 1, N).astype(np.float32)
    kappa = 3.0
    ctx = make_ctx(deg=0, n_max=1000, views=1, pixels=N)
    try:
        ti = torch.from_numpy(np.concatenate([a.reshape(-1) for a in imgs])).cuda()
        tr = torch.from_numpy(np.concatenate([a.reshape(-1) for a in rens])).cuda()
        tu = torch.from_numpy(u).cuda()
        ps = torch.zeros(N, device="cuda")
        idx = torch.zeros(N, dtype=torch.int32, device="cuda")
        n, counts = dcg.dcg_log_sample_views(ctx, cams, ti, tr, kappa, tu, idx, ps_out=ps)
        got = idx[:n].cpu().numpy().astype(np.int64)
        assert (np.diff(got) > 0).all() and n == counts.sum()
        ps_h = ps.cpu().numpy()
        for v, (W, H) in enumerate(sizes):
            o, P = int(offs[v]), W * H
            mine = got[(got >= o) & (got < o + P)] - o
            assert len(mine) == counts[v]
            # the one-view call: identical penalty and samples
            ps1 = torch.zeros(P, device="cuda")
            idx1 = torch.zeros(P, dtype=torch.int32, device="cuda")
            n1 = dcg.dcg_log_sample(ctx, ti[3 * o: 3 * (o + P)], tr[3 * o: 3 * (o + P)], W, H, kappa, tu[o: o + P],
                                    idx1, ps_out=ps1)
            assert np.array_equal(idx1[:n1].cpu().numpy(), mine)
            assert np.array_equal(ps1.cpu().numpy(), ps_h[o: o + P])
            # the reference
            want = ls.penalty(imgs[v], rens[v]).reshape(-1)
            assert np.abs(ps_h[o: o + P] - want).max() <= 1e-5 * want.max() + 1e-6
            amb = set(np.nonzero(np.abs(u[o: o + P] - np.minimum(1.0, kappa * want)) <= 1e-5)[0].tolist())
            assert set(mine.tolist()) ^ set(ls.sample(want, u[o: o + P], kappa).tolist()) <= amb
        # capacity: the counts still describe every sample
        small = torch.zeros(max(1, n // 2), dtype=torch.int32, device="cuda")
        with pytest.raises(dcg.DcgError) as e:
            dcg.dcg_log_sample_views(ctx, cams, ti, tr, kappa, tu, small)
        assert e.value.status == 6
        # back-projection of the whole window's samples with each view's pose
        depth = np.random.default_rng(5).uniform(0.5, 4.0, N).astype(np.float32)
        F = 14
        out = torch.zeros((F, n), device="cuda")
        dcg.dcg_backproject_views(ctx, idx, n, torch.from_numpy(depth).cuda(), ti, cams, -1.5, out)
        dcg.dcg_sync(ctx)
        gotp = out.T.cpu().numpy().astype(np.float64)
        for v, (W, H) in enumerate(sizes):
            o, P = int(offs[v]), W * H
            sel = (got >= o) & (got < o + P)
            want = ls.backproject(got[sel] - o, depth[o: o + P], imgs[v], cams[v], -1.5, F)
            assert np.allclose(gotp[sel], want, rtol=2e-6, atol=2e-6), v
    finally:
        dcg.dcg_destroy(ctx)
