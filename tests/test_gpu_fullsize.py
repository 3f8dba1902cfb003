"""The benchmark's keyframe window at its full size (2M Gaussians in 64 chunks
of 4 m, 8 views of 4 x 1200x680, 2 x 640x480 and 2 x 320x240 pixels) through
the chunk path, in the launch shapes the benchmark's autotuner picks from,
against the oracle on sampled pixels of two views: the images, and the
parameter and pose gradients of a loss seeded on those pixels only.

A pixel of this scene weighs about a hundred Gaussians, so one of them is
more often within the oracle's derived FP32 error band of a discrete
threshold (q = 9, alpha = 1/255, T = 1e-4) than in the sparse test scenes: the
oracle flags 0 to 1.2 % of the pixels of each of the eight views (0.36 % over
4800 sampled pixels), so at most 2 % of the sampled pixels may be flagged (and
skipped)."""
import numpy as np
import pytest

from paper_2511_23030_b300 import dcg, synth

from gpu_util import GRAD_TOL, GROUPS, check_image, make_ctx, out_buffers, planar, rel_l2, split_views

pytestmark = pytest.mark.gpu

VIEWS = (0, 5)  # one 1200x680 and one 640x480 keyframe


@pytest.fixture(scope="module")
def window():
    return synth.window_scene(0)


def _pixels(rng, c):
    """A dense 16 x 8 patch at the image centre plus 48 scattered pixels."""
    ys, xs = np.mgrid[c.H // 2 - 4: c.H // 2 + 4, c.W // 2 - 8: c.W // 2 + 8]
    patch = np.stack([xs.ravel(), ys.ravel()], 1).astype(np.int32)
    return np.unique(np.concatenate([patch, synth.pixel_sample(rng, c.W, c.H, 48)]), axis=0)


@pytest.mark.parametrize("stage", [16, 32])
def test_full_window_sampled_pixels_and_gradients(window, orc, stage):
    import torch

    P, cams = window["params"], window["cams"]
    n, F = P.shape
    npix = sum(c.W * c.H for c in cams)
    offs = np.cumsum([0] + [c.W * c.H for c in cams])
    ctx = make_ctx(deg=3, n_max=n, views=len(cams), pixels=npix, inst=40 << 20, chunk=window["chunk_size"], host=n,
                   dfar=60.0, tile=(16, 16), stage=stage)
    try:
        dcg.dcg_chunk_table_update(ctx, planar(P), n)
        g, na = dcg.dcg_gather_active(ctx, dcg.dcg_cull_chunks(ctx, cams))
        assert na == n
        A = dcg.active_tensor(g, n, F).T.cpu().numpy()  # the active set in gather order: the oracle's input
        rgb, depth = out_buffers(cams)
        dcg.dcg_render_fwd(ctx, g, n, cams, rgb, depth)
        dcg.dcg_sync(ctx)
        per_view = split_views(rgb, depth, cams)
        st = dcg.dcg_state_read(ctx, None, len(cams), n, npix)
        rng = np.random.default_rng(11)
        dr = np.zeros(3 * npix, np.float32)
        dd = np.zeros(npix, np.float32)
        want_g = np.zeros((n, F))
        want_pose = {}
        for v in VIEWS:
            c = cams[v]
            pix = _pixels(rng, c)
            o = orc.render(A, 3, c, pix=pix)
            rv, dv = per_view[v]
            T = st["T"][offs[v]: offs[v + 1]].reshape(c.H, c.W)
            check_image(o, rv[:, pix[:, 1], pix[:, 0]].T.astype(np.float64),
                        dv[pix[:, 1], pix[:, 0]].astype(np.float64), T[pix[:, 1], pix[:, 0]].astype(np.float64),
                        f"view {v} stage {stage}", max_flag=0.02)
            gr = rng.normal(size=(len(pix), 3))
            gd = rng.normal(size=len(pix)) * 0.1
            gr[o["flags"] != 0] = 0
            gd[o["flags"] != 0] = 0
            k = pix[:, 1].astype(np.int64) * c.W + pix[:, 0]
            Pv = c.W * c.H
            for ch in range(3):
                dr[3 * offs[v] + ch * Pv + k] = gr[:, ch]
            dd[offs[v] + k] = gd
            og, opose = orc.render_bwd(A, 3, c, gr.astype(np.float32).astype(np.float64),
                                       gd.astype(np.float32).astype(np.float64), pix=pix)
            want_g += og
            want_pose[v] = opose
        grads_t = torch.zeros((F, n), device="cuda")
        pose = torch.zeros(6 * len(cams), device="cuda")
        dcg.dcg_render_bwd(ctx, torch.from_numpy(dr).cuda(), torch.from_numpy(dd).cuda(), dcg.gaussians(grads_t, 3),
                           pose)
        dcg.dcg_sync(ctx)
        got = grads_t.T.cpu().numpy().astype(np.float64)
        for name, sl in GROUPS.items():
            e = rel_l2(got[:, sl], want_g[:, sl])
            assert e <= GRAD_TOL, (name, e)
        pose = pose.view(len(cams), 6).cpu().numpy().astype(np.float64)
        for v in range(len(cams)):
            if v in want_pose:
                assert rel_l2(pose[v], want_pose[v]) <= GRAD_TOL, (v, pose[v], want_pose[v])
            else:
                assert not pose[v].any()  # no seed in this view
    finally:
        dcg.dcg_destroy(ctx)
