"""The batched keyframe window captured as one CUDA graph equals the same
calls issued directly, replay after replay with new poses."""
import numpy as np
import pytest

from paper_2511_23030_b300 import dcg, synth

from gpu_util import make_ctx, planar

pytestmark = pytest.mark.gpu

SIZES = [(400, 224)] * 4 + [(224, 168)] * 2 + [(112, 84)] * 2


def _scene():
    sc = synth.window_scene(0, n=200_000, sizes=SIZES)
    return sc["params"], sc["cams"], sc


def _buffers(cams, F, n):
    import torch

    P = sum(c.W * c.H for c in cams)
    z = lambda k: torch.zeros(k, device="cuda")
    return dict(rgb=z(3 * P), depth=z(P), dr=z(3 * P), dd=z(P), loss=z(1), grads=torch.zeros((F, n), device="cuda"),
                pose=z(6 * len(cams)))


def _direct(ctx, g, n, cams, b, trgb, tdep, lam, deg, lam_s):
    b["loss"].zero_()
    dcg.dcg_render_fwd(ctx, g, n, cams, b["rgb"], b["depth"])
    dcg.dcg_loss(ctx, b["rgb"], b["depth"], trgb, tdep, cams, lam_s, lam, b["dr"], b["dd"], b["loss"])
    dcg.dcg_render_bwd(ctx, b["dr"], b["dd"], dcg.gaussians(b["grads"], deg), b["pose"])
    dcg.dcg_sync(ctx)


@pytest.mark.parametrize("stage", [128, 16])
@pytest.mark.parametrize("lam_s", [0.0, 0.2])
def test_window_graph_equals_direct_calls(lam_s, stage):
    import torch

    P, cams, sc = _scene()
    n, F = P.shape
    ctx = make_ctx(deg=3, n_max=n, views=8, pixels=sum(c.W * c.H for c in cams), stage=stage)
    try:
        g_t = planar(P)
        g = dcg.gaussians(g_t, 3)
        trgb = torch.from_numpy(np.concatenate([np.random.default_rng(1).uniform(0, 1, 3 * c.W * c.H) for c in cams])
                                .astype(np.float32)).cuda()
        tdep = torch.from_numpy(np.concatenate([np.random.default_rng(2).uniform(5, 30, c.W * c.H) for c in cams])
                                .astype(np.float32)).cuda()
        a, b = _buffers(cams, F, n), _buffers(cams, F, n)
        dcg.dcg_window_capture(ctx, g, n, cams, a["rgb"], a["depth"], trgb, tdep, 0.1, a["dr"], a["dd"], a["loss"],
                               dcg.gaussians(a["grads"], 3), a["pose"], lambda_s=lam_s)
        rng = np.random.default_rng(3)
        for it in range(3):
            if it:
                for c in cams:  # move every keyframe a little
                    T = np.asarray(c.Tcw, np.float64).copy()
                    T[:3, 3] += rng.normal(0, 0.2, 3)
                    c.Tcw = T.astype(np.float32)
            dcg.dcg_window_run(ctx, cams)
            dcg.dcg_sync(ctx)
            ra = {k: v.clone() for k, v in a.items()}
            _direct(ctx, g, n, cams, b, trgb, tdep, 0.1, 3, lam_s)
            assert torch.equal(ra["rgb"], b["rgb"]) and torch.equal(ra["depth"], b["depth"])
            assert torch.equal(ra["dr"], b["dr"]) and torch.equal(ra["dd"], b["dd"])
            assert abs(ra["loss"].item() - b["loss"].item()) <= 1e-6 * abs(b["loss"].item())
            rel = ((ra["grads"] - b["grads"]).norm() / b["grads"].norm()).item()
            assert rel <= 1e-5, rel  # only the order of the gradient atomics differs
            relp = ((ra["pose"] - b["pose"]).norm() / b["pose"].norm()).item()
            assert relp <= 1e-5, relp
        bad = list(cams)
        bad[0] = synth.Camera(cams[0].fx, cams[0].fy, cams[0].cx, cams[0].cy, cams[0].W + 16, cams[0].H, cams[0].Tcw)
        with pytest.raises(dcg.DcgError) as e:
            dcg.dcg_window_run(ctx, bad)
        assert e.value.status == 1
    finally:
        dcg.dcg_destroy(ctx)
