"""The loss of Eq. 2-4 with the SSIM term of Eq. 3 against the FP64 reference."""
import math

import numpy as np
import pytest

from oracle import ssim
from paper_2511_23030_b300 import dcg, synth

from gpu_util import make_ctx, rel_l2

pytestmark = pytest.mark.gpu

SIZES = [(37, 23), (64, 48), (130, 97), (16, 16), (5, 40)]


def _cams():
    return [synth.Camera(100.0, 100.0, W / 2, H / 2, W, H, np.eye(4, dtype=np.float32)) for W, H in SIZES]


def _images(seed):
    rng = np.random.default_rng(seed)
    rgb, tgt, dep, tdep = [], [], [], []
    for k, (W, H) in enumerate(SIZES):
        t = rng.uniform(0, 1, (3, H, W))
        # a rendered image near its target in part of the views, unrelated in others
        r = np.clip(t + rng.normal(0, 0.05, t.shape), 0, 1) if k % 2 == 0 else rng.uniform(0, 1, t.shape)
        rgb.append(r.astype(np.float32))
        tgt.append(t.astype(np.float32))
        dep.append(rng.uniform(1, 20, (H, W)).astype(np.float32))
        tdep.append(rng.uniform(1, 20, (H, W)).astype(np.float32))
    return rgb, tgt, dep, tdep


def _flat(xs):
    import torch

    return torch.from_numpy(np.concatenate([x.reshape(-1) for x in xs])).cuda()


@pytest.mark.parametrize("lam_s", [0.2, 1.0])
def test_loss_with_ssim_matches_reference(orc, lam_s):
    import torch

    cams = _cams()
    rgb, tgt, dep, tdep = _images(0)
    ctx = make_ctx(deg=0, n_max=1000, views=8, pixels=sum(W * H for W, H in SIZES))
    try:
        r, t, d, td = _flat(rgb), _flat(tgt), _flat(dep), _flat(tdep)
        dr, dd, loss = torch.zeros_like(r), torch.zeros_like(d), torch.zeros(1, device="cuda")
        dcg.dcg_loss(ctx, r, d, t, td, cams, lam_s, 0.1, dr, dd, loss)
        dcg.dcg_sync(ctx)
        L = 0.0
        o3 = o1 = 0
        for k, (W, H) in enumerate(SIZES):
            P = W * H
            Li, gr1, gd = orc.l1_loss(rgb[k], dep[k], tgt[k], tdep[k], 0.1)
            Ls, grs = ssim.ssim_term(rgb[k], tgt[k], lam_s)
            img_l1 = np.abs(rgb[k].astype(np.float64) - tgt[k]).sum() / (3 * P)
            L += (1 - lam_s) * img_l1 + (Li - img_l1) + Ls
            want = (1 - lam_s) * gr1 + grs
            got = dr[o3:o3 + 3 * P].cpu().numpy().astype(np.float64).reshape(3, H, W)
            assert rel_l2(got, want) <= 1e-5, (k, rel_l2(got, want))
            assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()
            assert np.allclose(dd[o1:o1 + P].cpu().numpy().reshape(H, W), gd, rtol=1e-6, atol=0)
            o3 += 3 * P
            o1 += P
        assert math.isclose(loss.item(), L, rel_tol=2e-6), (loss.item(), L)
    finally:
        dcg.dcg_destroy(ctx)


def test_lambda_s_zero_is_the_l1_loss():
    import torch

    cams = _cams()
    rgb, tgt, dep, tdep = _images(1)
    ctx = make_ctx(deg=0, n_max=1000, views=8, pixels=sum(W * H for W, H in SIZES))
    try:
        r, t, d, td = _flat(rgb), _flat(tgt), _flat(dep), _flat(tdep)
        def run(fn):
            dr, dd, loss = torch.zeros_like(r), torch.zeros_like(d), torch.zeros(1, device="cuda")
            fn(dr, dd, loss)
            dcg.dcg_sync(ctx)
            return dr, dd, loss

        out = [run(lambda dr, dd, loss: dcg.dcg_loss(ctx, r, d, t, td, cams, 0.0, 0.1, dr, dd, loss)),
               run(lambda dr, dd, loss: dcg.dcg_loss_l1(ctx, r, d, t, td, cams, 0.1, dr, dd, loss))]
        assert all(torch.equal(a, b) for a, b in zip(*out))
        with pytest.raises(dcg.DcgError) as e:
            dcg.dcg_loss(ctx, r, d, t, td, cams, 1.5, 0.1, out[0][0], out[0][1], out[0][2])
        assert e.value.status == 1
    finally:
        dcg.dcg_destroy(ctx)
