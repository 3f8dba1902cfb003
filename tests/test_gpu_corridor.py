"""Out-of-core mapping along a driving corridor (Sec. III-E: visible chunks
are loaded under a Gaussian budget, old ones evicted to the slower tier with
LRU).  Invariants: resident Gaussians never exceed the budget (the VRAM
plateau of Fig. 5), every step renders exactly what an unlimited budget
renders, and after a final flush the host tier holds exactly what the
unlimited run holds (eviction loses nothing)."""
import numpy as np
import pytest

from paper_2511_23030_b300 import dcg, synth

from gpu_util import make_ctx, planar

pytestmark = pytest.mark.gpu


def _corridor(length=400.0, per_m=1500):
    xy, head = synth.corridor_path(0, length)
    rng = np.random.default_rng(5)
    P = synth.corridor_gaussians(rng, xy, head, per_m, deg=1)
    cams = synth.corridor_cameras(xy, head, W=620, H=188, every=2)
    for c in cams:
        c.zfar = 40.0
    return P, cams


def _run(P, cams, budget, steps):
    import torch

    n, F = P.shape
    ctx = make_ctx(deg=1, n_max=n, views=1, pixels=620 * 188, chunk=8.0, budget=budget, host=n, page=512, dfar=40.0)
    imgs, resident_max = [], 0
    try:
        dcg.dcg_chunk_table_update(ctx, planar(P), n)
        rgb = torch.zeros(3 * 620 * 188, device="cuda")
        depth = torch.zeros(620 * 188, device="cuda")
        for t in steps:
            cam = cams[t]
            lst = dcg.dcg_cull_chunks(ctx, [cam])
            g, na = dcg.dcg_gather_active(ctx, lst)
            dcg.dcg_render_fwd(ctx, g, na, [cam], rgb, depth)
            act = dcg.active_tensor(g, na, F)
            act[0:3] += 1e-3 * (t % 7)  # a deterministic "update" of the active set
            dcg.dcg_scatter_back(ctx, g, na)
            st = dcg.dcg_tier_stats(ctx)
            resident_max = max(resident_max, st["resident"])
            imgs.append(rgb.clone())
        dcg.dcg_flush(ctx)
        dcg.dcg_sync(ctx)
        info = dcg.dcg_chunk_info(ctx)
        tier = [dcg.dcg_chunk_read(ctx, c, int(info["counts"][c]), F) for c in range(len(info["keys"]))]
        return imgs, resident_max, dcg.dcg_tier_stats(ctx), info, tier
    finally:
        dcg.dcg_destroy(ctx)


def test_corridor_budget_and_lossless_eviction():
    import torch

    P, cams = _corridor()
    n = P.shape[0]
    steps = list(range(0, len(cams), 3))
    budget = n // 4
    imgs_b, res_max, stats_b, info_b, tier_b = _run(P, cams, budget, steps)
    imgs_u, _, stats_u, info_u, tier_u = _run(P, cams, n, steps)
    assert res_max <= budget
    # the road is driven forward only: evicted chunks are not needed again
    assert stats_b["evictions"] > 10 and stats_b["loads"] >= stats_u["loads"]
    assert stats_u["evictions"] == 0
    assert np.array_equal(info_b["keys"], info_u["keys"])
    for a, b in zip(imgs_b, imgs_u):
        assert torch.equal(a, b)
    for a, b in zip(tier_b, tier_u):
        assert np.array_equal(a, b)
    assert sum(float(np.abs(im.cpu().numpy()).sum() > 0) for im in imgs_b) > 0.9 * len(imgs_b)
