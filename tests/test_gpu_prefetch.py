"""Learned chunk prefetch: the MLP is trained with the library's own kernels
on samples the mapper generates from a drive (exact cull labels, seed 1),
then drives asynchronous prefetching on another drive (seed 0).  The exact
cull still decides every active set, so the rendered images are identical
with and without prefetching; the trained network hides most chunk loads."""
import numpy as np
import pytest

from paper_2511_23030_b300 import dcg, prefetch, synth

from gpu_util import make_ctx, planar

pytestmark = pytest.mark.gpu

ZFAR = 60.0


def _drive(seed, length, per_m, W=320, H=96):
    xy, head = synth.corridor_path(seed, length)
    P = synth.corridor_gaussians(np.random.default_rng(seed + 5), xy, head, per_m, deg=0)
    cams = synth.corridor_cameras(xy, head, W=W, H=H, every=1)
    for c in cams:
        c.zfar = ZFAR
    return P, cams


def _ctx(P, budget):
    n = P.shape[0]
    c = make_ctx(deg=0, n_max=n, views=1, pixels=320 * 96, chunk=8.0, budget=budget, host=n, page=256, dfar=ZFAR)
    dcg.dcg_chunk_table_update(c, planar(P), n)
    return c


def test_prefetch_hides_loads_and_never_changes_images():
    import torch

    P_tr, cams_tr = _drive(1, 700.0, 40)
    ctx_tr = _ctx(P_tr, P_tr.shape[0])
    pm = prefetch.PrefetchMLP(max_batch=2048)
    try:
        X, y, n, pos = prefetch.make_dataset(ctx_tr, cams_tr, 8.0, 1.5 * ZFAR, max_samples=40_000)
        assert n > 20_000 and 0.05 < pos < 0.95

        dcg.dcg_mlp_set_params(pm.m, synth.mlp_init_params(0))
        losses = prefetch.train(pm, X, y, n, epochs=5, batch=1024, lr=1e-3)
        assert losses[-1] < 0.7 * losses[0], losses
        dcg.dcg_destroy(ctx_tr)
        ctx_tr = None

        P, cams = _drive(0, 260.0, 600)
        budget = P.shape[0] // 3
        results, images = {}, {}
        for mode in ("none", "cv", "mlp"):
            ctx = _ctx(P, budget)
            pm.bind(ctx)
            rgb = torch.zeros(3 * 320 * 96, device="cuda")
            depth = torch.zeros(320 * 96, device="cuda")
            shots = []

            def render(g, na, cam):
                dcg.dcg_render_fwd(ctx, g, na, [cam], rgb, depth)
                shots.append(rgb.clone())

            try:
                results[mode] = prefetch.run_corridor(ctx, cams, mode, 8.0, 1.5 * ZFAR, pm=pm, render=render)
                images[mode] = shots
                # the device never holds more than the budget, at any step of the drive
                assert results[mode]["resident_max"] <= budget and dcg.dcg_tier_stats(ctx)["resident"] <= budget
            finally:
                dcg.dcg_destroy(ctx)
        for mode in ("cv", "mlp"):
            assert all(torch.equal(a, b) for a, b in zip(images["none"], images[mode]))
        summary = {m: {k: results[m][k] for k in ("hits", "misses", "wasted_prefetches", "hidden_load_frac",
                                                    "stall_ms")} for m in results}
        print(summary)
        assert results["none"]["hits"] == 0 and results["none"]["misses"] > 20, summary
        assert results["mlp"]["hidden_load_frac"] >= 0.8, summary
        assert results["mlp"]["stall_ms"] < 0.5 * results["none"]["stall_ms"], summary
        # the learned predictor against the constant-velocity one, both proposing on the side stream
        # with the same period: both hide most loads; which hides more is reported, not assumed
        assert results["cv"]["hidden_load_frac"] >= 0.8, summary
        print("mlp vs cv: hits %d vs %d, misses %d vs %d, stall %.3f vs %.3f ms" % (
            results["mlp"]["hits"], results["cv"]["hits"], results["mlp"]["misses"], results["cv"]["misses"],
            results["mlp"]["stall_ms"], results["cv"]["stall_ms"]))
    finally:
        pm.close()
        if ctx_tr is not None:
            dcg.dcg_destroy(ctx_tr)
