"""Host-side faults of the chunk tier and load verification.

Each injected fault (a chunk load that fails before its copies are issued, a
load whose last page arrives only half copied, a budget failure) makes the
call that meets it return its status; the context stays usable, and the
repeated call renders exactly what a context that never saw the fault
renders.  With load verification on and no fault, nothing changes."""
import os

import numpy as np
import pytest

from paper_2511_23030_b300 import dcg, synth

from gpu_util import make_ctx, out_buffers, planar

pytestmark = pytest.mark.gpu

N = 64_000


@pytest.fixture(scope="module")
def scene():
    return synth.window_scene(0, n=N, deg=1)


def _ctx(sc, flags=0):
    ctx = make_ctx(deg=1, n_max=N, views=1, pixels=320 * 240, chunk=sc["chunk_size"], budget=40_000, host=N,
                   page=256, dfar=60.0, flags=flags)
    dcg.dcg_chunk_table_update(ctx, planar(sc["params"]), N)
    return ctx


def _cams(sc, k=0):
    """A 320 x 240 view from keyframe k's pose with three times its focal length
    (it sees 22-28 of the 64 chunks; views 0 and 6 together hold 42k Gaussians,
    more than the 40k budget)."""
    c = sc["cams"][k]
    s = 3 * 320.0 / c.W
    return [synth.Camera(c.fx * s, c.fy * s, 160.0, 120.0, 320, 240, c.Tcw, c.znear, c.zfar)]


def _step(ctx, cams):
    """cull, gather, render forward; the image on the host."""
    lst = dcg.dcg_cull_chunks(ctx, cams)
    g, n = dcg.dcg_gather_active(ctx, lst)
    rgb, depth = out_buffers(cams)
    dcg.dcg_render_fwd(ctx, g, n, cams, rgb, depth)
    dcg.dcg_sync(ctx)
    return rgb.cpu().numpy(), depth.cpu().numpy(), n


@pytest.fixture(scope="module")
def reference(scene):
    ctx = _ctx(scene)
    try:
        return _step(ctx, _cams(scene))
    finally:
        dcg.dcg_destroy(ctx)


@pytest.mark.parametrize("kind,status,skip", [("h2d_fail", 8, 0), ("short_copy", 8, 0), ("short_copy", 8, 3),
                                              ("budget", 4, 0)])
def test_injected_fault_returns_status_and_the_retry_matches(scene, reference, kind, status, skip):
    ctx = _ctx(scene)
    try:
        cams = _cams(scene)
        dcg.dcg_inject_fault(ctx, kind, skip)
        with pytest.raises(dcg.DcgError) as e:
            _step(ctx, cams)
        assert e.value.status == status, str(e.value)
        rgb, depth, n = _step(ctx, cams)  # the context is still usable; the fault fired once
        assert n == reference[2]
        assert np.array_equal(rgb, reference[0]) and np.array_equal(depth, reference[1])
        info = dcg.dcg_chunk_info(ctx)
        assert info["counts"][info["resident"] > 0].sum() <= 40_000
    finally:
        dcg.dcg_destroy(ctx)


def test_fault_armed_from_the_environment(scene, reference, monkeypatch):
    monkeypatch.setenv("DCG_FAULT", "budget")
    ctx = _ctx(scene)
    monkeypatch.delenv("DCG_FAULT")
    try:
        with pytest.raises(dcg.DcgError) as e:
            _step(ctx, _cams(scene))
        assert e.value.status == 4
        rgb, depth, _ = _step(ctx, _cams(scene))
        assert np.array_equal(rgb, reference[0]) and np.array_equal(depth, reference[1])
    finally:
        dcg.dcg_destroy(ctx)


def test_verified_loads_change_nothing_without_a_fault(scene, reference):
    ctx = _ctx(scene, flags=dcg.FLAG_VERIFY_LOADS)
    try:
        cams = _cams(scene)
        rgb, depth, n = _step(ctx, cams)
        assert np.array_equal(rgb, reference[0]) and np.array_equal(depth, reference[1])
        # another view that evicts (dirty chunks written back) and loads, then the first again
        g, na = dcg.dcg_gather_active(ctx, dcg.dcg_cull_chunks(ctx, _cams(scene, 6)))
        dcg.dcg_scatter_back(ctx, g, na)
        dcg.dcg_flush(ctx)
        st0 = dcg.dcg_tier_stats(ctx)
        rgb2, depth2, _ = _step(ctx, cams)
        st1 = dcg.dcg_tier_stats(ctx)
        assert st0["evictions"] > 0 and st1["loads"] > st0["loads"]  # the second view forced evictions and reloads
        assert np.array_equal(rgb2, reference[0]) and np.array_equal(depth2, reference[1])
    finally:
        dcg.dcg_destroy(ctx)
