"""The allocation-free cull (dcg_cull_chunks_noalloc) gives the same mask,
list and count as dcg_cull_chunks, on two calls in a row.

It is for callers that cannot allocate device memory (their memory is owned
by their own allocator, or planned against a fixed budget): its scratch is a
fixed device array, so this test also checks that a second call, which finds
the first call's flags still in that array, is not affected by them.  The
file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

from paper_2511_23030_b300 import dcg, synth

from gpu_util import make_ctx, planar

pytestmark = pytest.mark.gpu


def test_noalloc_cull_matches_context_cull_twice():
    import torch

    sc = synth.window_scene(0, n=64_000, deg=1)
    ctx = make_ctx(deg=1, n_max=64_000, chunk=sc["chunk_size"], dfar=60.0, page=512)
    try:
        dcg.dcg_chunk_table_update(ctx, planar(sc["params"]), 64_000)
        info = dcg.dcg_chunk_info(ctx)
        C = len(info["keys"])
        coords = torch.from_numpy(np.ascontiguousarray(info["coords"])).cuda()
        rng = np.random.default_rng(11)
        # first call: the window's eight keyframes; second call: fewer views that
        # see fewer chunks, so stale flags of the first call would show up
        eye = np.array([2.0, 2.0, 30.0])
        narrow = [synth.Camera(1000.0, 1000.0, 160.0, 120.0, 320, 240, synth.look_at(eye, eye + rng.normal(0, 0.3, 3)
                                                                                   + np.array([0, 0, -1.0])),
                               0.2, 40.0) for _ in range(2)]
        for cams in (sc["cams"], narrow):
            V = len(cams)
            mask_ref = torch.zeros(V * C, dtype=torch.uint8, device="cuda")
            lst_ref = dcg.dcg_cull_chunks(ctx, cams, mask_ref)
            mask = torch.full((V * C,), 7, dtype=torch.uint8, device="cuda")
            lst = torch.full((C,), -1, dtype=torch.int32, device="cuda")
            n = torch.full((1,), -1, dtype=torch.int32, device="cuda")
            dcg.dcg_cull_chunks_noalloc(coords, sc["chunk_size"], 60.0, cams, mask, lst, n)
            torch.cuda.synchronize()
            assert torch.equal(mask, mask_ref)
            k = int(n.item())
            assert k == len(lst_ref)
            assert np.array_equal(lst[:k].cpu().numpy(), lst_ref)
        assert 0 < k < C
    finally:
        dcg.dcg_destroy(ctx)


def test_noalloc_cull_rejects_oversized_requests():
    import torch

    c = synth.Camera(100.0, 100.0, 64.0, 48.0, 128, 96, np.eye(4, dtype=np.float32), 0.2, 10.0)
    coords = torch.zeros(((1 << 20) + 1, 3), dtype=torch.int32, device="cuda")
    lst = torch.zeros(1, dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(dcg.DcgError) as e:
        dcg.dcg_cull_chunks_noalloc(coords, 4.0, 10.0, [c], None, lst, n)
    assert e.value.status == 6
    with pytest.raises(dcg.DcgError) as e:
        dcg.dcg_cull_chunks_noalloc(coords[:4], 4.0, 10.0, [c] * 17, None, lst, n)
    assert e.value.status == 6


def test_noalloc_cull_cameras_in_pinned_memory_may_be_reused_at_once():
    """The cameras are taken at the call, also from page-locked memory: the
    caller overwrites them right after the call, while the stream is still
    held back by a sleeping kernel, and the cull still sees the originals."""
    import ctypes

    import torch

    sc = synth.window_scene(0, n=64_000, deg=1)
    ctx = make_ctx(deg=1, n_max=64_000, chunk=sc["chunk_size"], dfar=60.0, page=512)
    try:
        dcg.dcg_chunk_table_update(ctx, planar(sc["params"]), 64_000)
        info = dcg.dcg_chunk_info(ctx)
        C = len(info["keys"])
        coords = torch.from_numpy(np.ascontiguousarray(info["coords"])).cuda()
        cams = sc["cams"][:4]
        V = len(cams)
        mask_ref = torch.zeros(V * C, dtype=torch.uint8, device="cuda")
        lst_ref = dcg.dcg_cull_chunks(ctx, cams, mask_ref)
        nbytes = ctypes.sizeof(dcg.dcg_camera) * V
        pinned = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
        ctypes.memmove(pinned.data_ptr(), dcg.make_cameras(cams), nbytes)
        away = [synth.Camera(c.fx, c.fy, c.cx, c.cy, c.W, c.H, synth.look_at([0, 0, 500.0], [0, 0, 600.0]), 0.2, 1.0)
                for c in cams]
        mask = torch.zeros(V * C, dtype=torch.uint8, device="cuda")
        lst = torch.full((C,), -1, dtype=torch.int32, device="cuda")
        n = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        stream = torch.cuda.current_stream()
        torch.cuda._sleep(20_000_000)  # about 10 ms of GPU time ahead of the cull on this stream
        st = dcg.lib().dcg_cull_chunks_noalloc(dcg.ptr(coords), C, float(sc["chunk_size"]), 60.0,
                                               ctypes.cast(pinned.data_ptr(), ctypes.POINTER(dcg.dcg_camera)), V,
                                               dcg.ptr(mask), dcg.ptr(lst), dcg.ptr(n), dcg.stream_ptr(stream))
        assert st == dcg.DCG_OK
        ctypes.memmove(pinned.data_ptr(), dcg.make_cameras(away), nbytes)  # the caller reuses its array
        torch.cuda.synchronize()
        assert torch.equal(mask, mask_ref)
        k = int(n.item())
        assert k == len(lst_ref) > 0 and np.array_equal(lst[:k].cpu().numpy(), lst_ref)
    finally:
        dcg.dcg_destroy(ctx)
