"""Chunk path on the GPU against the oracle: Eq. 5/6 ids bit-exact, cull masks
bit-exact, gather order, gather/scatter round trip, LRU residency."""
import numpy as np
import pytest

from paper_2511_23030_b300 import dcg, synth

from gpu_util import make_ctx, planar

pytestmark = pytest.mark.gpu


def _keys_gpu(ctx, means):
    import torch

    m = torch.from_numpy(np.ascontiguousarray(means, np.float32)).cuda()
    k = torch.zeros(means.shape[0], dtype=torch.int64, device="cuda")
    dcg.dcg_chunk_keys(ctx, m, k)
    return k


def test_chunk_keys_bit_exact(orc):
    ctx = make_ctx(deg=0, n_max=1000, chunk=8.0)
    try:
        rng = np.random.default_rng(0)
        p = rng.uniform(-2e4, 2e4, (200_000, 3)).astype(np.float32)
        p[:5000, 0] = (rng.integers(-500, 500, 5000) * 8.0 + 4.0).astype(np.float32)  # exact boundaries
        p[5000:6000, 1] = np.float32(-4.0)
        p[6000:7000] = np.nextafter(np.float32(-4.0), np.float32(-10.0))
        p[7000] = (0.0, -0.0, 0.0)
        k = _keys_gpu(ctx, p)
        dcg.dcg_sync(ctx)
        _, ok, bad = orc.chunk_keys(p, 8.0)
        assert not bad.any()
        assert np.array_equal(k.cpu().numpy().view(np.uint64), ok)
        # golden ids with s = 10
        ctx2 = make_ctx(deg=0, n_max=1000, chunk=10.0)
        g = np.array([[0, 0, 0], [5, 0, 0], [-5, 0, 0], [-5.0000005, 0, 0]], np.float32)
        kk = _keys_gpu(ctx2, g).cpu().numpy().view(np.uint64)
        dcg.dcg_sync(ctx2)
        assert list(kk) == [4611688217451692032, 4611692615498203136, 4611688217451692032, 4611683819405180928]
        # out of range / NaN -> DCG_ERR_KEY_RANGE at sync, key 0
        bad_p = np.array([[1e9, 0, 0], [np.nan, 0, 0], [1, 2, 3]], np.float32)
        kb = _keys_gpu(ctx2, bad_p)
        with pytest.raises(dcg.DcgError) as e:
            dcg.dcg_sync(ctx2)
        assert e.value.status == 5
        assert list(kb.cpu().numpy()[:2]) == [0, 0]
        dcg.dcg_sync(ctx2)  # cleared
        dcg.dcg_destroy(ctx2)
    finally:
        dcg.dcg_destroy(ctx)


def _window_table(n=64_000, deg=1, budget=None, page=512):
    sc = synth.window_scene(0, n=n, deg=deg)
    ctx = make_ctx(deg=deg, n_max=n, chunk=sc["chunk_size"], budget=budget, host=n, page=page, dfar=60.0)
    g = planar(sc["params"])
    dcg.dcg_chunk_table_update(ctx, g, n)
    return ctx, sc


def test_table_update_groups_and_round_trips(orc):
    ctx, sc = _window_table()
    try:
        P = sc["params"]
        info = dcg.dcg_chunk_info(ctx)
        coords, keys, _ = orc.chunk_keys(P[:, :3], sc["chunk_size"])
        uk, cnt = np.unique(keys, return_counts=True)
        assert np.array_equal(info["keys"], uk) and np.array_equal(info["counts"], cnt)
        assert len(uk) == 64
        for c in (0, 17, 63):
            got = dcg.dcg_chunk_read(ctx, c, int(info["counts"][c]), P.shape[1])
            want = P[keys == info["keys"][c]]  # stored order = input order within the chunk
            assert np.array_equal(got.T, want)
    finally:
        dcg.dcg_destroy(ctx)


def test_cull_bit_exact_flat_and_hierarchical(orc):
    import torch

    ctx, sc = _window_table()
    try:
        info = dcg.dcg_chunk_info(ctx)
        C = len(info["keys"])
        rng = np.random.default_rng(1)
        cams = list(sc["cams"])
        for _ in range(12):  # extra random poses, some inside the volume
            eye = rng.uniform(-10, 14, 3)
            cams.append(synth.Camera(300.0, 300.0, 320.0, 240.0, 640, 480,
                                     synth.look_at(eye, eye + rng.normal(0, 1, 3)), 0.2, float(rng.uniform(5, 40))))
        for k0 in range(0, len(cams), 8):
            cs = cams[k0:k0 + 8]
            mask = torch.zeros(len(cs) * C, dtype=torch.uint8, device="cuda")
            lst = dcg.dcg_cull_chunks(ctx, cs, mask)
            m = mask.view(len(cs), C).cpu().numpy()
            for v, cam in enumerate(cs):
                flat = orc.cull(info["coords"], sc["chunk_size"], cam, 60.0)
                hier = orc.cull(info["coords"], sc["chunk_size"], cam, 60.0, hierarchical=True)
                assert np.array_equal(m[v], flat) and np.array_equal(flat, hier)
            assert np.array_equal(lst, np.nonzero(m.any(0))[0])
    finally:
        dcg.dcg_destroy(ctx)


def test_gather_order_and_scatter_round_trip(orc):
    import torch

    ctx, sc = _window_table()
    try:
        P = sc["params"]
        info = dcg.dcg_chunk_info(ctx)
        lst = dcg.dcg_cull_chunks(ctx, sc["cams"][:3])
        g, n = dcg.dcg_gather_active(ctx, lst)
        vis = np.zeros(len(info["keys"]), bool)
        vis[lst] = True
        order, n_ref = orc.gather_order(info["keys"], info["counts"], vis)
        assert n == n_ref
        F = P.shape[1]
        _, keys, _ = orc.chunk_keys(P[:, :3], sc["chunk_size"])
        want = np.concatenate([P[keys == info["keys"][c]] for c, _ in order])
        act_np = _read_active(g, n, F)
        assert np.array_equal(act_np, want)
        # modify, scatter back, flush, read from the host tier
        mod = torch.from_numpy(np.ascontiguousarray((want * 2 + 1).T)).cuda()
        g2 = dcg.gaussians(mod, 1)
        dcg.dcg_scatter_back(ctx, g2, n)
        dcg.dcg_flush(ctx)
        for c, _ in order[:5]:
            got = dcg.dcg_chunk_read(ctx, c, int(info["counts"][c]), F)
            assert np.array_equal(got.T, P[keys == info["keys"][c]] * 2 + 1)
    finally:
        dcg.dcg_destroy(ctx)


def test_active_map_names_each_active_row():
    """dcg_active_map: every active row's chunk and row within the chunk, checked against the chunk
    contents (bit-exact) and the gather order (listed chunks ascending, stored order within)."""
    import torch

    ctx, sc = _window_table()
    try:
        with pytest.raises(dcg.DcgError) as e:  # nothing gathered yet
            dcg.dcg_active_map(ctx, torch.zeros(1, dtype=torch.int32, device="cuda"))
        assert e.value.status == 9
        F = sc["params"].shape[1]
        info = dcg.dcg_chunk_info(ctx)
        lst = dcg.dcg_cull_chunks(ctx, sc["cams"][2:5])
        g, n = dcg.dcg_gather_active(ctx, lst)
        chunk = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        row = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        dcg.dcg_active_map(ctx, chunk, row)
        dcg.dcg_sync(ctx)
        chunk, row = chunk.cpu().numpy(), row.cpu().numpy()
        want_chunk = np.concatenate([np.full(int(info["counts"][c]), c) for c in lst])
        want_row = np.concatenate([np.arange(int(info["counts"][c])) for c in lst])
        assert np.array_equal(chunk, want_chunk) and np.array_equal(row, want_row)
        act = _read_active(g, n, F)
        for c in lst[:: max(1, len(lst) // 6)]:
            stored = dcg.dcg_chunk_read(ctx, int(c), int(info["counts"][c]), F).T
            sel = chunk == c
            assert np.array_equal(act[sel], stored[row[sel]])
        only_rows = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        dcg.dcg_active_map(ctx, None, only_rows)  # either output may be omitted
        dcg.dcg_sync(ctx)
        assert np.array_equal(only_rows.cpu().numpy(), want_row)
    finally:
        dcg.dcg_destroy(ctx)


def test_active_map_after_table_update_and_on_the_reuse_path():
    """The map keeps the gather-time rows when a table update afterwards grows a
    gathered chunk and adds a chunk with a lower id (which renumbers the table):
    chunk_out names the chunks by their new table index, with the counts they had
    when gathered.  A repeat gather of the same list after scatter_back (the
    library's buffer handed out again without a copy) gives the same map."""
    import torch

    ctx, sc = _window_table()
    try:
        P = sc["params"]
        F = P.shape[1]
        info0 = dcg.dcg_chunk_info(ctx)
        lst = dcg.dcg_cull_chunks(ctx, sc["cams"][2:5])
        g, n = dcg.dcg_gather_active(ctx, lst)
        keys0 = info0["keys"][lst]
        counts0 = info0["counts"][lst]
        # grow the first listed chunk by 100 copies of its own Gaussians, and add 50
        # Gaussians in a chunk below every existing one (x coordinate -6 chunks)
        first = dcg.dcg_chunk_read(ctx, int(lst[0]), int(counts0[0]), F).T[:100].copy()
        low = first[:50].copy()
        low[:, 0] = -6.0 * sc["chunk_size"]
        dcg.dcg_chunk_table_update(ctx, planar(np.concatenate([first, low]).astype(np.float32)), 150)
        info1 = dcg.dcg_chunk_info(ctx)
        assert len(info1["keys"]) == len(info0["keys"]) + 1 and info1["keys"][0] < info0["keys"][0]
        new_idx = np.searchsorted(info1["keys"], keys0)
        assert np.array_equal(info1["keys"][new_idx], keys0) and np.array_equal(new_idx, lst + 1)
        assert info1["counts"][new_idx[0]] == counts0[0] + 100
        chunk = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        row = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        dcg.dcg_active_map(ctx, chunk, row)
        dcg.dcg_sync(ctx)
        want_chunk = np.concatenate([np.full(int(c), k) for k, c in zip(new_idx, counts0)])
        want_row = np.concatenate([np.arange(int(c)) for c in counts0])
        assert np.array_equal(chunk.cpu().numpy(), want_chunk) and np.array_equal(row.cpu().numpy(), want_row)
    finally:
        dcg.dcg_destroy(ctx)
    ctx, sc = _window_table()
    try:
        info = dcg.dcg_chunk_info(ctx)
        lst = dcg.dcg_cull_chunks(ctx, sc["cams"][1:3])
        g, n = dcg.dcg_gather_active(ctx, lst)
        dcg.dcg_scatter_back(ctx, g, n)  # the library's own buffer: write-back deferred
        g2, n2 = dcg.dcg_gather_active(ctx, lst)  # the same list: handed out again without a copy
        assert n2 == n and g2.data == g.data
        chunk = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        row = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        dcg.dcg_active_map(ctx, chunk, row)
        dcg.dcg_sync(ctx)
        want_chunk = np.concatenate([np.full(int(info["counts"][c]), c) for c in lst])
        want_row = np.concatenate([np.arange(int(info["counts"][c])) for c in lst])
        assert np.array_equal(chunk.cpu().numpy(), want_chunk) and np.array_equal(row.cpu().numpy(), want_row)
    finally:
        dcg.dcg_destroy(ctx)


def _read_active(g, n, F):
    """Copy of the library-owned active buffer (planar, stride g.stride) as numpy [n, F]."""
    return dcg.active_tensor(g, n, F).T.cpu().numpy()


def test_lru_eviction_follows_oracle(orc):
    """Budget of ~40% of the scene; a sequence of views; residency after every
    gather equals the oracle's LRU simulation; evicted dirty chunks are saved."""
    import torch

    n = 64_000
    ctx, sc = _window_table(n=n, budget=26_000, page=256)
    try:
        info = dcg.dcg_chunk_info(ctx)
        C = len(info["keys"])
        counts = info["counts"]
        resident = np.zeros(C, bool)
        last = np.full(C, -1)
        step = 0
        rng = np.random.default_rng(2)
        for it in range(14):
            eye = rng.uniform(-6, 10, 3)
            cam = synth.Camera(120.0, 120.0, 160.0, 120.0, 320, 240, synth.look_at(eye, eye + rng.normal(0, 1, 3)),
                               0.2, 8.0)
            lst = dcg.dcg_cull_chunks(ctx, [cam])
            if counts[lst].sum() > 26_000 or len(lst) == 0:
                continue
            vis = np.zeros(C, bool)
            vis[lst] = True
            step += 1
            deficit = counts[resident].sum() + counts[vis & ~resident].sum() - 26_000
            sel = orc.lru_select(resident, vis, last, info["keys"], counts, deficit)
            assert sel is not None
            resident[sel] = False
            resident[vis] = True
            last[vis] = step
            g, nact = dcg.dcg_gather_active(ctx, lst)
            # write back +1 to make the chunks dirty
            F = synth.n_fields(1)
            cur = torch.from_numpy(np.ascontiguousarray(_read_active(g, nact, F).T + 1)).cuda()
            dcg.dcg_scatter_back(ctx, dcg.gaussians(cur, 1), nact)
            got = dcg.dcg_chunk_info(ctx)
            assert np.array_equal(got["resident"].astype(bool), resident), it
            assert got["counts"][resident].sum() <= 26_000
        assert step >= 5
        dcg.dcg_flush(ctx)
    finally:
        dcg.dcg_destroy(ctx)


def test_budget_error_when_visible_exceeds_budget():
    ctx, sc = _window_table(n=64_000, budget=10_000, page=256)
    try:
        lst = np.arange(dcg.dcg_chunk_count(ctx), dtype=np.int32)
        with pytest.raises(dcg.DcgError) as e:
            dcg.dcg_gather_active(ctx, lst)
        assert e.value.status == 4
    finally:
        dcg.dcg_destroy(ctx)


def test_deferred_write_back_of_the_active_set(orc):
    """scatter_back of the library's own active buffer defers the copy into the
    chunk pages: the same list is handed out again as is, and the deferred copy
    lands before an eviction or a flush saves the chunks."""
    probe, _ = _window_table()
    info = dcg.dcg_chunk_info(probe)
    dcg.dcg_destroy(probe)
    counts = info["counts"]
    A, B = np.arange(0, 10, dtype=np.int32), np.arange(30, 46, dtype=np.int32)
    assert counts[B].sum() >= counts[A].sum()
    budget = int(counts[B].sum()) + 1  # gathering B evicts every other chunk
    ctx, sc = _window_table(budget=budget, page=256)
    try:
        P = sc["params"]
        F = P.shape[1]
        _, keys, _ = orc.chunk_keys(P[:, :3], sc["chunk_size"])

        def rows(lst):
            return np.concatenate([P[keys == info["keys"][c]] for c in lst])

        g, n = dcg.dcg_gather_active(ctx, A)
        dcg.active_tensor(g, n, F).mul_(3.0)
        g, n = dcg.dcg_gather_active(ctx, A)  # no scatter_back in between: copied again
        assert np.array_equal(_read_active(g, n, F), rows(A))
        dcg.active_tensor(g, n, F).mul_(2.0)
        dcg.dcg_scatter_back(ctx, g, n)
        before = dcg.dcg_tier_stats(ctx)
        g2, n2 = dcg.dcg_gather_active(ctx, A)  # handed out as is
        assert (g2.data, n2) == (g.data, n) and dcg.dcg_tier_stats(ctx) == before
        want = rows(A) * np.float32(2.0)
        assert np.array_equal(_read_active(g, n, F), want)
        dcg.active_tensor(g, n, F).add_(1.0)
        dcg.dcg_scatter_back(ctx, g, n)
        want = want + np.float32(1.0)
        g, n = dcg.dcg_gather_active(ctx, B)  # write-back, then A is evicted to the host tier
        assert not dcg.dcg_chunk_info(ctx)["resident"][A].any()
        assert np.array_equal(_read_active(g, n, F), rows(B))
        g, n = dcg.dcg_gather_active(ctx, A)  # reloaded from the host tier
        assert np.array_equal(_read_active(g, n, F), want)
        dcg.active_tensor(g, n, F).add_(1.0)
        dcg.dcg_scatter_back(ctx, g, n)
        want = want + np.float32(1.0)
        dcg.dcg_flush(ctx)
        off = 0
        for c in A:
            cnt = int(counts[c])
            assert np.array_equal(dcg.dcg_chunk_read(ctx, int(c), cnt, F).T, want[off: off + cnt])
            off += cnt
    finally:
        dcg.dcg_destroy(ctx)
