"""Loop-closure correction and chunk redistribution on the GPU against the
reference: the same Gaussians move, to the same chunks, in the same order,
with their optimizer moments."""
import numpy as np
import pytest

from oracle import loopclosure as lc
from paper_2511_23030_b300 import dcg, synth

from gpu_util import make_ctx, planar

pytestmark = pytest.mark.gpu

N = 64_000
QUAT = [6, 7, 8, 9]


def _rot(axis, deg):
    a = np.deg2rad(deg)
    c, s = np.cos(a), np.sin(a)
    R = {"x": [[1, 0, 0], [0, c, -s], [0, s, c]], "z": [[c, -s, 0], [s, c, 0], [0, 0, 1]]}[axis]
    return np.asarray(R)


def _corr(axis, deg, t):
    C = np.eye(4)
    C[:3, :3] = _rot(axis, deg)
    C[:3, 3] = t
    return C.astype(np.float32)


def _setup(budget=None):
    import torch

    sc = synth.window_scene(0, n=N, deg=1)
    ctx = make_ctx(deg=1, n_max=N, chunk=sc["chunk_size"], budget=budget, host=N, page=512, dfar=60.0, moments=1)
    dcg.dcg_chunk_table_update(ctx, planar(sc["params"]), N)
    F = sc["params"].shape[1]
    # give the moments non-zero values: one Adam step with gradient sin(3 p), elementwise, so
    # gathering the chunks in groups that fit the budget gives every context the same map
    info = dcg.dcg_chunk_info(ctx)
    cap = N if budget is None else budget
    groups, cur, tot = [], [], 0
    for c, cnt in enumerate(info["counts"]):
        if tot + cnt > cap:
            groups.append(cur)
            cur, tot = [], 0
        cur.append(c)
        tot += int(cnt)
    groups.append(cur)
    for grp in groups:
        g, n = dcg.dcg_gather_active(ctx, np.asarray(grp, np.int32))
        grad = torch.sin(3.0 * dcg.active_tensor(g, n, F)).contiguous()
        dcg.dcg_adam_step(ctx, g, dcg.gaussians(grad, 1), n, np.full(F, 1e-3, np.float32), step=1)
        dcg.dcg_scatter_back(ctx, g, n)
    dcg.dcg_flush(ctx)
    return ctx, sc, F


def _read_all(ctx, F):
    info = dcg.dcg_chunk_info(ctx)
    out = {}
    for c, k in enumerate(info["keys"]):
        cnt = int(info["counts"][c])
        p = dcg.dcg_chunk_read(ctx, c, cnt, F)
        m, v = dcg.dcg_chunk_read_moments(ctx, c, cnt, F)
        out[int(k)] = np.concatenate([p, m, v]).T.copy()
    return out


def _same(after, want):
    assert sorted(after) == sorted(want)
    for k in want:
        a, w = after[k], want[k]
        assert a.shape == w.shape, k
        cols = [c for c in range(a.shape[1]) if c not in QUAT]
        assert np.array_equal(a[:, cols], w[:, cols]), k
        qa, qw = a[:, QUAT].astype(np.float64), w[:, QUAT].astype(np.float64)
        err = np.minimum(np.abs(qa - qw).max(1), np.abs(qa + qw).max(1))  # q and -q are one rotation
        assert (err <= 2e-6 * np.abs(qw).max(1) + 1e-30).all(), k


# (keyframes, corrections): two keyframes whose frusta gather every chunk (moved rows go to gathered
# chunks and to new ones); one keyframe gathering 48 of the 64 chunks, shifted 4 m (moved rows also go
# to 13 existing chunks outside the union, which are written back and appended to)
SCENARIOS = {
    "two_keyframes": ([0, 3], [("z", 2.0, (0.8, -0.4, 0.3)), ("x", 1.5, (-0.6, 0.5, 0.2))]),
    "partial_union": ([3], [("z", 3.0, (0.0, 0.0, 4.0))]),
}


@pytest.mark.parametrize("scenario", list(SCENARIOS))
def test_loop_closure_matches_reference(scenario):
    ctx, sc, F = _setup()
    try:
        kf_ids, cs = SCENARIOS[scenario]
        kfs = [sc["cams"][k] for k in kf_ids]
        corrs = [_corr(*c) for c in cs]
        before = _read_all(ctx, F)
        dcg.dcg_profile(ctx, True)
        nt, nm = dcg.dcg_loop_closure(ctx, kfs, corrs)
        prof = dcg.dcg_profile_read(ctx)
        dcg.dcg_profile(ctx, False)
        # device intervals: cull, transform + keys, moved rows, destinations, permutation, page writes
        # (the batch load of the union is timed as a gather)
        assert prof["loop_closure"][1] == 6 and prof["loop_closure"][0] > 0
        dcg.dcg_flush(ctx)
        after = _read_all(ctx, F)
        want, wt, wm = lc.loop_closure(before, sc["chunk_size"], 60.0, kfs, corrs)
        assert (nt, nm) == (wt, wm) and nt > 1000 and nm > 100
        _same(after, want)
        # the corrected map renders
        import torch

        g, n = dcg.dcg_gather_active(ctx, np.arange(dcg.dcg_chunk_count(ctx), dtype=np.int32))
        c = sc["cams"][0]
        rgb, depth = torch.zeros(3 * c.W * c.H, device="cuda"), torch.zeros(c.W * c.H, device="cuda")
        dcg.dcg_render_fwd(ctx, g, n, [c], rgb, depth)
        dcg.dcg_sync(ctx)
        assert n == N and float(rgb.abs().sum()) > 0
    finally:
        dcg.dcg_destroy(ctx)


def _zoomed(c, f=3.0):
    """A 320 x 240 view from pose c with f times its field-of-view scale (sees 22-28 of the 64 chunks)."""
    s = f * 320.0 / c.W
    return synth.Camera(c.fx * s, c.fy * s, 160.0, 120.0, 320, 240, c.Tcw, c.znear, c.zfar)


def test_keyframe_by_keyframe_when_the_union_exceeds_the_budget():
    """Sec. III-F: when the affected keyframes' chunks do not fit together, the keyframes are
    processed one at a time with the global transformation mask carried across the loads.  The
    result is the batch result, bit for bit (a context whose budget holds the union), and the
    reference's."""
    kfs = [_zoomed(c) for c in synth.window_scene(0, n=1000, deg=1)["cams"][:3]]
    corrs = [_corr("z", 2.0, (0.8, -0.4, 0.3)), _corr("x", 1.5, (-0.6, 0.5, 0.2)), _corr("z", -1.0, (0.3, 0.6, 0.0))]
    big, sc, F = _setup()
    small, _, _ = _setup(budget=30_000)
    try:
        before = _read_all(small, F)
        assert all(np.array_equal(before[k], v) for k, v in _read_all(big, F).items())
        info = dcg.dcg_chunk_info(small)
        lists = [dcg.dcg_cull_chunks(small, [k]) for k in kfs]
        own = [int(info["counts"][l].sum()) for l in lists]
        union = int(info["counts"][np.unique(np.concatenate(lists))].sum())
        assert max(own) <= 30_000 < union  # only the keyframe order fits
        nt_b, nm_b = dcg.dcg_loop_closure(big, kfs, corrs)
        nt_s, nm_s = dcg.dcg_loop_closure(small, kfs, corrs)
        dcg.dcg_flush(big)
        dcg.dcg_flush(small)
        after_b, after_s = _read_all(big, F), _read_all(small, F)
        assert (nt_s, nm_s) == (nt_b, nm_b) and nt_s > 1000 and nm_s > 100
        assert sorted(after_s) == sorted(after_b)
        assert all(np.array_equal(after_s[k], after_b[k]) for k in after_b)
        want, wt, wm = lc.loop_closure(before, sc["chunk_size"], 60.0, kfs, corrs)
        assert (nt_s, nm_s) == (wt, wm)
        _same(after_s, want)
        # the corrected map still gathers and renders within the budget
        import torch

        c = kfs[1]
        g, n = dcg.dcg_gather_active(small, dcg.dcg_cull_chunks(small, [c]))
        rgb, depth = torch.zeros(3 * c.W * c.H, device="cuda"), torch.zeros(c.W * c.H, device="cuda")
        dcg.dcg_render_fwd(small, g, n, [c], rgb, depth)
        dcg.dcg_sync(small)
        assert 0 < n <= 30_000 and float(rgb.abs().sum()) > 0
    finally:
        dcg.dcg_destroy(big)
        dcg.dcg_destroy(small)


def test_identity_correction_changes_nothing_and_budget_error_leaves_the_table():
    ctx, sc, F = _setup()
    try:
        before = _read_all(ctx, F)
        nt, nm = dcg.dcg_loop_closure(ctx, [sc["cams"][1]], [np.eye(4, dtype=np.float32)])
        dcg.dcg_flush(ctx)
        assert nt > 0 and nm == 0
        after = _read_all(ctx, F)
        assert sorted(after) == sorted(before)
        assert all(np.array_equal(after[k], before[k]) for k in before)
    finally:
        dcg.dcg_destroy(ctx)
    small, sc, F = _setup(budget=N // 16)
    try:
        before = _read_all(small, F)
        with pytest.raises(dcg.DcgError) as e:
            dcg.dcg_loop_closure(small, sc["cams"][:4], [_corr("z", 1.0, (0.1, 0, 0))] * 4)
        assert e.value.status == 4
        after = _read_all(small, F)
        assert all(np.array_equal(after[k], before[k]) for k in before)
    finally:
        dcg.dcg_destroy(small)


def test_reset_active_caps_opacity_and_zeroes_moments():
    ctx, sc, F = _setup()
    try:
        g, n = dcg.dcg_gather_active(ctx, np.arange(4, dtype=np.int32))
        p0 = dcg.active_tensor(g, n, F).cpu().numpy().copy()
        dcg.dcg_reset_active(ctx, g, n, 0.01)
        dcg.dcg_sync(ctx)
        p1 = dcg.active_tensor(g, n, F).cpu().numpy()
        cap = np.float32(np.log(0.01 / 0.99))
        assert np.array_equal(p1[10], np.minimum(p0[10], cap))
        assert np.array_equal(np.delete(p1, 10, 0), np.delete(p0, 10, 0))
        m, v = dcg.dcg_active_moments(ctx)
        assert not dcg.active_tensor(m, n, F).any() and not dcg.active_tensor(v, n, F).any()
    finally:
        dcg.dcg_destroy(ctx)
