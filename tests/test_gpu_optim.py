"""Adam over the active set with per-Gaussian moments stored in the chunks:
the kernel against the FP64 reference, and the moments travelling losslessly
with their Gaussians through eviction to the host tier and back."""
import numpy as np
import pytest

from oracle import optim
from paper_2511_23030_b300 import dcg, synth

from gpu_util import make_ctx, planar

pytestmark = pytest.mark.gpu

# the C ABI takes the hyper-parameters as FP32; the reference uses the same values
B1, B2, EPS = (float(np.float32(x)) for x in (0.9, 0.999, 1e-8))


def _table(n=64_000, deg=1, budget=None, page=512, moments=1):
    sc = synth.window_scene(0, n=n, deg=deg)
    ctx = make_ctx(deg=deg, n_max=n, chunk=sc["chunk_size"], budget=budget, host=n, page=page, dfar=60.0,
                   moments=moments)
    dcg.dcg_chunk_table_update(ctx, planar(sc["params"]), n)
    return ctx, sc


def _lr(F):
    rng = np.random.default_rng(7)
    return rng.uniform(1e-4, 5e-2, F).astype(np.float32)


@pytest.mark.parametrize("grad_stride_pad", [0, 3])
def test_adam_step_matches_reference(grad_stride_pad):
    import torch

    ctx, sc = _table()
    try:
        F = sc["params"].shape[1]
        lst = dcg.dcg_cull_chunks(ctx, sc["cams"][:2])
        g, n = dcg.dcg_gather_active(ctx, lst)
        m, v = dcg.dcg_active_moments(ctx)
        rng = np.random.default_rng(grad_stride_pad)
        mt, vt = dcg.active_tensor(m, n, F), dcg.active_tensor(v, n, F)
        mt.copy_(torch.from_numpy(rng.normal(0, 0.1, (F, n)).astype(np.float32)))
        vt.copy_(torch.from_numpy(rng.uniform(0, 0.02, (F, n)).astype(np.float32)))
        # gradient rows padded to an odd stride exercise the unvectorised path
        S = n + grad_stride_pad
        gr = torch.zeros((F, S), device="cuda")
        gr[:, :n] = torch.from_numpy(rng.normal(0, 0.1, (F, n)).astype(np.float32))
        gr[:, n // 3] = 0.0  # zero gradients: only the moments decay
        pt = dcg.active_tensor(g, n, F)
        p0, m0, v0 = (x.double().cpu().numpy() for x in (pt, mt, vt))
        g0 = gr[:, :n].double().cpu().numpy()
        lr = _lr(F)
        dcg.dcg_adam_step(ctx, g, dcg.gaussians(gr, 1), n, lr, B1, B2, EPS, step=3)
        dcg.dcg_sync(ctx)
        p1, m1, v1 = (x.double().cpu().numpy() for x in (pt, mt, vt))
        pr, mr, vr = optim.adam_step(p0, g0, m0, v0, lr.astype(np.float64), B1, B2, EPS, 3)
        assert np.all(np.abs(p1 - pr) <= 1.2e-7 * np.abs(pr) + 1e-5 * np.abs(pr - p0) + 1e-12)
        assert np.all(np.abs(m1 - mr) <= 1e-6 * (B1 * np.abs(m0) + (1 - B1) * np.abs(g0)) + 1e-30)
        assert np.all(np.abs(v1 - vr) <= 1e-6 * (B2 * v0 + (1 - B2) * g0 * g0) + 1e-30)
        assert np.abs(p1 - p0).max() > 1e-4  # the step did move the parameters
    finally:
        dcg.dcg_destroy(ctx)


def _drive(budget, lists, steps, lr):
    """Gather each list in turn, take one Adam step with a gradient that is a
    fixed function of the parameters, scatter back.  Returns the context."""
    import torch

    ctx, sc = _table(budget=budget)
    F = sc["params"].shape[1]
    for t in range(1, steps + 1):
        g, n = dcg.dcg_gather_active(ctx, lists[(t - 1) % len(lists)])
        pt = dcg.active_tensor(g, n, F)
        grad = torch.sin(3.0 * pt).contiguous()
        dcg.dcg_adam_step(ctx, g, dcg.gaussians(grad, 1), n, lr, B1, B2, EPS, step=t)
        dcg.dcg_scatter_back(ctx, g, n)
    dcg.dcg_flush(ctx)
    dcg.dcg_sync(ctx)
    return ctx, F


def test_moments_survive_eviction_bit_exactly():
    # sliding groups of 8 of the 64 chunks; a budget of about 20 chunks forces
    # evictions; every Gaussian's parameters and moments must equal those of a
    # run where everything stays resident
    n = 64_000
    lists = [np.arange(k, k + 8, dtype=np.int32) % 64 for k in range(0, 64, 4)]
    lists = [np.sort(l) for l in lists]
    lr = _lr(11 + 3 * 4)
    small, F = _drive(int(n * 20 / 64), lists, 40, lr)
    big, _ = _drive(n, lists, 40, lr)
    try:
        st = dcg.dcg_tier_stats(small)
        assert st["evictions"] > 10 and dcg.dcg_tier_stats(big)["evictions"] == 0
        info = dcg.dcg_chunk_info(small)
        touched = 0
        for c in range(len(info["keys"])):
            cnt = int(info["counts"][c])
            pa, pb = dcg.dcg_chunk_read(small, c, cnt, F), dcg.dcg_chunk_read(big, c, cnt, F)
            (ma, va), (mb, vb) = dcg.dcg_chunk_read_moments(small, c, cnt, F), dcg.dcg_chunk_read_moments(big, c, cnt, F)
            assert np.array_equal(pa, pb) and np.array_equal(ma, mb) and np.array_equal(va, vb), c
            touched += int(np.abs(ma).max() > 0)
        assert touched == 64
    finally:
        dcg.dcg_destroy(small)
        dcg.dcg_destroy(big)


def test_fresh_moments_are_zero_and_errors():
    import torch

    ctx, sc = _table(n=8_000)
    plain, _ = _table(n=8_000, moments=0)
    try:
        F = sc["params"].shape[1]
        info = dcg.dcg_chunk_info(ctx)
        for c in range(3):
            m, v = dcg.dcg_chunk_read_moments(ctx, c, int(info["counts"][c]), F)
            assert not m.any() and not v.any()
        lst = np.arange(4, dtype=np.int32)
        g, n = dcg.dcg_gather_active(ctx, lst)
        gr = torch.zeros((F, n), device="cuda")
        with pytest.raises(dcg.DcgError) as e:  # n differs from the gathered set
            dcg.dcg_adam_step(ctx, g, dcg.gaussians(gr, 1), n - 1, _lr(F))
        assert e.value.status == 9
        with pytest.raises(dcg.DcgError) as e:  # bad hyper-parameters
            dcg.dcg_adam_step(ctx, g, dcg.gaussians(gr, 1), n, _lr(F), beta1=1.0)
        assert e.value.status == 1
        g2, n2 = dcg.dcg_gather_active(plain, lst)
        with pytest.raises(dcg.DcgError) as e:  # a context without moments
            dcg.dcg_adam_step(plain, g2, dcg.gaussians(torch.zeros((F, n2), device="cuda"), 1), n2, _lr(F))
        assert e.value.status == 1
        with pytest.raises(dcg.DcgError):
            dcg.dcg_active_moments(plain)
    finally:
        dcg.dcg_destroy(ctx)
        dcg.dcg_destroy(plain)
