"""Helpers of the GPU tests: marshal synthetic scenes into the C-ABI calls."""
from __future__ import annotations

import numpy as np

from paper_2511_23030_b300 import dcg, synth


def torch():
    import torch as _t

    return _t


def planar(params_aos: np.ndarray, stride: int | None = None):
    """[n, F] float32 numpy -> planar [F, stride] CUDA tensor."""
    t = torch()
    n, F = params_aos.shape
    stride = n if stride is None else stride
    out = t.zeros((F, max(stride, 1)), dtype=t.float32, device="cuda")
    if n:
        out[:, :n] = t.from_numpy(np.ascontiguousarray(params_aos.T))
    return out


def make_ctx(deg=3, n_max=600_000, views=8, pixels=None, inst=1 << 24, chunk=4.0, budget=None, host=None,
             tile=(16, 16), stage=16, dfar=100.0, page=2048, max_chunks=8192, flags=0, moments=0):
    pixels = 8 * 1241 * 376 if pixels is None else pixels
    budget = n_max if budget is None else budget
    host = n_max if host is None else host
    cfg = dcg.config(sh_degree=deg, max_active=n_max, max_views=views, max_pixels=pixels, max_instances=inst,
                     chunk_size=chunk, device_budget=budget, host_capacity=host, tile_w=tile[0], tile_h=tile[1],
                     stage=stage, dfar=dfar, page_gaussians=page, max_chunks=max_chunks, flags=flags,
                     with_moments=moments)
    return dcg.dcg_create(cfg)


def out_buffers(cams):
    t = torch()
    P = sum(c.W * c.H for c in cams)
    return t.zeros(3 * P, device="cuda"), t.zeros(P, device="cuda")


def split_views(rgb, depth, cams):
    """Stacked outputs -> per view ([3,H,W], [H,W]) numpy arrays."""
    out = []
    off = 0
    r = rgb.detach().cpu().numpy()
    d = depth.detach().cpu().numpy()
    for c in cams:
        P = c.W * c.H
        out.append((r[3 * off: 3 * off + 3 * P].reshape(3, c.H, c.W), d[off: off + P].reshape(c.H, c.W)))
        off += P
    return out


def render(ctx, params_aos, deg, cams, state=None):
    t = torch()
    g_t = planar(params_aos)
    g = dcg.gaussians(g_t, deg)
    rgb, depth = out_buffers(cams)
    dcg.dcg_render_fwd(ctx, g, params_aos.shape[0], cams, rgb, depth, state)
    dcg.dcg_sync(ctx)
    t.cuda.synchronize()
    return g_t, g, rgb, depth


def backward(ctx, g_t, deg, n, dr, dd, V, state=None):
    t = torch()
    grads_t = t.zeros_like(g_t)
    grads = dcg.gaussians(grads_t, deg)
    pose = t.zeros(V * 6, device="cuda")
    dcg.dcg_render_bwd(ctx, dr, dd, grads, pose, state)
    dcg.dcg_sync(ctx)
    return grads_t[:, :n].T.cpu().numpy().astype(np.float64), pose.view(V, 6).cpu().numpy().astype(np.float64)


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


GROUPS = {"mean": slice(0, 3), "log_scale": slice(3, 6), "quat": slice(6, 10), "opacity": slice(10, 11),
          "sh": slice(11, None)}


RGB_TOL = 1e-5  # RGB and T absolute, depth relative (to max(1, |depth|)), at unflagged pixels
T_TOL = 1e-5
GRAD_TOL = 1e-4  # relative L2 per parameter group and for the pose twist


def check_image(orc_out, rgb, depth, T, tag, max_flag=0.005):
    """GPU pixels against the oracle's, skipping the pixels the oracle flags
    (a discrete decision within rounding of its threshold)."""
    ok = orc_out["flags"] == 0
    assert ok.mean() >= 1 - max_flag, f"{tag}: flagged {1 - ok.mean():.4%}"
    e_rgb = np.abs(rgb[ok] - orc_out["rgb"][ok]).max()
    dz = np.abs(depth[ok] - orc_out["depth"][ok]) / np.maximum(1.0, np.abs(orc_out["depth"][ok]))
    e_T = np.abs(T[ok] - orc_out["T"][ok]).max()
    e_zabs = np.abs(depth[ok] - orc_out["depth"][ok]).max()
    print(f"{tag}: flagged {1 - ok.mean():.4%} rgb {e_rgb:.2e} T {e_T:.2e} depth rel {dz.max():.2e} abs {e_zabs:.2e}"
          f" (max depth {np.abs(orc_out['depth'][ok]).max():.2f})")
    assert e_rgb <= RGB_TOL, f"{tag}: rgb err {e_rgb}"
    assert dz.max() <= RGB_TOL, f"{tag}: depth err {dz.max()}"
    assert e_T <= T_TOL, f"{tag}: T err {e_T}"
    return e_rgb
