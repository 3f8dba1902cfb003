"""The bounds-check build (libdcg_checks.so: the same sources compiled with
-DDCG_CHECKS=1, whose kernels test pair, instance, tile and pixel indices
against their buffers and record a violation in the device error word
instead of accessing) on the window workload, forward and backward through
the chunk path: no violation is reported, and it renders what the normal
build renders.  Each build runs in a process of its own (the binding loads
one library per process, chosen by DCG_LIB)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

STEP = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[2])
import torch
from paper_2511_23030_b300 import build, dcg, synth
from gpu_util import make_ctx, out_buffers, planar
build.build(checks=dcg.LIB_PATH.endswith("libdcg_checks.so"))
sc = synth.window_scene(0, n=64_000, deg=3)
cams = sc["cams"][:4]
n, F = sc["params"].shape
ctx = make_ctx(deg=3, n_max=n, views=4, pixels=sum(c.W * c.H for c in cams), inst=8 << 20, chunk=sc["chunk_size"],
               dfar=60.0, page=512)
status = "DCG_OK"
try:
    dcg.dcg_chunk_table_update(ctx, planar(sc["params"]), n)
    g, na = dcg.dcg_gather_active(ctx, dcg.dcg_cull_chunks(ctx, cams))
    rgb, depth = out_buffers(cams)
    dcg.dcg_render_fwd(ctx, g, na, cams, rgb, depth)
    dr = torch.sin(rgb * 7.0) * 1e-3
    dd = torch.cos(depth) * 1e-4
    grads = torch.zeros((F, na), device="cuda")
    pose = torch.zeros(6 * len(cams), device="cuda")
    dcg.dcg_render_bwd(ctx, dr, dd, dcg.gaussians(grads, 3), pose)
    dcg.dcg_scatter_back(ctx, g, na)
    dcg.dcg_flush(ctx)
    dcg.dcg_sync(ctx)
except dcg.DcgError as e:
    status = str(e)
np.savez(sys.argv[3], rgb=rgb.cpu().numpy(), depth=depth.cpu().numpy(), grads=grads.cpu().numpy(),
         pose=pose.cpu().numpy())
print(json.dumps({"lib": dcg.LIB_PATH, "status": status, "active": int(na)}))
dcg.dcg_destroy(ctx)
"""


def _run(tmp_path, lib):
    env = dict(os.environ)
    env.pop("DCG_LIB", None)
    if lib:
        env["DCG_LIB"] = lib
    out = tmp_path / f"{lib or 'normal'}.npz"
    r = subprocess.run([sys.executable, "-c", STEP, ROOT, HERE, str(out)], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1]), np.load(out)


def test_bounds_check_build_reports_nothing_and_renders_the_same(tmp_path):
    info_c, res_c = _run(tmp_path, "checks")
    info_n, res_n = _run(tmp_path, None)
    assert info_c["lib"].endswith("libdcg_checks.so") and info_n["lib"].endswith("libdcg.so")
    assert info_c["status"] == "DCG_OK" and info_n["status"] == "DCG_OK", (info_c, info_n)
    assert info_c["active"] == info_n["active"] > 10_000
    assert np.array_equal(res_c["rgb"], res_n["rgb"]) and np.array_equal(res_c["depth"], res_n["depth"])
    for k in ("grads", "pose"):  # gradient atomics may add in another order
        a, b = res_c[k].astype(np.float64), res_n[k].astype(np.float64)
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b), k
