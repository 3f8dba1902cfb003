"""Plain, slow FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product library never calls it and shares
no code with it.

The arithmetic lives in ``oracle.cpp`` (chunk ids, cull, projection, per-pixel
blending, analytic gradient); this module only marshals numpy arrays, plus a
few plain Python definitions (LRU selection, gather order, the L1 loss of
Eq. 2-4) that are short enough to read against the paper directly.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so (g++, FP64, no FMA contraction)."""
    src = os.path.join(_HERE, "oracle.cpp")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", _SO + ".tmp", src]
        subprocess.check_call(cmd)
        os.replace(_SO + ".tmp", _SO)
    return _SO


class OrcCam(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_double), ("fy", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("W", ctypes.c_int32), ("H", ctypes.c_int32), ("pad0", ctypes.c_int32), ("pad1", ctypes.c_int32),
                ("Tcw", ctypes.c_double * 16), ("znear", ctypes.c_double), ("zfar", ctypes.c_double)]


def _cam(c) -> OrcCam:
    # every value is taken from the float32 camera fields, widened exactly
    oc = OrcCam()
    oc.fx, oc.fy = float(np.float32(c.fx)), float(np.float32(c.fy))
    oc.cx, oc.cy = float(np.float32(c.cx)), float(np.float32(c.cy))
    oc.W, oc.H = int(c.W), int(c.H)
    T = np.asarray(c.Tcw, np.float32).astype(np.float64).reshape(16)
    for k in range(16):
        oc.Tcw[k] = T[k]
    oc.znear, oc.zfar = float(np.float32(c.znear)), float(np.float32(c.zfar))
    return oc


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_SO)
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------- Eq. 5 / Eq. 6
def chunk_keys(means: np.ndarray, s: float):
    """(coords int32 [n,3], keys uint64 [n], bad uint8 [n]) -- Eq. 5 and Eq. 6 in FP32."""
    means = np.ascontiguousarray(means, np.float32)
    n = means.shape[0]
    coords = np.zeros((n, 3), np.int32)
    keys = np.zeros(n, np.uint64)
    bad = np.zeros(n, np.uint8)
    lib().orc_chunk_keys(_p(means), ctypes.c_int64(n), ctypes.c_float(s), _p(coords), _p(keys), _p(bad))
    return coords, keys, bad


def decode_key(key: int):
    """Inverse of Eq. 6 for tests: (cx, cy, cz)."""
    m = (1 << 21) - 1
    key = int(key)
    return ((key >> 42) & m) - (1 << 20), ((key >> 21) & m) - (1 << 20), (key & m) - (1 << 20)


# ---------------------------------------------------------------- frustum cull
def cull(coords: np.ndarray, s: float, cam, dfar: float, hierarchical: bool = False) -> np.ndarray:
    coords = np.ascontiguousarray(coords, np.int32)
    mask = np.zeros(coords.shape[0], np.uint8)
    oc = _cam(cam)
    lib().orc_cull(_p(coords), ctypes.c_int64(coords.shape[0]), ctypes.c_double(float(np.float32(s))),
                   ctypes.byref(oc), ctypes.c_double(float(np.float32(dfar))), ctypes.c_int(int(hierarchical)),
                   _p(mask))
    return mask


def frustum_planes(cam):
    planes = np.zeros((6, 4))
    C = np.zeros(3)
    oc = _cam(cam)
    lib().orc_frustum_planes(ctypes.byref(oc), _p(planes), _p(C))
    return planes, C


# ---------------------------------------------------------------- LRU (Sec. III-E)
def lru_select(resident, visible, last_access, keys, counts, deficit):
    """Greedy LRU eviction of Sec. III-E: among resident chunks that the
    current step does not need, sorted oldest first (ties by chunk id), take
    the shortest prefix whose Gaussian count covers `deficit`.
    Returns the list of chunk indices, or None if even all of them are not enough."""
    if deficit <= 0:
        return []
    cand = [k for k in range(len(resident)) if resident[k] and not visible[k]]
    cand.sort(key=lambda k: (int(last_access[k]), int(keys[k])))
    freed = 0
    out = []
    for k in cand:
        out.append(k)
        freed += int(counts[k])
        if freed >= deficit:
            return out
    return None


def gather_order(keys: np.ndarray, counts: np.ndarray, visible: np.ndarray):
    """Active-set order of Sec. III-E "index only the visible Gaussians":
    visible chunks by ascending id, Gaussians within a chunk in stored order.
    Returns [(chunk index, offset in active set)] and the active count."""
    order = [k for k in np.argsort(keys, kind="stable") if visible[k]]
    out, off = [], 0
    for k in order:
        out.append((int(k), off))
        off += int(counts[k])
    return out, off


# ---------------------------------------------------------------- SH basis
def sh_basis(deg: int, dirs: np.ndarray) -> np.ndarray:
    dirs = np.ascontiguousarray(dirs, np.float64)
    out = np.zeros((dirs.shape[0], 16))
    lib().orc_sh_basis(ctypes.c_int(deg), _p(dirs), ctypes.c_int64(dirs.shape[0]), _p(out))
    return out


# ---------------------------------------------------------------- projection / rendering
PROJ_FIELDS = ["vis", "u", "v", "z", "A", "B", "C", "o", "r", "g", "b", "ex", "ey", "a", "b2", "c"]
# Blend order and the near-plane test use the FP32 depth key (see depth_f32).


def project(params: np.ndarray, deg: int, cam) -> dict:
    P = np.ascontiguousarray(params, np.float64)
    out = np.zeros((P.shape[0], 16))
    oc = _cam(cam)
    lib().orc_project_all(_p(P), ctypes.c_int64(P.shape[0]), ctypes.c_int(deg), ctypes.byref(oc), _p(out))
    return {k: out[:, i] for i, k in enumerate(PROJ_FIELDS)}


def clamp_flags(params: np.ndarray, deg: int, cam) -> np.ndarray:
    """Per Gaussian: bit 0 if x/z, bit 1 if y/z is clamped in the perspective
    Jacobian (the image extended by 15 % per side)."""
    P = np.ascontiguousarray(params, np.float64)
    out = np.zeros(P.shape[0], np.int32)
    lib().orc_clamp_flags(_p(P), ctypes.c_int64(P.shape[0]), ctypes.c_int(deg), ctypes.byref(_cam(cam)), _p(out))
    return out


def depth_f32(means: np.ndarray, cam) -> np.ndarray:
    means = np.ascontiguousarray(means, np.float32)
    T = np.ascontiguousarray(np.asarray(cam.Tcw, np.float32).reshape(16))
    z = np.zeros(means.shape[0], np.float32)
    lib().orc_depth_f32(_p(means), ctypes.c_int64(means.shape[0]), _p(T), _p(z))
    return z


# Flag bands around the discrete thresholds q = 9, alpha = 1/255, T = 1e-4:
# constant relative floors (none) and the factor on the first-order FP32 error
# bounds the oracle derives per pixel and Gaussian (see orc_collect).
DEFAULT_EPS = (0.0, 0.0, 0.0, 4.0)


def all_pixels(W: int, H: int) -> np.ndarray:
    ys, xs = np.mgrid[0:H, 0:W]
    return np.stack([xs.ravel(), ys.ravel()], 1).astype(np.int32)


def render(params, deg, cam, pix=None, eps=DEFAULT_EPS, n_threads=0):
    """Render the listed pixels ([m,2] int32 x,y; all pixels if None).
    Returns dict rgb [m,3], depth [m], T [m], n [m], flags [m]."""
    P = np.ascontiguousarray(params, np.float64)
    pix = all_pixels(cam.W, cam.H) if pix is None else np.ascontiguousarray(pix, np.int32)
    m = pix.shape[0]
    rgb = np.zeros((m, 3))
    depth = np.zeros(m)
    T = np.zeros(m)
    n = np.zeros(m, np.int32)
    fl = np.zeros(m, np.int32)
    e = np.asarray(eps, np.float64)
    oc = _cam(cam)
    lib().orc_render(_p(P), ctypes.c_int64(P.shape[0]), ctypes.c_int(deg), ctypes.byref(oc), _p(pix),
                     ctypes.c_int64(m), _p(e), ctypes.c_int(n_threads), _p(rgb), _p(depth), _p(T), _p(n), _p(fl))
    return dict(rgb=rgb, depth=depth, T=T, n=n, flags=fl, pix=pix)


def render_bwd(params, deg, cam, dL_drgb, dL_ddepth, pix=None, n_threads=0):
    """Gradient of sum_k (dL_drgb[k] . rgb[k] + dL_ddepth[k] * depth[k]) over the
    listed pixels, w.r.t. the parameters ([n,F]) and the pose twist (6)."""
    P = np.ascontiguousarray(params, np.float64)
    pix = all_pixels(cam.W, cam.H) if pix is None else np.ascontiguousarray(pix, np.int32)
    gr = np.ascontiguousarray(dL_drgb, np.float64).reshape(-1, 3)
    gd = np.ascontiguousarray(dL_ddepth, np.float64).reshape(-1)
    grad = np.zeros_like(P)
    gpose = np.zeros(6)
    oc = _cam(cam)
    lib().orc_render_bwd(_p(P), ctypes.c_int64(P.shape[0]), ctypes.c_int(deg), ctypes.byref(oc), _p(pix),
                         ctypes.c_int64(pix.shape[0]), _p(gr), _p(gd), ctypes.c_int(n_threads), _p(grad), _p(gpose))
    return grad, gpose


# ---------------------------------------------------------------- loss, Eq. 2-4 (L1 parts)
def l1_loss(rgb, depth, tgt_rgb, tgt_depth, lam):
    """L = mean|C - C_gt| + lam * mean|D - D_gt| for one view (rgb as [P,3] or
    [3,H,W] consistently with the target); returns (L, dL/drgb, dL/ddepth)."""
    rgb = np.asarray(rgb, np.float64)
    depth = np.asarray(depth, np.float64)
    P = depth.size
    dr = rgb - np.asarray(tgt_rgb, np.float64)
    dd = depth - np.asarray(tgt_depth, np.float64)
    L = np.abs(dr).sum() / (3 * P) + lam * np.abs(dd).sum() / P
    return L, np.sign(dr) / (3 * P), lam * np.sign(dd) / P
