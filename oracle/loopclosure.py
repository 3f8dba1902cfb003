"""Reference of the loop-closure correction of the chunk map -- TEST INFRASTRUCTURE ONLY.

Sec. III-F of the paper: for every affected keyframe the chunks its frustum
cull keeps are collected (and loaded together); the Gaussians visible from the
keyframe are moved with the keyframe's pose correction (positions and
rotations), a global transformation mask making sure a Gaussian visible from
several keyframes is moved once ("Cross-Chunk Transformation"); afterwards the
chunk of every moved Gaussian is recomputed (Eq. 5/6) and Gaussians that left
their chunk are moved to the right one ("Chunk Redistribution").

Readings (the paper leaves them open): a Gaussian is visible from keyframe k
if its chunk passes k's cull and its centre projects into k's image with
znear < z <= zfar; the first keyframe in the given order that sees it moves
it; the correction C_k acts as x' = C_k x on the centre and as
q' = q(C_k) (x) q on the rotation; a chunk keeps its remaining Gaussians in
stored order and receives incoming ones after them in gather order (chunks by
ascending id, each in stored order); emptied chunks stay.  The visibility
decision, the corrected centre and hence the chunk ids are FP32 with one
rounding per operation in the order ((a x + b y) + c z) + d, as the kernel
computes them: they decide integers, so both sides take them in the same
precision.  The quaternion product is compared with a tolerance.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial.transform import Rotation

import oracle


def _dot3(r, x, y, z, t):
    f = np.float32
    return ((f(r[0]) * x + f(r[1]) * y) + f(r[2]) * z) + f(t)


def _qmul(a, b):
    """Hamilton product a (x) b of (w, x, y, z) quaternions (FP64)."""
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def decode_coords(key: int):
    m = (1 << 21) - 1
    return np.array([((key >> 42) & m) - (1 << 20), ((key >> 21) & m) - (1 << 20), (key & m) - (1 << 20)], np.int32)


def loop_closure(chunks: dict, chunk_size: float, dfar: float, keyframes, corrections):
    """chunks: {key: rows [count, Fs] float32 (parameters then any moments), stored order}.
    Returns (new chunks dict, n_transformed, n_moved)."""
    keys = sorted(chunks)
    coords = np.stack([decode_coords(k) for k in keys]) if keys else np.zeros((0, 3), np.int32)
    masks = [oracle.cull(coords, chunk_size, cam, dfar) for cam in keyframes]
    union = [i for i in range(len(keys)) if any(m[i] for m in masks)]
    corr = [np.asarray(c, np.float32).reshape(4, 4) for c in corrections]
    qc = []
    for C in corr:
        xyzw = Rotation.from_matrix(C[:3, :3].astype(np.float64)).as_quat()
        qc.append(np.array([xyzw[3], xyzw[0], xyzw[1], xyzw[2]]))
    f = np.float32
    out = {k: chunks[k].copy() for k in keys}
    gathered = []  # (chunk index, row) in gather order
    n_t = 0
    for ci in union:
        rows = out[keys[ci]]
        for r in range(rows.shape[0]):
            x, y, z = rows[r, 0], rows[r, 1], rows[r, 2]
            for k, cam in enumerate(keyframes):
                if not masks[k][ci]:
                    continue
                T = np.asarray(cam.Tcw, np.float32).reshape(4, 4)
                tx = _dot3(T[0, :3], x, y, z, T[0, 3])
                ty = _dot3(T[1, :3], x, y, z, T[1, 3])
                tz = _dot3(T[2, :3], x, y, z, T[2, 3])
                if not (tz > f(cam.znear) and tz <= f(cam.zfar)):
                    continue
                u = f(cam.fx) * (tx / tz) + f(cam.cx)
                v = f(cam.fy) * (ty / tz) + f(cam.cy)
                if not (u >= f(0) and u < f(cam.W) and v >= f(0) and v < f(cam.H)):
                    continue
                C = corr[k]
                rows[r, 0] = _dot3(C[0, :3], x, y, z, C[0, 3])
                rows[r, 1] = _dot3(C[1, :3], x, y, z, C[1, 3])
                rows[r, 2] = _dot3(C[2, :3], x, y, z, C[2, 3])
                rows[r, 6:10] = _qmul(qc[k], rows[r, 6:10].astype(np.float64)).astype(np.float32)
                n_t += 1
                break
            gathered.append((ci, r))
    # redistribution
    stay = {keys[ci]: [] for ci in union}
    incoming = {}
    n_m = 0
    for ci, r in gathered:
        row = out[keys[ci]][r]
        _, nk, bad = oracle.chunk_keys(row[None, :3].astype(np.float32), chunk_size)
        assert not bad.any()
        nk = int(nk[0])
        if nk == keys[ci]:
            stay[keys[ci]].append(row)
        else:
            incoming.setdefault(nk, []).append(row)
            n_m += 1
    new = {}
    Fs = next(iter(chunks.values())).shape[1] if chunks else 0
    empty = np.zeros((0, Fs), np.float32)
    for k in keys:
        if k in stay:
            new[k] = np.array(stay[k] + incoming.pop(k, []), np.float32).reshape(-1, Fs)
        else:
            new[k] = out[k]
    for k, rows in incoming.items():
        new[k] = np.concatenate([new.get(k, empty), np.array(rows, np.float32).reshape(-1, Fs)])
    return new, n_t, n_m
