"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers and lays out scenes and camera paths;
it holds none of the mapper's arithmetic (no projection, blending, keys or
culling).  Both the CUDA path and the CPU oracle take their inputs from here.

Gaussian records are returned as float32 arrays of shape [n, F] with
F = 11 + 3 * (deg + 1)**2 and columns
    0..2 mean, 3..5 log-scale, 6..9 quaternion (w, x, y, z), 10 opacity logit,
    11 + 3k + ch  SH coefficient k of colour channel ch.
Cameras use the pinhole model with x right, y down, z forward and a
world-to-camera rigid transform Tcw (4x4, float32).

Workloads (the paper's datasets -- Replica, TUM-RGBD, KITTI -- are not
available; these stand in for them with their shapes):
  room_*     : one 128x96 view of 4096 Gaussians (small parity case), and a
               640x480 indoor box room of 500k Gaussians on its walls, floor
               and ceiling (Replica/TUM-like indoor scale).
  window_*   : 2M Gaussians in 64 chunks of 4 m, eight keyframes of mixed size
               (4 x 1200x680, 2 x 640x480, 2 x 320x240).
  corridor_* : 1241x376 views (KITTI size) along a piecewise-clothoid road at
               1 m/frame, road plane plus box facades in 8 m chunks.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

Y00 = 0.5 / math.sqrt(math.pi)  # value of the l=0 real SH; maps a DC colour to a coefficient


def n_sh(deg: int) -> int:
    return (deg + 1) ** 2


def n_fields(deg: int) -> int:
    return 11 + 3 * n_sh(deg)


@dataclasses.dataclass
class Camera:
    fx: float
    fy: float
    cx: float
    cy: float
    W: int
    H: int
    Tcw: np.ndarray  # float32 [4,4], world -> camera
    znear: float = 0.2
    zfar: float = 100.0

    @property
    def n_pixels(self) -> int:
        return int(self.W) * int(self.H)


def look_at(eye, target, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """World->camera transform of a camera at `eye` looking at `target` (x right, y down, z forward)."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    if np.linalg.norm(r) < 1e-9:
        r = np.cross(f, np.array([0.0, 1.0, 0.0]))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)  # "down" completes a right-handed x-right, y-down, z-forward frame
    Rcw = np.stack([r, d, f], 0)
    T = np.eye(4)
    T[:3, :3] = Rcw
    T[:3, 3] = -Rcw @ eye
    return T.astype(np.float32)


def random_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def _gaussians(rng, means, deg, log_s_range, sh_sigma=None, dc_rgb=None, logit_sigma=1.0):
    n = means.shape[0]
    F = n_fields(deg)
    P = np.zeros((n, F), np.float32)
    P[:, 0:3] = means
    P[:, 3:6] = rng.uniform(math.log(log_s_range[0]), math.log(log_s_range[1]), (n, 3))
    P[:, 6:10] = random_quats(rng, n)
    P[:, 10] = rng.standard_normal(n) * logit_sigma
    if dc_rgb is not None:
        P[:, 11:14] = (dc_rgb - 0.5) / Y00
    if sh_sigma is not None:
        P[:, 11:] = rng.standard_normal((n, 3 * n_sh(deg))) * sh_sigma
    return P


# ----------------------------------------------------------------------------
# small single-view case
# ----------------------------------------------------------------------------
def room_small(seed: int = 0, n: int = 4096, W: int = 128, H: int = 96):
    """One 128x96 pinhole view (fx=fy=100, cx=64, cy=48, identity pose) of 4096
    Gaussians: means U([-2,2]^2 x [1,5]), log-uniform scales [0.01, 0.1], random
    unit quaternions, opacity logit N(0,1), SH degree 0 with DC colour U[0,1];
    L1 loss against a U[0,1] target."""
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-2, 2, n), rng.uniform(-2, 2, n), rng.uniform(1, 5, n)], 1).astype(np.float32)
    rgb = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    P = _gaussians(rng, means, 0, (0.01, 0.1), dc_rgb=rgb)
    cam = Camera(100.0, 100.0, W / 2.0, H / 2.0, W, H, np.eye(4, dtype=np.float32), 0.2, 100.0)
    target = rng.uniform(0, 1, (3, H, W)).astype(np.float32)
    return dict(params=P, deg=0, cams=[cam], target_rgb=[target], target_depth=[np.zeros((H, W), np.float32)],
                lambda_depth=0.0, chunk_size=4.0)


# ----------------------------------------------------------------------------
# indoor room
# ----------------------------------------------------------------------------
def _box_surface_points(rng, lo, hi, n):
    """n points uniform (area-weighted) on the six faces of box [lo, hi]."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    ext = hi - lo
    areas = np.array([ext[1] * ext[2], ext[1] * ext[2], ext[0] * ext[2], ext[0] * ext[2], ext[0] * ext[1], ext[0] * ext[1]])
    face = rng.choice(6, size=n, p=areas / areas.sum())
    pts = lo + rng.uniform(0, 1, (n, 3)) * ext
    axis = face // 2
    side = face % 2
    pts[np.arange(n), axis] = np.where(side == 0, lo[axis], hi[axis])
    return pts


def room_trajectory(rng, n_steps, lo=(-5.0, -4.0, 0.0), hi=(5.0, 4.0, 3.0), margin=1.2):
    """Smooth random walk inside the room: Ornstein-Uhlenbeck position, low-pass yaw/pitch."""
    lo = np.asarray(lo) + margin
    hi = np.asarray(hi) - margin
    lo[2], hi[2] = 1.2, 1.8
    centre = (lo + hi) / 2
    pos = centre.copy()
    vel = np.zeros(3)
    yaw, pitch, dyaw = rng.uniform(0, 2 * math.pi), 0.0, 0.0
    poses = []
    for _ in range(n_steps):
        vel = 0.85 * vel + 0.05 * rng.standard_normal(3) - 0.02 * (pos - centre)
        vel[2] *= 0.2
        pos = np.clip(pos + vel, lo, hi)
        dyaw = 0.9 * dyaw + 0.03 * rng.standard_normal()
        yaw += dyaw
        pitch = 0.9 * pitch + 0.02 * rng.standard_normal()
        fwd = np.array([math.cos(yaw) * math.cos(pitch), math.sin(yaw) * math.cos(pitch), math.sin(pitch)])
        poses.append(look_at(pos, pos + fwd))
    return poses


def room_indoor(seed: int = 0, n: int = 500_000, W: int = 640, H: int = 480, n_steps: int = 8):
    """500k Gaussians on the walls, floor and ceiling of a 10x8x3 m room (area
    weighted) with N(0, 0.05 m) jitter; SH degree 3, coefficients N(0, 0.2);
    log-uniform scales [0.005, 0.05]; 4 m chunks; one keyframe per step on a
    smooth random walk; loss L1 RGB + 0.1 L1 depth."""
    rng = np.random.default_rng(seed)
    lo, hi = (-5.0, -4.0, 0.0), (5.0, 4.0, 3.0)
    means = _box_surface_points(rng, lo, hi, n) + rng.normal(0, 0.05, (n, 3))
    P = _gaussians(rng, means.astype(np.float32), 3, (0.005, 0.05), sh_sigma=0.2)
    f = 0.8 * W
    cams = [Camera(f, f, W / 2.0, H / 2.0, W, H, T, 0.2, 20.0) for T in room_trajectory(rng, n_steps, lo, hi)]
    targets = [rng.uniform(0, 1, (3, H, W)).astype(np.float32) for _ in cams]
    tdepth = [rng.uniform(0.5, 6.0, (H, W)).astype(np.float32) for _ in cams]
    return dict(params=P, deg=3, cams=cams, target_rgb=targets, target_depth=tdepth, lambda_depth=0.1,
                chunk_size=4.0)


# ----------------------------------------------------------------------------
# batched keyframe window: 2M Gaussians, 64 chunks of 4 m, 8 mixed views
# ----------------------------------------------------------------------------
def clamp_scene(seed: int = 21, deg: int = 3):
    """A 48x40 view (f = 30, identity pose) and 13 Gaussians: ten whose centres
    project beyond the image extended by 15 % of its size on each side (right,
    left, below, above and two corners; x/z or y/z or both outside the limits
    of the perspective Jacobian) with scales large enough that their 3-sigma
    ellipses reach into the image, and three inside it."""
    W, H = 48, 40
    cam = Camera(30.0, 30.0, 23.5, 19.5, W, H, np.eye(4, dtype=np.float32), 0.2, 50.0)
    # (x/z, y/z, z, scale)
    spec = [(1.30, 0.05, 3.0, 0.80), (1.22, -0.30, 3.6, 0.90), (-1.25, 0.10, 3.2, 0.85), (-1.18, 0.40, 2.8, 0.75),
            (0.10, 1.05, 3.1, 0.80), (-0.20, 0.98, 3.5, 0.75), (0.20, -1.02, 3.3, 0.80), (-0.10, -0.97, 2.9, 0.70),
            (1.20, 1.00, 3.4, 1.00), (-1.15, -0.95, 3.0, 1.00),
            (0.10, 0.05, 4.0, 0.10), (-0.40, 0.20, 3.7, 0.12), (0.35, -0.30, 3.9, 0.08)]
    rng = np.random.default_rng(seed)
    n = len(spec)
    P = np.zeros((n, n_fields(deg)))
    for i, (rx, ry, z, s) in enumerate(spec):
        P[i, 0:3] = (rx * z, ry * z, z)
        P[i, 3:6] = np.log(s * rng.uniform(0.6, 1.0, 3))
    P[:, 6:10] = random_quats(rng, n)
    P[:, 10] = rng.uniform(-0.5, 0.5, n)
    P[:, 11:] = rng.normal(0, 0.3, (n, P.shape[1] - 11))
    return P, cam


WINDOW_SIZES = [(1200, 680)] * 4 + [(640, 480)] * 2 + [(320, 240)] * 2


def window_scene(seed: int = 0, n: int = 2_000_000, chunk: float = 4.0, per_axis: int = 4, sizes=None,
                 deg: int = 3):
    """`per_axis`^3 chunks of side `chunk` (64 chunks of 4 m by default); chunk
    c spans [c*s - s/2, c*s + s/2) with c in {-1, 0, 1, 2}.  Each chunk holds the
    same number of Gaussians on the surface of one random axis-aligned box
    (side 1-3 m) inside it, with 1 cm jitter.  SH degree 3 with N(0, 0.2)
    coefficients, log-uniform scales [0.005, 0.05], opacity logit N(0,1).
    Eight keyframes look at the volume from a ring 13-17 m around its centre."""
    rng = np.random.default_rng(seed)
    sizes = WINDOW_SIZES if sizes is None else sizes
    n_chunks = per_axis ** 3
    per = np.full(n_chunks, n // n_chunks)
    per[: n - per.sum()] += 1
    cs = np.arange(per_axis) - (per_axis // 2 - 1)
    parts = []
    for k, (ix, iy, iz) in enumerate(np.array(np.meshgrid(cs, cs, cs, indexing="ij")).reshape(3, -1).T):
        centre = np.array([ix, iy, iz], np.float64) * chunk
        side = rng.uniform(1.0, 3.0, 3)
        off = rng.uniform(-(chunk - side) / 2 + 0.05, (chunk - side) / 2 - 0.05)
        lo = centre + off - side / 2
        parts.append(_box_surface_points(rng, lo, lo + side, int(per[k])))
    means = np.concatenate(parts, 0) + rng.normal(0, 0.01, (n, 3))
    P = _gaussians(rng, means.astype(np.float32), deg, (0.005, 0.05), sh_sigma=0.2)
    vol_c = np.full(3, (cs[0] + cs[-1]) / 2 * chunk)
    cams = []
    for k, (W, H) in enumerate(sizes):
        ang = 2 * math.pi * k / len(sizes) + rng.uniform(-0.2, 0.2)
        rad = rng.uniform(13.0, 17.0)
        eye = vol_c + np.array([rad * math.cos(ang), rad * math.sin(ang), rng.uniform(-3.0, 5.0)])
        tgt = vol_c + rng.normal(0, 1.0, 3)
        f = 0.9 * W
        cams.append(Camera(f, f, W / 2.0, H / 2.0, W, H, look_at(eye, tgt), 0.2, 60.0))
    targets = [rng.uniform(0, 1, (3, c.H, c.W)).astype(np.float32) for c in cams]
    tdepth = [rng.uniform(5.0, 30.0, (c.H, c.W)).astype(np.float32) for c in cams]
    return dict(params=P, deg=deg, cams=cams, target_rgb=targets, target_depth=tdepth, lambda_depth=0.1,
                chunk_size=chunk)


# ----------------------------------------------------------------------------
# driving corridor (out-of-core)
# ----------------------------------------------------------------------------
def corridor_path(seed: int = 0, length_m: float = 5000.0, step_m: float = 1.0):
    """Piecewise-clothoid road centre line: curvature varies linearly within
    segments of 50-300 m, |kappa| <= 1/150 m^-1.  Returns [n,2] xy points at
    step_m spacing and the heading at each point."""
    rng = np.random.default_rng(seed + 17)
    n = int(length_m / step_m) + 1
    xy = np.zeros((n, 2))
    head = np.zeros(n)
    kappa = 0.0
    k_target = 0.0
    seg_left = 0.0
    dk = 0.0
    for i in range(1, n):
        if seg_left <= 0:
            seg_len = rng.uniform(50, 300)
            k_target = rng.uniform(-1 / 150, 1 / 150) if rng.uniform() < 0.6 else 0.0
            dk = (k_target - kappa) / (seg_len / step_m)
            seg_left = seg_len
        kappa += dk
        seg_left -= step_m
        head[i] = head[i - 1] + kappa * step_m
        xy[i] = xy[i - 1] + step_m * np.array([math.cos(head[i]), math.sin(head[i])])
    return xy, head


def corridor_gaussians(rng, xy, head, per_m: int, deg: int = 3, road_half: float = 6.0, facade_off: float = 10.0,
                       facade_h: float = 12.0, i0: int = 0, i1: int | None = None):
    """Gaussians for path samples [i0, i1): road plane (width 2*road_half) and
    two facades at +-facade_off, height facade_h.  per_m Gaussians per metre
    of path, split 1/3 road, 2/3 facades."""
    i1 = len(xy) if i1 is None else i1
    m = i1 - i0
    n = m * per_m
    seg = rng.integers(i0, i1, n)
    along = rng.uniform(0, 1, n)
    c, s = np.cos(head[seg]), np.sin(head[seg])
    base = xy[seg] + along[:, None] * np.stack([c, s], 1)
    nrm = np.stack([-s, c], 1)
    kind = rng.uniform(0, 1, n)
    lat = np.where(kind < 1 / 3, rng.uniform(-road_half, road_half, n),
                   np.where(kind < 2 / 3, -facade_off, facade_off))
    z = np.where(kind < 1 / 3, 0.0, rng.uniform(0.0, facade_h, n))
    p = np.concatenate([base + lat[:, None] * nrm, z[:, None]], 1) + rng.normal(0, 0.03, (n, 3))
    return _gaussians(rng, p.astype(np.float32), deg, (0.02, 0.2), sh_sigma=0.2)


def corridor_cameras(xy, head, W=1241, H=376, height=1.6, every=1):
    f = 0.6 * W
    cams = []
    for i in range(0, len(xy) - 1, every):
        eye = np.array([xy[i, 0], xy[i, 1], height])
        fwd = np.array([math.cos(head[i]), math.sin(head[i]), -0.03])
        cams.append(Camera(f, f, W / 2.0, H / 2.0, W, H, look_at(eye, eye + fwd), 0.2, 60.0))
    return cams


def pixel_sample(rng: np.random.Generator, W: int, H: int, m: int) -> np.ndarray:
    """m distinct pixel coordinates (x, y) as int32 [m, 2]."""
    idx = rng.choice(W * H, size=min(m, W * H), replace=False)
    return np.stack([idx % W, idx // W], 1).astype(np.int32)


# Parameter layout of the chunk-prefetch MLP (128 -> 256 -> 256 -> 256 -> 1):
# W1[128][256] b1 W2[256][256] b2 W3[256][256] b3 w4[256] b4, row-major.
MLP_SIZES = [("W1", (128, 256)), ("b1", (256,)), ("W2", (256, 256)), ("b2", (256,)), ("W3", (256, 256)),
             ("b3", (256,)), ("w4", (256,)), ("b4", (1,))]


def mlp_init_params(seed: int = 0) -> np.ndarray:
    """Seeded initial weights of the prefetch MLP (flat float32 in the layout
    above): uniform in +-1/sqrt(fan_in), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shp in MLP_SIZES:
        if name.startswith("b"):
            parts.append(np.zeros(shp))
        else:
            parts.append(rng.uniform(-1, 1, shp) / np.sqrt(shp[0]))
    return np.concatenate([p.reshape(-1) for p in parts]).astype(np.float32)

