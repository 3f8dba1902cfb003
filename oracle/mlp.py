"""FP64 reference of the chunk-prefetch MLP -- TEST INFRASTRUCTURE ONLY.

Network (the learned prefetch proposal): 128 inputs -> 256 -> 256 -> 256 -> 1,
GELU(x) = x Phi(x) = x (1 + erf(x / sqrt 2)) / 2 after each hidden layer,
sigmoid output, binary cross-entropy averaged over the batch, Adam.
Flat parameter layout: W1[128][256] b1 W2[256][256] b2 W3[256][256] b3 w4[256] b4.

`bf16_storage=True` rounds to bfloat16 (nearest, ties to even) exactly where
the kernels store BF16: the weights W1..W3, w4, the inputs, every hidden
activation and every back-propagated pre-activation gradient.  With it off
the network is evaluated in plain FP64.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

N_IN, N_HID = 128, 256
SIZES = [("W1", (N_IN, N_HID)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
         ("W3", (N_HID, N_HID)), ("b3", (N_HID,)), ("w4", (N_HID,)), ("b4", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(flat):
    out, o = {}, 0
    for name, shp in SIZES:
        k = int(np.prod(shp))
        out[name] = np.asarray(flat[o:o + k], np.float64).reshape(shp)
        o += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in SIZES])


def bf16(a):
    """Round float values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return (u.astype(np.uint32)).view(np.float32).astype(np.float64)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(flat, x, bf16_storage=True):
    p = unpack(flat)
    q = bf16 if bf16_storage else (lambda a: np.asarray(a, np.float64))
    h = q(x)
    cache = {"h0": h}
    for l in (1, 2, 3):
        z = h @ q(p[f"W{l}"]) + p[f"b{l}"]
        h = q(gelu(z))
        cache[f"z{l}"], cache[f"h{l}"] = z, h
    logit = h @ q(p["w4"]) + p["b4"][0]
    cache["logit"] = logit
    return 1.0 / (1.0 + np.exp(-logit)), cache


def loss_and_grads(flat, x, y, bf16_storage=True):
    p = unpack(flat)
    q = bf16 if bf16_storage else (lambda a: np.asarray(a, np.float64))
    _, c = forward(flat, x, bf16_storage)
    z = c["logit"]
    y = np.asarray(y, np.float64)
    B = len(y)
    L = float(np.mean(np.maximum(z, 0) - z * y + np.log1p(np.exp(-np.abs(z)))))
    dz = (1.0 / (1.0 + np.exp(-z)) - y) / B
    g = {"w4": c["h3"].T @ dz, "b4": np.array([dz.sum()])}
    dZ = q(np.outer(dz, q(p["w4"])) * gelu_grad(c["z3"]))
    for l in (3, 2, 1):
        g[f"W{l}"] = c[f"h{l - 1}"].T @ dZ
        g[f"b{l}"] = dZ.sum(0)
        if l > 1:
            dZ = q((dZ @ q(p[f"W{l}"]).T) * gelu_grad(c[f"z{l - 1}"]))
    return L, pack(g)


def adam_step(flat, grad, m1, m2, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) with bias correction; returns new (params, m1, m2)."""
    m1 = b1 * m1 + (1 - b1) * grad
    m2 = b2 * m2 + (1 - b2) * grad * grad
    mh = m1 / (1 - b1 ** t)
    vh = m2 / (1 - b2 ** t)
    return flat - lr * mh / (np.sqrt(vh) + eps), m1, m2


# ------------------------------------------------------------------ features
def se3_log(T):
    """Twist (u, w) of a rigid 4x4 transform via the matrix logarithm."""
    from scipy.linalg import logm

    L = np.real(logm(np.asarray(T, np.float64)))
    w = np.array([L[2, 1], L[0, 2], L[1, 0]])
    return np.concatenate([L[:3, 3], w])


def features(pose_hist_tcw, chunk_coords, s):
    """Rows of 128: twists log(T_t^-1 T_{t-k}) of the camera-to-world poses,
    k = 0..15 (translation / 16 m), then each chunk centre in the current
    camera frame / 60 m, then zeros."""
    Tcw = [np.asarray(T, np.float64).reshape(4, 4) for T in pose_hist_tcw]
    tw = []
    for k in range(16):
        rel = Tcw[0] @ np.linalg.inv(Tcw[k])
        xi = se3_log(rel)
        tw.append(np.concatenate([xi[:3] / 16.0, xi[3:]]))
    tw = np.concatenate(tw)
    rows = np.zeros((len(chunk_coords), N_IN))
    rows[:, :96] = tw
    centres = np.asarray(chunk_coords, np.float64) * s
    rows[:, 96:99] = (centres @ Tcw[0][:3, :3].T + Tcw[0][:3, 3]) / 60.0
    return rows
