"""Learned chunk prefetch along a trajectory: orchestration of library calls.

Every computation runs in libdcg.so (exact cull, feature kernel, MLP
training and inference kernels, asynchronous chunk copies); this module only
sequences the calls, keeps per-step bookkeeping and marshals arguments.

Dataset (the mapper generates it itself): for frame t, the candidates are the
chunks whose cube lies within 1.5 zfar of the camera centre; the label of a
candidate is 1 iff the exact frustum cull finds it visible in any of frames
t+1 .. t+20; the features are the SE(3) logarithms of the last 16 poses
relative to the current one and the candidate's centre in the camera frame.
"""
from __future__ import annotations

import numpy as np

from . import dcg

HIST = 16
HORIZON = 20


def cam_centre(cam):
    T = np.asarray(cam.Tcw, np.float64)
    return (-T[:3, :3].T @ T[:3, 3]).astype(np.float32)


def pose_history(cams, t):
    """[16, 16] float32: world->camera 3x4 of frames t, t-1, ..., t-15 (clamped at 0)."""
    ph = np.zeros((HIST, 16), np.float32)
    for k in range(HIST):
        ph[k, :12] = np.asarray(cams[max(t - k, 0)].Tcw, np.float32)[:3].reshape(-1)
    return ph


def visibility(ctx, cams):
    """Exact cull of every frame: bool [T, C]."""
    import torch

    C = dcg.dcg_chunk_count(ctx)
    out = np.zeros((len(cams), C), bool)
    mask = torch.zeros(C, dtype=torch.uint8, device="cuda")
    for t, c in enumerate(cams):
        dcg.dcg_cull_chunks(ctx, [c], mask)
        out[t] = mask.cpu().numpy().astype(bool)
    return out


class _Ready:
    def __init__(self, p):
        self.p = p

    def result(self):
        return self.p


class _Pending:
    def __init__(self, ev, buf, n):
        self.ev, self.buf, self.n = ev, buf, n

    def result(self):
        self.ev.synchronize()
        return self.buf[: self.n].numpy().copy()


class PrefetchMLP:
    """The MLP plus feature buffers; `bind(ctx)` points it at a chunk table."""

    def __init__(self, ctx=None, max_batch=4096):
        import torch

        self.max_batch = max_batch
        self.m = dcg.dcg_mlp_create(max_batch)
        self.x = torch.zeros((max_batch, 128), dtype=torch.int16, device="cuda")
        self.prob = torch.zeros(max_batch, device="cuda")
        self.coords = None
        if ctx is not None:
            self.bind(ctx)

    def bind(self, ctx):
        import torch

        info = dcg.dcg_chunk_info(ctx)
        self.coords = torch.from_numpy(np.ascontiguousarray(info["coords"])).cuda()
        self.cand = torch.zeros(max(len(info["keys"]), 1), dtype=torch.int32, device="cuda")

    def close(self):
        if self.m is not None:
            dcg.dcg_mlp_destroy(self.m)
            self.m = None

    def score_async(self, ph, cand, chunk_size, stream):
        """Launch the scoring of `cand` on `stream` (features, MLP, copy of the
        probabilities to pinned memory); `.result()` of the returned handle
        waits for that stream only.  One batch (len(cand) <= max_batch)."""
        import torch

        n = len(cand)
        if n == 0 or n > self.max_batch:
            return _Ready(self.score(ph, cand, chunk_size))
        rows = (n + 63) // 64 * 64
        if getattr(self, "prob_h", None) is None:
            self.prob_h = torch.zeros(self.max_batch).pin_memory()
            self.cand_h = torch.zeros(self.max_batch, dtype=torch.int32).pin_memory()
        self.cand_h[:n] = torch.from_numpy(np.ascontiguousarray(cand, np.int32))
        with torch.cuda.stream(stream):
            self.cand[:n].copy_(self.cand_h[:n], non_blocking=True)
            dcg.dcg_mlp_features(ph, self.coords, chunk_size, self.cand, n, rows, self.x, stream=stream)
            dcg.dcg_mlp_forward(self.m, self.x, rows, self.prob, stream=stream)
            self.prob_h[:n].copy_(self.prob[:n], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        return _Pending(ev, self.prob_h, n)

    def score(self, ph, cand, chunk_size):
        import torch

        n = len(cand)
        if n == 0:
            return np.zeros(0, np.float32)
        rows = (n + 63) // 64 * 64
        self.cand[:n].copy_(torch.from_numpy(np.ascontiguousarray(cand, np.int32)))
        out = []
        for r0 in range(0, rows, self.max_batch):
            nb = min(self.max_batch, rows - r0)
            k = max(0, min(n - r0, nb))
            dcg.dcg_mlp_features(ph, self.coords, chunk_size, self.cand[r0:], k, nb, self.x)
            dcg.dcg_mlp_forward(self.m, self.x, nb, self.prob)
            out.append(self.prob[:k].cpu().numpy())
        return np.concatenate(out)


def make_dataset(ctx, cams, chunk_size, radius, max_samples, seed=0):
    """(X dev [N,128] BF16 as int16, y dev [N] float32, N, positive fraction)."""
    import torch

    info = dcg.dcg_chunk_info(ctx)
    coords = torch.from_numpy(np.ascontiguousarray(info["coords"])).cuda()
    vis = visibility(ctx, cams)
    T = len(cams)
    frames = np.arange(HIST - 1, T - HORIZON)
    rng = np.random.default_rng(seed)
    rng.shuffle(frames)
    X = torch.zeros((max_samples + 64, 128), dtype=torch.int16, device="cuda")
    y = np.zeros(max_samples + 64, np.float32)
    cand_dev = torch.zeros(max(len(info["keys"]), 1), dtype=torch.int32, device="cuda")
    n = 0
    for t in frames:
        cand = dcg.dcg_chunks_near(ctx, cam_centre(cams[t]), radius)
        k = min(len(cand), max_samples - n)
        if k <= 0:
            break
        cand = cand[:k]
        fut = vis[t + 1: t + 1 + HORIZON][:, cand].any(0)
        cand_dev[:k].copy_(torch.from_numpy(cand))
        dcg.dcg_mlp_features(pose_history(cams, t), coords, chunk_size, cand_dev, k, k, X[n:])
        y[n:n + k] = fut
        n += k
    return X[:n], torch.from_numpy(y[:n]).cuda(), n, float(y[:n].mean())


def train(pm: PrefetchMLP, X, y, n, epochs=4, batch=2048, lr=1e-3, seed=0):
    """Adam on shuffled mini-batches (row gather kernel); returns mean loss per epoch."""
    import torch

    rng = np.random.default_rng(seed)
    nb = n // batch
    Xs = torch.empty_like(X[: nb * batch])
    ys = torch.empty(nb * batch, device="cuda")
    losses = []
    for _ in range(epochs):
        perm = torch.from_numpy(rng.permutation(n)[: nb * batch].astype(np.int32)).cuda()
        dcg.dcg_mlp_gather_rows(X, y, perm, nb * batch, Xs, ys)
        tot = torch.zeros(1, device="cuda")
        for b in range(nb):
            dcg.dcg_mlp_train_step(pm.m, Xs[b * batch:(b + 1) * batch], ys[b * batch:(b + 1) * batch], batch, lr, tot)
        losses.append(tot.item() / max(nb, 1))
    return losses


def constant_velocity_cams(cams, t, ahead=(5, 10, 15, 20)):
    """Poses extrapolated from the last step's relative motion (a non-learned predictor)."""
    from . import synth

    T1 = np.asarray(cams[t].Tcw, np.float64)
    T0 = np.asarray(cams[max(t - 1, 0)].Tcw, np.float64)
    step = T1 @ np.linalg.inv(T0)  # camera motion of the last frame, world->camera form
    out = []
    for k in ahead:
        Tk = np.linalg.matrix_power(step, k) @ T1
        c = cams[t]
        out.append(synth.Camera(c.fx, c.fy, c.cx, c.cy, c.W, c.H, Tk.astype(np.float32), c.znear, c.zfar))
    return out


class _PendingList:
    def __init__(self, ev, buf, n_h):
        self.ev, self.buf, self.n_h = ev, buf, n_h

    def result(self):
        self.ev.synchronize()
        return self.buf[: int(self.n_h[0])].numpy().copy()


class ConstantVelocity:
    """The non-learned predictor: the exact cull of the poses extrapolated from
    the last step's motion, run like the MLP on a side stream while the frame
    renders (one asynchronous cull of all extrapolated poses; the list comes
    back through pinned memory and is waited for after the frame)."""

    def __init__(self, ctx):
        import torch

        C = max(dcg.dcg_chunk_count(ctx), 1)
        self.list = torch.zeros(C, dtype=torch.int32, device="cuda")
        self.n = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.list_h = torch.zeros(C, dtype=torch.int32).pin_memory()
        self.n_h = torch.zeros(1, dtype=torch.int32).pin_memory()

    def propose_async(self, ctx, cams, t, stream):
        import torch

        with torch.cuda.stream(stream):
            dcg.dcg_cull_chunks_async(ctx, constant_velocity_cams(cams, t), self.list, self.n, stream=stream)
            self.list_h.copy_(self.list, non_blocking=True)
            self.n_h.copy_(self.n, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        return _PendingList(ev, self.list_h, self.n_h)


def run_corridor(ctx, cams, mode, chunk_size, radius, pm: PrefetchMLP | None = None, threshold=0.3, render=None,
                 warm=1, every=1):
    """Map along `cams` one keyframe per step: cull, gather (synchronous loads
    of missing chunks), `render(g, n, cam)`, scatter, then propose prefetches
    ('none' | 'cv' | 'mlp') every `every` steps (a proposal covers the next
    20 frames, so it need not be renewed each frame).  The first `warm` steps
    (the cold start, which no predictor can see coming) are run but not
    counted.  Returns statistics."""
    import torch

    info = dcg.dcg_chunk_info(ctx)
    counts = info["counts"]
    pending = set()  # prefetched, not used yet
    hits = misses = wasted = 0
    hit_g = miss_g = 0
    dcg.dcg_profile(ctx, True)
    dcg.dcg_profile_read(ctx)
    # The phase timers hold a bounded number of intervals between reads (about
    # 22 a step here), so they are read, and summed, every `read_every` steps.
    read_every = 200
    prof = {}

    def read_timers():
        for k, (ms, cnt) in dcg.dcg_profile_read(ctx).items():
            a = prof.setdefault(k, [0.0, 0])
            a[0] += ms
            a[1] += cnt

    side = torch.cuda.Stream()
    cvp = ConstantVelocity(ctx) if mode == "cv" else None
    resident_trace = []  # Gaussians on the device after each step's gather
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for t, cam in enumerate(cams):
        if t == warm:
            torch.cuda.synchronize()
            dcg.dcg_profile_read(ctx)
            hits = misses = wasted = hit_g = miss_g = 0
            resident_trace = []
            e0.record()
        elif t > warm and (t - warm) % read_every == 0:
            read_timers()
        lst = dcg.dcg_cull_chunks(ctx, [cam])
        res = dcg.dcg_chunk_info(ctx)["resident"].astype(bool)
        for c in lst:
            if not res[c]:
                misses += 1
                miss_g += int(counts[c])
                pending.discard(int(c))
            elif int(c) in pending:
                hits += 1
                hit_g += int(counts[c])
                pending.discard(int(c))
        g, n = dcg.dcg_gather_active(ctx, lst)
        resident_trace.append(dcg.dcg_tier_stats(ctx)["resident"])
        # proposals for the coming frames are computed on a side stream while
        # this frame renders (they depend only on poses and residency); both
        # predictors wait for that stream only after the frame is enqueued
        prop = []
        pending_scores = pending_cv = None
        propose = t % every == 0
        if mode == "mlp" and propose:
            cand = dcg.dcg_chunks_near(ctx, cam_centre(cam), radius, only_nonresident=True)
            pending_scores = pm.score_async(pose_history(cams, t), cand, chunk_size, side)
        elif mode == "cv" and propose:
            pending_cv = cvp.propose_async(ctx, cams, t, side)
        if render is not None:
            render(g, n, cam)
        dcg.dcg_scatter_back(ctx, g, n)
        if pending_scores is not None:
            p = pending_scores.result()
            order = np.argsort(-p, kind="stable")
            prop = [int(cand[i]) for i in order if p[i] > threshold]
        elif pending_cv is not None:
            fut = pending_cv.result()
            res = dcg.dcg_chunk_info(ctx)["resident"].astype(bool)
            prop = [int(c) for c in fut if not res[c]]
        if prop:
            before = dcg.dcg_chunk_info(ctx)["resident"].astype(bool)
            dcg.dcg_prefetch(ctx, prop)
            after = dcg.dcg_chunk_info(ctx)["resident"].astype(bool)
            for c in np.nonzero(after & ~before)[0]:
                pending.add(int(c))
            for c in list(pending):
                if not after[c]:
                    pending.discard(c)
                    wasted += 1
    e1.record()
    torch.cuda.synchronize()
    read_timers()
    dcg.dcg_profile(ctx, False)
    wasted += len(pending)
    tr = np.asarray(resident_trace, np.int64)
    return {"mode": mode, "steps": len(cams) - warm, "ms": e0.elapsed_time(e1), "stall_ms": prof["stall"][0],
            "hits": hits, "misses": misses, "wasted_prefetches": wasted,
            "hidden_load_frac": hit_g / max(hit_g + miss_g, 1), "tier": dcg.dcg_tier_stats(ctx),
            "resident_max": int(tr.max()) if tr.size else 0,
            "resident_trace": [int(v) for v in tr[:: max(1, len(tr) // 40)]],
            # device time of each phase per counted step (the phase timers' CUDA events)
            "phases_ms_per_step": {k: round(v[0] / max(len(cams) - warm, 1), 4) for k, v in prof.items() if v[1]}}
