"""Thin ctypes binding of libdcg.so (include/dcg.h) -- argument marshalling only.

Every function below has the name of the C entry point it calls and only
turns torch tensors / numpy arrays / camera objects into pointers and structs.
All computation happens in the CUDA library; if the library is missing or
does not load, importing the functions raises instead of falling back.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# DCG_LIB=checks selects the bounds-check build of the same library (libdcg_checks.so)
LIB_PATH = os.path.join(_HERE, "libdcg_checks.so" if os.environ.get("DCG_LIB") == "checks" else "libdcg.so")

DCG_OK = 0
STATUS = {0: "DCG_OK", 1: "DCG_ERR_ARG", 2: "DCG_ERR_OOM", 3: "DCG_ERR_CUDA", 4: "DCG_ERR_BUDGET",
          5: "DCG_ERR_KEY_RANGE", 6: "DCG_ERR_CAPACITY", 7: "DCG_ERR_TIMEOUT", 8: "DCG_ERR_FAULT", 9: "DCG_ERR_STATE",
          10: "DCG_ERR_BOUNDS"}


class DcgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class dcg_camera(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("W", ctypes.c_int32), ("H", ctypes.c_int32), ("Tcw", ctypes.c_float * 16),
                ("znear", ctypes.c_float), ("zfar", ctypes.c_float)]


class dcg_gaussians(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("stride", ctypes.c_int64), ("sh_degree", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


class dcg_config(ctypes.Structure):
    _fields_ = [("chunk_size", ctypes.c_float), ("sh_degree", ctypes.c_int32), ("device_budget", ctypes.c_int64),
                ("host_capacity", ctypes.c_int64), ("max_chunks", ctypes.c_int32), ("max_views", ctypes.c_int32),
                ("max_active", ctypes.c_int64), ("max_pixels", ctypes.c_int64), ("max_instances", ctypes.c_int64),
                ("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("stage", ctypes.c_int32),
                ("dfar", ctypes.c_float), ("page_gaussians", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("with_moments", ctypes.c_int32)]


_lib = None
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32

_SIGS = {
    "dcg_config_default": (None, [ctypes.POINTER(dcg_config)]),
    "dcg_create": (ctypes.c_int, [ctypes.POINTER(dcg_config), ctypes.POINTER(_P)]),
    "dcg_destroy": (ctypes.c_int, [_P]),
    "dcg_last_error": (ctypes.c_char_p, [_P]),
    "dcg_sync": (ctypes.c_int, [_P, _P]),
    "dcg_chunk_keys": (ctypes.c_int, [_P, _P, _I64, _P, _P]),
    "dcg_chunk_table_update": (ctypes.c_int, [_P, _P, _I64, _I64, _P, _P]),
    "dcg_chunk_count": (_I32, [_P]),
    "dcg_chunk_info": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "dcg_cull_chunks": (ctypes.c_int, [_P, ctypes.POINTER(dcg_camera), _I32, _P, _P, _P, _P]),
    "dcg_gather_active": (ctypes.c_int, [_P, _P, _I32, ctypes.POINTER(dcg_gaussians), ctypes.POINTER(_I64), _P]),
    "dcg_scatter_back": (ctypes.c_int, [_P, ctypes.POINTER(dcg_gaussians), _I64, _P]),
    "dcg_flush": (ctypes.c_int, [_P, _P]),
    "dcg_chunk_read": (ctypes.c_int, [_P, _I32, _P, _I64]),
    "dcg_state_create": (ctypes.c_int, [_P, ctypes.POINTER(_P)]),
    "dcg_state_destroy": (ctypes.c_int, [_P]),
    "dcg_default_state": (_P, [_P]),
    "dcg_render_fwd": (ctypes.c_int, [_P, ctypes.POINTER(dcg_gaussians), _I64, ctypes.POINTER(dcg_camera), _I32, _P, _P,
                                      _P, _P]),
    "dcg_render_bwd": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(dcg_gaussians), _P, _P]),
    "dcg_loss_l1": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.POINTER(dcg_camera), _I32, ctypes.c_float, _P, _P, _P,
                                   _P]),
    "dcg_set_launch": (ctypes.c_int, [_P, _I32, _I32, _I32]),
    "dcg_state_stats": (ctypes.c_int, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I64), _P]),
    "dcg_state_read": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "dcg_profile": (ctypes.c_int, [_P, _I32]),
    "dcg_autotune": (ctypes.c_int, [_P, ctypes.POINTER(dcg_gaussians), _I64, ctypes.POINTER(dcg_camera), _I32, _P, _P,
                                    _P, _P, ctypes.POINTER(dcg_gaussians), _I32, ctypes.POINTER(_I32),
                                    ctypes.POINTER(_I32), ctypes.POINTER(_I32), _P, _P]),
    "dcg_state_evals": (ctypes.c_int, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), _P]),
    "dcg_profile_read": (ctypes.c_int, [_P, _P, _P]),
    "dcg_launch_count": (ctypes.c_uint64, []),
    "dcg_window_capture": (ctypes.c_int, [_P, ctypes.POINTER(dcg_gaussians), _I64, ctypes.POINTER(dcg_camera), _I32,
                                          _P, _P, _P, _P, ctypes.c_float, ctypes.c_float, _P, _P, _P,
                                          ctypes.POINTER(dcg_gaussians), _P, _P]),
    "dcg_loss": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.POINTER(dcg_camera), _I32, ctypes.c_float, ctypes.c_float,
                                _P, _P, _P, _P]),
    "dcg_window_run": (ctypes.c_int, [_P, ctypes.POINTER(dcg_camera), _I32, _P]),
    "dcg_state_generation": (_I64, [_P]),
    "dcg_prefetch": (ctypes.c_int, [_P, _P, _I32, ctypes.POINTER(_I32), _P]),
    "dcg_chunks_near": (ctypes.c_int, [_P, _P, ctypes.c_float, _I32, _P, ctypes.POINTER(_I32)]),
    "dcg_mlp_create": (ctypes.c_int, [_I32, ctypes.POINTER(_P)]),
    "dcg_mlp_destroy": (ctypes.c_int, [_P]),
    "dcg_mlp_num_params": (_I32, []),
    "dcg_mlp_set_params": (ctypes.c_int, [_P, _P]),
    "dcg_mlp_get_params": (ctypes.c_int, [_P, _P]),
    "dcg_mlp_forward": (ctypes.c_int, [_P, _P, _I32, _P, _P]),
    "dcg_mlp_grads": (ctypes.c_int, [_P, _P, _P, _I32, _P, _P, _P]),
    "dcg_mlp_train_step": (ctypes.c_int, [_P, _P, _P, _I32, ctypes.c_float, _P, _P]),
    "dcg_mlp_features": (ctypes.c_int, [_P, _P, ctypes.c_float, _P, _I32, _I32, _P, _P]),
    "dcg_mlp_gather_rows": (ctypes.c_int, [_P, _P, _P, _I32, _P, _P, _P]),
    "dcg_tier_stats": (ctypes.c_int, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                                      ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "dcg_chunk_read_moments": (ctypes.c_int, [_P, _I32, _P, _P, _I64]),
    "dcg_active_moments": (ctypes.c_int, [_P, _P, _P]),
    "dcg_adam_step": (ctypes.c_int, [_P, _P, _P, _I64, _P, ctypes.c_float, ctypes.c_float, ctypes.c_float, _I64,
                                     _P]),
    "dcg_loop_closure": (ctypes.c_int, [_P, ctypes.POINTER(dcg_camera), _P, _I32, ctypes.POINTER(_I64),
                                        ctypes.POINTER(_I64), _P]),
    "dcg_reset_active": (ctypes.c_int, [_P, _P, _I64, ctypes.c_float, _P]),
    "dcg_log_sample": (ctypes.c_int, [_P, _P, _P, _I32, _I32, ctypes.c_float, _P, _P, _P, _I32, ctypes.POINTER(_I32),
                                      _P]),
    "dcg_backproject": (ctypes.c_int, [_P, _P, _I32, _P, _P, ctypes.POINTER(dcg_camera), ctypes.c_float, _P, _I64,
                                       _P]),
    "dcg_active_map": (ctypes.c_int, [_P, _P, _P, _P]),
    "dcg_log_sample_views": (ctypes.c_int, [_P, ctypes.POINTER(dcg_camera), _I32, _P, _P, ctypes.c_float, _P, _P, _P,
                                            _I64, _P, ctypes.POINTER(_I64), _P]),
    "dcg_backproject_views": (ctypes.c_int, [_P, _P, _I64, _P, _P, ctypes.POINTER(dcg_camera), _I32, ctypes.c_float,
                                             _P, _I64, _P]),
    "dcg_cull_chunks_noalloc": (ctypes.c_int, [_P, _I32, ctypes.c_float, ctypes.c_float, ctypes.POINTER(dcg_camera),
                                               _I32, _P, _P, _P, _P]),
    "dcg_inject_fault": (ctypes.c_int, [_P, _I32, _I32]),
    "dcg_mlp_set_gemm": (ctypes.c_int, [_P, _I32]),
    "dcg_cull_chunks_async": (ctypes.c_int, [_P, ctypes.POINTER(dcg_camera), _I32, _P, _P, _P, _P]),
    "dcg_fault_parse": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
}

FAULTS = {"none": 0, "h2d_fail": 1, "short_copy": 2, "budget": 3}
FLAG_VERIFY_LOADS = 4  # dcg_config.flags bit 2: chunk loads checked by checksum

PHASES = ["cull", "gather", "preprocess_fwd", "binning", "blend_fwd", "loss", "blend_bwd", "preprocess_bwd", "scatter",
          "stall", "log_sample", "loop_closure"]


def lib():
    """Load libdcg.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} not built; run paper_2511_23030_b300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


# --------------------------------------------------------------------------- marshalling helpers
def ptr(x):
    """Device or host pointer of a torch tensor / numpy array (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(x.data_ptr())


def stream_ptr(stream=None):
    import torch

    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def make_cameras(cams):
    arr = (dcg_camera * len(cams))()
    for k, c in enumerate(cams):
        a = arr[k]
        a.fx, a.fy, a.cx, a.cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
        a.W, a.H = int(c.W), int(c.H)
        T = np.asarray(c.Tcw, np.float32).reshape(16)
        for j in range(16):
            a.Tcw[j] = float(T[j])
        a.znear, a.zfar = float(c.znear), float(c.zfar)
    return arr


def gaussians(t, deg: int, n: int | None = None) -> dcg_gaussians:
    """View of a planar [F, stride] float32 CUDA tensor."""
    g = dcg_gaussians()
    g.data = t.data_ptr()
    g.stride = t.stride(0)
    g.sh_degree = deg
    return g


class _CudaArray:
    """Exposes a device pointer through __cuda_array_interface__ (zero copy)."""

    def __init__(self, data: int, shape, strides_bytes, typestr="<f4"):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(data), False),
                                         "strides": tuple(strides_bytes), "version": 3}


def active_tensor(g: dcg_gaussians, n: int, F: int):
    """Torch view [F, n] of a library-owned planar buffer (e.g. the active set)."""
    import torch

    return torch.as_tensor(_CudaArray(g.data, (F, n), (4 * g.stride, 4)), device="cuda")


def check(ctx, status: int):
    if status != DCG_OK:
        msg = lib().dcg_last_error(ctx)
        raise DcgError(status, msg.decode() if msg else "")


def config(**kw) -> dcg_config:
    c = dcg_config()
    lib().dcg_config_default(ctypes.byref(c))
    for k, v in kw.items():
        if not hasattr(c, k):
            raise KeyError(k)
        setattr(c, k, v)
    return c


# --------------------------------------------------------------------------- C entry points
def dcg_create(cfg: dcg_config):
    h = ctypes.c_void_p()
    st = lib().dcg_create(ctypes.byref(cfg), ctypes.byref(h))
    if st != DCG_OK:
        raise DcgError(st, "dcg_create failed")
    return h


def dcg_destroy(ctx):
    check(ctx, lib().dcg_destroy(ctx))


def dcg_sync(ctx, stream=None):
    check(ctx, lib().dcg_sync(ctx, stream_ptr(stream)))


def dcg_chunk_keys(ctx, means, keys_out, stream=None):
    check(ctx, lib().dcg_chunk_keys(ctx, ptr(means), means.shape[0], ptr(keys_out), stream_ptr(stream)))


def dcg_chunk_table_update(ctx, params, n, keys_out=None, stream=None):
    check(ctx, lib().dcg_chunk_table_update(ctx, ptr(params), params.stride(0), n, ptr(keys_out), stream_ptr(stream)))


def dcg_chunk_count(ctx) -> int:
    return int(lib().dcg_chunk_count(ctx))


def dcg_chunk_info(ctx):
    C = dcg_chunk_count(ctx)
    coords = np.zeros((C, 3), np.int32)
    keys = np.zeros(C, np.uint64)
    counts = np.zeros(C, np.int64)
    res = np.zeros(C, np.uint8)
    last = np.zeros(C, np.int64)
    check(ctx, lib().dcg_chunk_info(ctx, ptr(coords), ptr(keys), ptr(counts), ptr(res), ptr(last)))
    return dict(coords=coords, keys=keys, counts=counts, resident=res, last_access=last)


def dcg_cull_chunks(ctx, cams, mask_out=None, stream=None):
    arr = make_cameras(cams)
    C = dcg_chunk_count(ctx)
    lst = np.zeros(max(C, 1), np.int32)
    n = np.zeros(1, np.int32)
    check(ctx, lib().dcg_cull_chunks(ctx, arr, len(cams), ptr(mask_out), ptr(lst), ptr(n), stream_ptr(stream)))
    return lst[: int(n[0])].copy()


def dcg_gather_active(ctx, chunk_list, stream=None):
    lst = np.ascontiguousarray(chunk_list, np.int32)
    g = dcg_gaussians()
    n = _I64()
    check(ctx, lib().dcg_gather_active(ctx, ptr(lst), len(lst), ctypes.byref(g), ctypes.byref(n), stream_ptr(stream)))
    return g, int(n.value)


def dcg_scatter_back(ctx, active: dcg_gaussians, n: int, stream=None):
    check(ctx, lib().dcg_scatter_back(ctx, ctypes.byref(active), n, stream_ptr(stream)))


def dcg_flush(ctx, stream=None):
    check(ctx, lib().dcg_flush(ctx, stream_ptr(stream)))


def dcg_chunk_read(ctx, chunk: int, n: int, F: int) -> np.ndarray:
    out = np.zeros((F, n), np.float32)
    check(ctx, lib().dcg_chunk_read(ctx, chunk, ptr(out), n))
    return out


def dcg_chunk_read_moments(ctx, chunk: int, n: int, F: int):
    """Adam moments (m, v) of a chunk from the host tier, each [F, n] float32."""
    m = np.zeros((F, n), np.float32)
    v = np.zeros((F, n), np.float32)
    check(ctx, lib().dcg_chunk_read_moments(ctx, chunk, ptr(m), ptr(v), n))
    return m, v


def dcg_active_moments(ctx):
    """Views (m, v) of the active set's Adam moments (library-owned)."""
    m, v = dcg_gaussians(), dcg_gaussians()
    check(ctx, lib().dcg_active_moments(ctx, ctypes.byref(m), ctypes.byref(v)))
    return m, v


def dcg_adam_step(ctx, params: dcg_gaussians, grads: dcg_gaussians, n: int, lr, beta1=0.9, beta2=0.999, eps=1e-15,
                  step=1, stream=None):
    """One Adam step over the gathered active set; lr: one learning rate per component (F values)."""
    lr_a = np.ascontiguousarray(np.asarray(lr, np.float32).reshape(-1))
    check(ctx, lib().dcg_adam_step(ctx, ctypes.byref(params), ctypes.byref(grads), n, ptr(lr_a), float(beta1),
                                   float(beta2), float(eps), int(step), stream_ptr(stream)))


def dcg_loop_closure(ctx, keyframes, corrections, stream=None):
    """Loop-closure correction; corrections: K rigid 4x4 transforms. Returns (n_transformed, n_moved)."""
    arr = make_cameras(keyframes)
    C = np.ascontiguousarray(np.asarray(corrections, np.float32).reshape(len(keyframes), 16))
    nt, nm = _I64(), _I64()
    check(ctx, lib().dcg_loop_closure(ctx, arr, ptr(C), len(keyframes), ctypes.byref(nt), ctypes.byref(nm),
                                      stream_ptr(stream)))
    return int(nt.value), int(nm.value)


def dcg_reset_active(ctx, params: dcg_gaussians, n: int, max_opacity=0.01, stream=None):
    check(ctx, lib().dcg_reset_active(ctx, ctypes.byref(params), n, float(max_opacity), stream_ptr(stream)))


def dcg_log_sample(ctx, image, rendered, W: int, H: int, kappa: float, u, idx_out, ps_out=None, stream=None) -> int:
    """Eq. 1 penalty sampling of one view; returns the number of sampled pixels written to idx_out."""
    n = _I32()
    check(ctx, lib().dcg_log_sample(ctx, ptr(image), ptr(rendered), W, H, float(kappa), ptr(u), ptr(ps_out),
                                    ptr(idx_out), idx_out.numel(), ctypes.byref(n), stream_ptr(stream)))
    return int(n.value)


def dcg_active_map(ctx, chunk_out=None, row_out=None, stream=None):
    """Chunk index and row within the chunk of every row of the last gathered active set."""
    check(ctx, lib().dcg_active_map(ctx, ptr(chunk_out), ptr(row_out), stream_ptr(stream)))


def dcg_log_sample_views(ctx, cams, image, rendered, kappa: float, u, idx_out, ps_out=None, stream=None):
    """Eq. 1 penalty sampling of a window of views at once; returns (total, per-view counts) with the
    sampled window indices written to idx_out."""
    arr = make_cameras(cams)
    n = _I64()
    counts = np.zeros(len(cams), np.int64)
    check(ctx, lib().dcg_log_sample_views(ctx, arr, len(cams), ptr(image), ptr(rendered), float(kappa), ptr(u),
                                          ptr(ps_out), ptr(idx_out), idx_out.numel(), ptr(counts), ctypes.byref(n),
                                          stream_ptr(stream)))
    return int(n.value), counts


def dcg_backproject_views(ctx, idx, n: int, depth, image, cams, opacity_logit: float, params_out, stream=None):
    arr = make_cameras(cams)
    check(ctx, lib().dcg_backproject_views(ctx, ptr(idx), n, ptr(depth), ptr(image), arr, len(cams),
                                           float(opacity_logit), ptr(params_out), params_out.stride(0),
                                           stream_ptr(stream)))


def dcg_backproject(ctx, idx, n: int, depth, image, cam, opacity_logit: float, params_out, stream=None):
    arr = make_cameras([cam])
    check(ctx, lib().dcg_backproject(ctx, ptr(idx), n, ptr(depth), ptr(image), arr, float(opacity_logit),
                                     ptr(params_out), params_out.stride(0), stream_ptr(stream)))


def dcg_state_create(ctx):
    h = ctypes.c_void_p()
    check(ctx, lib().dcg_state_create(ctx, ctypes.byref(h)))
    return h


def dcg_state_destroy(state):
    lib().dcg_state_destroy(state)


def dcg_render_fwd(ctx, g: dcg_gaussians, n: int, cams, rgb, depth, state=None, stream=None):
    arr = make_cameras(cams)
    check(ctx, lib().dcg_render_fwd(ctx, ctypes.byref(g), n, arr, len(cams), ptr(rgb), ptr(depth), state,
                                    stream_ptr(stream)))


def dcg_render_bwd(ctx, dL_drgb, dL_ddepth, grads: dcg_gaussians, dL_dpose=None, state=None, stream=None):
    check(ctx, lib().dcg_render_bwd(ctx, state, ptr(dL_drgb), ptr(dL_ddepth), ctypes.byref(grads), ptr(dL_dpose),
                                    stream_ptr(stream)))


def dcg_loss_l1(ctx, rgb, depth, tgt_rgb, tgt_depth, cams, lam, dL_drgb, dL_ddepth, loss, stream=None):
    arr = make_cameras(cams)
    check(ctx, lib().dcg_loss_l1(ctx, ptr(rgb), ptr(depth), ptr(tgt_rgb), ptr(tgt_depth), arr, len(cams),
                                 float(lam), ptr(dL_drgb), ptr(dL_ddepth), ptr(loss), stream_ptr(stream)))


def dcg_loss(ctx, rgb, depth, tgt_rgb, tgt_depth, cams, lambda_s, lambda_depth, dL_drgb, dL_ddepth, loss, stream=None):
    arr = make_cameras(cams)
    check(ctx, lib().dcg_loss(ctx, ptr(rgb), ptr(depth), ptr(tgt_rgb), ptr(tgt_depth), arr, len(cams), float(lambda_s),
                              float(lambda_depth), ptr(dL_drgb), ptr(dL_ddepth), ptr(loss), stream_ptr(stream)))


def dcg_set_launch(ctx, tile_w: int, tile_h: int, stage: int):
    check(ctx, lib().dcg_set_launch(ctx, tile_w, tile_h, stage))


def dcg_default_state(ctx):
    return ctypes.c_void_p(lib().dcg_default_state(ctx))


def dcg_state_stats(ctx, state=None, stream=None):
    a, b, c = _I64(), _I64(), _I64()
    st = state if state is not None else dcg_default_state(ctx)
    check(ctx, lib().dcg_state_stats(st, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), stream_ptr(stream)))
    return int(a.value), int(b.value), int(c.value)


def dcg_state_read(ctx, state, n_views, n, n_pix, stream=None):
    """Returns dict(ranges [T,2] u32, ids [K] u32, masks [K] u16, depth [V*n] f32, rect [V*n,4] i32, T [P],
    n_contrib [P])."""
    nv, K, T = dcg_state_stats(ctx, state, stream)
    ranges = np.zeros((T, 2), np.uint32)
    ids = np.zeros(max(K, 1), np.uint32)
    masks = np.zeros(max(K, 1), np.uint16)
    depth = np.zeros(max(n_views * n, 1), np.float32)
    rect = np.zeros((max(n_views * n, 1), 4), np.int32)
    Tf = np.zeros(max(n_pix, 1), np.float32)
    nc = np.zeros(max(n_pix, 1), np.int32)
    st = state if state is not None else dcg_default_state(ctx)
    check(ctx, lib().dcg_state_read(st, ptr(ranges), ptr(ids), ptr(masks), ptr(depth), ptr(rect), ptr(Tf), ptr(nc),
                                    stream_ptr(stream)))
    return dict(ranges=ranges, ids=ids[:K], masks=masks[:K], depth=depth[: n_views * n], rect=rect[: n_views * n],
                T=Tf[:n_pix], n_contrib=nc[:n_pix], n_visible=nv)


def dcg_profile(ctx, enable: bool):
    check(ctx, lib().dcg_profile(ctx, 1 if enable else 0))


def dcg_profile_read(ctx):
    ms = np.zeros(len(PHASES), np.float32)
    cnt = np.zeros(len(PHASES), np.int32)
    check(ctx, lib().dcg_profile_read(ctx, ptr(ms), ptr(cnt)))
    return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(PHASES)}


def dcg_launch_count() -> int:
    return int(lib().dcg_launch_count())


def dcg_state_evals(ctx, state=None, stream=None):
    """(evaluations, composited pairs) of the last forward blend."""
    v, b = _I64(), _I64()
    st = state if state is not None else dcg_default_state(ctx)
    check(ctx, lib().dcg_state_evals(st, ctypes.byref(v), ctypes.byref(b), stream_ptr(stream)))
    return int(v.value), int(b.value)


TUNE_TILES = [(16, 16), (32, 16), (32, 32)]
TUNE_STAGES = [64, 96, 128, 192, 256, 32, 16]  # 32: warp-per-block kernels, 16: half-warp kernels


def dcg_autotune(ctx, g: dcg_gaussians, n: int, cams, rgb, depth, dL_drgb, dL_ddepth, grads: dcg_gaussians, reps=3,
                 stream=None):
    arr = make_cameras(cams)
    tw, th, sg = _I32(), _I32(), _I32()
    ns = len(TUNE_STAGES)
    ms = np.zeros(len(TUNE_TILES) * ns, np.float32)
    check(ctx, lib().dcg_autotune(ctx, ctypes.byref(g), n, arr, len(cams), ptr(rgb), ptr(depth), ptr(dL_drgb),
                                  ptr(dL_ddepth), ctypes.byref(grads), reps, ctypes.byref(tw), ctypes.byref(th),
                                  ctypes.byref(sg), ptr(ms), stream_ptr(stream)))
    table = {f"{TUNE_TILES[i // ns][0]}x{TUNE_TILES[i // ns][1]}/{TUNE_STAGES[i % ns]}": round(float(ms[i]), 4)
             for i in range(len(ms))}
    return {"tile": [tw.value, th.value], "stage": sg.value, "ms": table}


def dcg_cull_chunks_noalloc(coords, chunk_size: float, dfar: float, cams, mask_out, list_out, n_out, stream=None):
    """Allocation-free cull: coords (dev int32 [C,3]), outputs on the device."""
    arr = make_cameras(cams)
    st = lib().dcg_cull_chunks_noalloc(ptr(coords), int(coords.shape[0]), float(chunk_size), float(dfar), arr,
                                       len(cams), ptr(mask_out), ptr(list_out), ptr(n_out), stream_ptr(stream))
    if st != DCG_OK:
        raise DcgError(st, "dcg_cull_chunks_noalloc failed")


def dcg_window_capture(ctx, g: dcg_gaussians, n: int, cams, rgb, depth, tgt_rgb, tgt_depth, lam, dL_drgb, dL_ddepth,
                       loss, grads: dcg_gaussians, dL_dpose=None, stream=None, lambda_s=0.0):
    arr = make_cameras(cams)
    check(ctx, lib().dcg_window_capture(ctx, ctypes.byref(g), n, arr, len(cams), ptr(rgb), ptr(depth), ptr(tgt_rgb),
                                        ptr(tgt_depth), float(lam), float(lambda_s), ptr(dL_drgb), ptr(dL_ddepth),
                                        ptr(loss), ctypes.byref(grads), ptr(dL_dpose), stream_ptr(stream)))


def dcg_window_run(ctx, cams, stream=None):
    arr = make_cameras(cams)
    check(ctx, lib().dcg_window_run(ctx, arr, len(cams), stream_ptr(stream)))


def dcg_state_generation(state) -> int:
    return int(lib().dcg_state_generation(state))


def dcg_prefetch(ctx, chunk_list, stream=None) -> int:
    lst = np.ascontiguousarray(chunk_list, np.int32)
    k = _I32()
    check(ctx, lib().dcg_prefetch(ctx, ptr(lst), len(lst), ctypes.byref(k), stream_ptr(stream)))
    return int(k.value)


def dcg_tier_stats(ctx) -> dict:
    v = [_I64() for _ in range(5)]
    check(ctx, lib().dcg_tier_stats(ctx, *[ctypes.byref(x) for x in v]))
    return dict(zip(["loads", "evictions", "bytes_h2d", "bytes_d2h", "resident"], [int(x.value) for x in v]))


# ------------------------------------------------------------------ prefetch MLP
def _mlp_check(st, what):
    if st != DCG_OK:
        raise DcgError(st, what)


def dcg_mlp_create(max_batch: int):
    h = ctypes.c_void_p()
    _mlp_check(lib().dcg_mlp_create(max_batch, ctypes.byref(h)), "dcg_mlp_create")
    return h


def dcg_mlp_destroy(m):
    _mlp_check(lib().dcg_mlp_destroy(m), "dcg_mlp_destroy")


def dcg_mlp_num_params() -> int:
    return int(lib().dcg_mlp_num_params())


def dcg_mlp_set_params(m, params: np.ndarray):
    p = np.ascontiguousarray(params, np.float32)
    assert p.size == dcg_mlp_num_params()
    _mlp_check(lib().dcg_mlp_set_params(m, ptr(p)), "dcg_mlp_set_params")


def dcg_mlp_get_params(m) -> np.ndarray:
    p = np.zeros(dcg_mlp_num_params(), np.float32)
    _mlp_check(lib().dcg_mlp_get_params(m, ptr(p)), "dcg_mlp_get_params")
    return p


def dcg_mlp_forward(m, x, B, prob, stream=None):
    _mlp_check(lib().dcg_mlp_forward(m, ptr(x), B, ptr(prob), stream_ptr(stream)), "dcg_mlp_forward")


def dcg_mlp_grads(m, x, y, B, grads, loss, stream=None):
    _mlp_check(lib().dcg_mlp_grads(m, ptr(x), ptr(y), B, ptr(grads), ptr(loss), stream_ptr(stream)), "dcg_mlp_grads")


def dcg_mlp_train_step(m, x, y, B, lr, loss, stream=None):
    _mlp_check(lib().dcg_mlp_train_step(m, ptr(x), ptr(y), B, float(lr), ptr(loss), stream_ptr(stream)),
               "dcg_mlp_train_step")


def dcg_mlp_features(pose_hist: np.ndarray, coords, chunk_size, cand, n_cand, n_rows, x, stream=None):
    ph = np.ascontiguousarray(pose_hist, np.float32).reshape(16, 16)
    _mlp_check(lib().dcg_mlp_features(ptr(ph), ptr(coords), float(chunk_size), ptr(cand), n_cand, n_rows, ptr(x),
                                      stream_ptr(stream)), "dcg_mlp_features")


def dcg_mlp_gather_rows(x, y, perm, n, x_out, y_out, stream=None):
    _mlp_check(lib().dcg_mlp_gather_rows(ptr(x), ptr(y), ptr(perm), n, ptr(x_out), ptr(y_out), stream_ptr(stream)),
               "dcg_mlp_gather_rows")


def dcg_chunks_near(ctx, p, radius: float, only_nonresident: bool = False) -> np.ndarray:
    C = dcg_chunk_count(ctx)
    out = np.zeros(max(C, 1), np.int32)
    k = _I32()
    pp = np.ascontiguousarray(p, np.float32)
    check(ctx, lib().dcg_chunks_near(ctx, ptr(pp), float(radius), int(only_nonresident), ptr(out), ctypes.byref(k)))
    return out[: k.value].copy()


def dcg_inject_fault(ctx, kind, skip: int = 0):
    """Arm one host-side fault of the chunk tier (kind: name or DCG_FAULT_* value)."""
    k = FAULTS[kind] if isinstance(kind, str) else int(kind)
    check(ctx, lib().dcg_inject_fault(ctx, k, int(skip)))


def dcg_fault_parse(spec: str):
    """(kind, skip) of a DCG_FAULT specification; DcgError if it is malformed."""
    k, n = ctypes.c_int32(), ctypes.c_int32()
    st = lib().dcg_fault_parse(spec.encode(), ctypes.byref(k), ctypes.byref(n))
    if st != DCG_OK:
        raise DcgError(st, f"bad fault specification {spec!r}")
    return k.value, n.value


def dcg_cull_chunks_async(ctx, cams, list_out, n_out, mask_out=None, stream=None):
    """Cull left on the device (list_out: dev int32 [chunk count], n_out: dev int32 [1])."""
    arr = make_cameras(cams)
    check(ctx, lib().dcg_cull_chunks_async(ctx, arr, len(cams), ptr(mask_out), ptr(list_out), ptr(n_out),
                                           stream_ptr(stream)))


MLP_GEMM = {"tcgen05": 0, "mma_sync": 1}


def dcg_mlp_set_gemm(m, kind: str):
    """Select the MLP's GEMM kernels: "tcgen05" (TMA + tcgen05.mma, the default on sm_100+) or "mma_sync"."""
    st = lib().dcg_mlp_set_gemm(m, MLP_GEMM[kind])
    if st != DCG_OK:
        raise DcgError(st, "dcg_mlp_set_gemm failed")
