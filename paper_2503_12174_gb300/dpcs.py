"""Python binding of libdpcs (include/dpcs.h).

Functions named ``dpcs_*`` map one-to-one onto the C ABI and only marshal
arguments.  ``Context`` wraps them for PyTorch tensors: it checks device,
dtype, shape and contiguity, passes raw device pointers and the current CUDA
stream, and raises ``DPCSError`` on a non-zero status.  Every step of the
path runs in the library's kernels; if the library cannot be loaded this
module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

DPCS_OK = 0
DPCS_ERR_INVALID_ARG = -1
DPCS_ERR_OOM = -2
DPCS_ERR_CUDA = -3
DPCS_ERR_DEVICE_CHECK = -4
DPCS_ERR_TRAVERSAL_LIMIT = -5
DPCS_ERR_TIMEOUT = -6
DPCS_ERR_BUSY = -7
DPCS_ERR_NOT_FOUND = -8
DPCS_MAX_BOUNCES = 8
DPCS_ACCUM_F32 = 0
DPCS_ACCUM_F64 = 1
DPCS_PATH_MEGAKERNEL = 0
DPCS_PATH_WAVEFRONT = 1
DPCS_BVH_LBVH = 0
DPCS_BVH_PLOC = 1

EXPORTED = [
    "dpcs_create", "dpcs_destroy", "dpcs_last_error", "dpcs_sync", "dpcs_memory_used", "dpcs_launch_count",
    "dpcs_scene_upload", "dpcs_scene_free", "dpcs_scene_export", "dpcs_trace", "dpcs_render",
    "dpcs_render_backward", "dpcs_l2_loss", "dpcs_adam", "dpcs_timing_enable", "dpcs_timing_read",
    "dpcs_counters_read", "dpcs_debug_set_visit_cap", "dpcs_render_noalloc", "dpcs_serve_create", "dpcs_serve_destroy", "dpcs_serve_add_scene",
    "dpcs_serve_submit", "dpcs_serve_step", "dpcs_serve_query", "dpcs_serve_drain", "dpcs_serve_stats_get",
    "dpcs_gbuffer", "dpcs_denoise", "dpcs_denoise_backward",
    "dpcs_l1_loss", "dpcs_tv_loss", "dpcs_scene_update", "dpcs_render_loss_backward", "dpcs_render_keep",
    "dpcs_render_backward_kept", "dpcs_render_principled", "dpcs_render_backward_principled",
    "dpcs_scene_transform", "dpcs_render_loss_backward_principled", "dpcs_render_keep_principled",
    "dpcs_render_backward_kept_principled", "dpcs_set_grad_accum", "dpcs_set_render_path", "dpcs_pose_backward",
    "dpcs_set_bvh_builder", "dpcs_pose_backward_principled",
]

DPCS_REQ_RELIGHT = 0
DPCS_REQ_COMPENSATE = 1
DPCS_REQ_WAITING = 0
DPCS_REQ_ACTIVE = 1
DPCS_REQ_DONE = 2
DPCS_REQ_FAILED = -1


class DPCSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"dpcs status {status}: {msg}")
        self.status = status


class DpcsParams(ctypes.Structure):
    _fields_ = [("gamma_p", ctypes.c_float * 3), ("gain_p", ctypes.c_float),
                ("gamma_c", ctypes.c_float * 3), ("gain_c", ctypes.c_float),
                ("wb", ctypes.c_float * 3), ("k_proj", ctypes.c_float),
                ("ks", ctypes.c_float), ("f0", ctypes.c_float),
                ("rr_start", ctypes.c_int32), ("rr_q", ctypes.c_float),
                ("clip", ctypes.c_float), ("jitter", ctypes.c_int32)]


class DpcsMaterial(ctypes.Structure):
    """dpcs_material: device pointers of the principled maps (NULL = absent)."""
    _fields_ = [("albedo", ctypes.c_void_p), ("rough", ctypes.c_void_p), ("metallic", ctypes.c_void_p),
                ("normal", ctypes.c_void_p), ("Ht", ctypes.c_int32), ("Wt", ctypes.c_int32)]


class DpcsView(ctypes.Structure):
    _fields_ = [("Kc", ctypes.c_float * 9), ("Hc", ctypes.c_int32), ("Wc", ctypes.c_int32),
                ("Kp", ctypes.c_float * 9), ("Rp", ctypes.c_float * 9), ("tp", ctypes.c_float * 3),
                ("Hp", ctypes.c_int32), ("Wp", ctypes.c_int32)]


class DpcsServeConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_active", ctypes.c_int32), ("max_inflight", ctypes.c_int32),
                ("samples_per_iteration", ctypes.c_int64), ("quantum_samples", ctypes.c_int64),
                ("policy", ctypes.c_int32), ("pad", ctypes.c_int32), ("relight_slack", ctypes.c_double),
                ("compensation_slack", ctypes.c_double), ("est_samples_per_s", ctypes.c_double),
                ("compensation_share", ctypes.c_double)]


DPCS_SERVE_DEADLINE = 0
DPCS_SERVE_FIXED_SHARE = 1
DPCS_SERVE_QUANTA_DEADLINE = 2


class DpcsRequest(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("scene", ctypes.c_int32), ("Hc", ctypes.c_int32), ("Wc", ctypes.c_int32),
                ("spp", ctypes.c_int32), ("seed", ctypes.c_uint64), ("steps", ctypes.c_int32), ("lr", ctypes.c_float),
                ("Ip", ctypes.c_void_p), ("target", ctypes.c_void_p), ("Ic_out", ctypes.c_void_p),
                ("Ip_out", ctypes.c_void_p)]


class DpcsServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("waiting", ctypes.c_int64), ("active", ctypes.c_int64), ("iterations", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("memory_used", ctypes.c_size_t),
                ("memory_high_water", ctypes.c_size_t)]


class DpcsDenoiseParams(ctypes.Structure):
    _fields_ = [("radius", ctypes.c_int32), ("sigma_s", ctypes.c_float), ("sigma_albedo", ctypes.c_float),
                ("sigma_normal", ctypes.c_float), ("sigma_depth", ctypes.c_float)]


def make_denoise_params(radius: int = 5, sigma_s: float = 2.0, sigma_albedo: float = 0.1, sigma_normal: float = 0.3,
                        sigma_depth: float = 0.1) -> DpcsDenoiseParams:
    return DpcsDenoiseParams(int(radius), float(sigma_s), float(sigma_albedo), float(sigma_normal), float(sigma_depth))


_lib = None
_lib_path = None

_P = ctypes.c_void_p
_SIGS = {
    "dpcs_create": (ctypes.c_int32, [ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(_P)]),
    "dpcs_destroy": (ctypes.c_int32, [_P]),
    "dpcs_last_error": (ctypes.c_char_p, [_P]),
    "dpcs_sync": (ctypes.c_int32, [_P, _P]),
    "dpcs_memory_used": (ctypes.c_size_t, [_P]),
    "dpcs_launch_count": (ctypes.c_uint64, [_P]),
    "dpcs_scene_upload": (ctypes.c_int32, [_P, _P, ctypes.c_int32, _P, ctypes.c_int32, _P, _P,
                                           ctypes.POINTER(ctypes.c_uint64)]),
    "dpcs_scene_free": (ctypes.c_int32, [_P, ctypes.c_uint64]),
    "dpcs_scene_update": (ctypes.c_int32, [_P, ctypes.c_uint64, _P, ctypes.c_int32, _P]),
    "dpcs_scene_transform": (ctypes.c_int32, [_P, ctypes.c_uint64, _P, _P, _P]),
    "dpcs_scene_export": (ctypes.c_int32, [_P, ctypes.c_uint64, _P, _P, _P, _P]),
    "dpcs_trace": (ctypes.c_int32, [_P, ctypes.c_uint64, _P, _P, ctypes.c_int64, _P, _P, _P]),
    "dpcs_render": (ctypes.c_int32, [_P, ctypes.c_uint64, _P, _P, ctypes.c_int32, ctypes.c_int32, _P,
                                     ctypes.POINTER(DpcsView), ctypes.POINTER(DpcsParams), ctypes.c_int32,
                                     ctypes.c_int32, ctypes.c_uint64, _P, _P, _P]),
    "dpcs_render_noalloc": (ctypes.c_int32, [_P, ctypes.c_uint64, _P, _P, ctypes.c_int32, ctypes.c_int32, _P,
                                             ctypes.POINTER(DpcsView), ctypes.POINTER(DpcsParams), ctypes.c_int32,
                                             ctypes.c_int32, ctypes.c_uint64, _P, _P, _P]),
    "dpcs_render_keep": (ctypes.c_int32, [_P, ctypes.c_uint64, _P, _P, ctypes.c_int32, ctypes.c_int32, _P,
                                          ctypes.POINTER(DpcsView), ctypes.POINTER(DpcsParams), ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_uint64, _P, _P, _P]),
    "dpcs_render_backward_kept": (ctypes.c_int32, [_P, ctypes.c_uint64, _P, _P, ctypes.c_int32, ctypes.c_int32, _P,
                                                   ctypes.POINTER(DpcsView), ctypes.POINTER(DpcsParams),
                                                   ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, _P, _P, _P, _P, _P,
                                                   _P, _P, _P]),
    "dpcs_render_backward": (ctypes.c_int32, [_P, ctypes.c_uint64, _P, _P, ctypes.c_int32, ctypes.c_int32, _P,
                                              ctypes.POINTER(DpcsView), ctypes.POINTER(DpcsParams), ctypes.c_int32,
                                              ctypes.c_int32, ctypes.c_uint64, _P, _P, _P, _P, _P, _P, _P, _P]),
    "dpcs_pose_backward": (ctypes.c_int32, [_P, ctypes.c_uint64, _P, _P, ctypes.c_int32, ctypes.c_int32, _P,
                                            ctypes.POINTER(DpcsView), ctypes.POINTER(DpcsParams), ctypes.c_int32,
                                            ctypes.c_int32, ctypes.c_uint64, _P, _P, _P, ctypes.c_int32,
                                            ctypes.c_int32, _P, _P]),
    "dpcs_pose_backward_principled": (ctypes.c_int32, [_P, ctypes.c_uint64, ctypes.POINTER(DpcsMaterial), _P,
                                                       ctypes.POINTER(DpcsView), ctypes.POINTER(DpcsParams),
                                                       ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, _P, _P, _P,
                                                       ctypes.c_int32, ctypes.c_int32, _P, _P]),
    "dpcs_render_loss_backward": (ctypes.c_int32, [_P, ctypes.c_uint64, _P, _P, ctypes.c_int32, ctypes.c_int32, _P,
                                                   ctypes.POINTER(DpcsView), ctypes.POINTER(DpcsParams),
                                                   ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, _P, ctypes.c_int32,
                                                   ctypes.c_float, _P, _P, _P, _P, _P, _P, _P, _P]),
    "dpcs_render_principled": (ctypes.c_int32, [_P, ctypes.c_uint64, ctypes.POINTER(DpcsMaterial), _P,
                                                ctypes.POINTER(DpcsView), ctypes.POINTER(DpcsParams), ctypes.c_int32,
                                                ctypes.c_int32, ctypes.c_uint64, _P, _P, _P]),
    "dpcs_render_backward_principled": (ctypes.c_int32, [_P, ctypes.c_uint64, ctypes.POINTER(DpcsMaterial), _P,
                                                         ctypes.POINTER(DpcsView), ctypes.POINTER(DpcsParams),
                                                         ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, _P, _P, _P,
                                                         _P, _P, _P, _P, _P, _P, _P]),
    "dpcs_render_loss_backward_principled": (ctypes.c_int32, [_P, ctypes.c_uint64, ctypes.POINTER(DpcsMaterial), _P,
                                                              ctypes.POINTER(DpcsView), ctypes.POINTER(DpcsParams),
                                                              ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, _P,
                                                              ctypes.c_int32, ctypes.c_float, _P, _P, _P, _P, _P, _P,
                                                              _P, _P, _P, _P]),
    "dpcs_render_keep_principled": (ctypes.c_int32, [_P, ctypes.c_uint64, ctypes.POINTER(DpcsMaterial), _P,
                                                     ctypes.POINTER(DpcsView), ctypes.POINTER(DpcsParams),
                                                     ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, _P, _P, _P]),
    "dpcs_render_backward_kept_principled": (ctypes.c_int32, [_P, ctypes.c_uint64, ctypes.POINTER(DpcsMaterial), _P,
                                                              ctypes.POINTER(DpcsView), ctypes.POINTER(DpcsParams),
                                                              ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, _P, _P,
                                                              _P, _P, _P, _P, _P, _P, _P, _P]),
    "dpcs_timing_enable": (ctypes.c_int32, [_P, ctypes.c_int32]),
    "dpcs_timing_read": (ctypes.c_int32, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_int64)]),
    "dpcs_counters_read": (ctypes.c_int32, [_P, _P, ctypes.c_int32]),
    "dpcs_debug_set_visit_cap": (ctypes.c_int32, [_P, ctypes.c_int32]),
    "dpcs_set_grad_accum": (ctypes.c_int32, [_P, ctypes.c_int32]),
    "dpcs_set_render_path": (ctypes.c_int32, [_P, ctypes.c_int32, ctypes.c_int64]),
    "dpcs_set_bvh_builder": (ctypes.c_int32, [_P, ctypes.c_int32]),
    "dpcs_gbuffer": (ctypes.c_int32, [_P, ctypes.c_uint64, _P, _P, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.POINTER(DpcsView), _P, _P]),
    "dpcs_denoise": (ctypes.c_int32, [_P, _P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(DpcsDenoiseParams),
                                      _P, _P, _P]),
    "dpcs_denoise_backward": (ctypes.c_int32, [_P, _P, _P, _P, ctypes.c_int32, ctypes.c_int32,
                                               ctypes.POINTER(DpcsDenoiseParams), _P, _P]),
    "dpcs_serve_create": (ctypes.c_int32, [_P, ctypes.POINTER(DpcsServeConfig), ctypes.POINTER(_P)]),
    "dpcs_serve_destroy": (ctypes.c_int32, [_P]),
    "dpcs_serve_add_scene": (ctypes.c_int32, [_P, ctypes.c_uint64, _P, _P, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.POINTER(DpcsView), ctypes.POINTER(DpcsParams), ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_int32)]),
    "dpcs_serve_submit": (ctypes.c_int32, [_P, ctypes.POINTER(DpcsRequest), ctypes.POINTER(ctypes.c_uint64)]),
    "dpcs_serve_step": (ctypes.c_int32, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "dpcs_serve_query": (ctypes.c_int32, [_P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_double)]),
    "dpcs_serve_drain": (ctypes.c_int32, [_P, ctypes.c_double]),
    "dpcs_serve_stats_get": (ctypes.c_int32, [_P, ctypes.POINTER(DpcsServeStats)]),
    "dpcs_l2_loss": (ctypes.c_int32, [_P, _P, _P, ctypes.c_int64, _P, _P, _P]),
    "dpcs_l1_loss": (ctypes.c_int32, [_P, _P, _P, ctypes.c_int64, ctypes.c_float, _P, _P, _P]),
    "dpcs_tv_loss": (ctypes.c_int32, [_P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, _P, _P,
                                      _P]),
    "dpcs_adam": (ctypes.c_int32, [_P, _P, _P, _P, _P, ctypes.c_int64, ctypes.c_float, ctypes.c_float,
                                   ctypes.c_float, ctypes.c_float, ctypes.c_int32, ctypes.c_float, ctypes.c_float,
                                   _P]),
}


def library_path() -> str:
    return _build.lib_path()


def open_library(path: str):
    """ctypes handle of a libdpcs build at ``path`` with every signature set."""
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def load_library(path: str | None = None):
    """Load libdpcs.so (building it first if it is missing).  Raises if the
    library cannot be built or loaded: there is no fallback path."""
    global _lib, _lib_path
    if _lib is not None and (path is None or path == _lib_path):
        return _lib
    if path is None:
        path = library_path()
        if not os.path.exists(path):
            path = _build.build()
    _lib, _lib_path = open_library(path), path
    return _lib


def check_library():
    """The DPCS_CHECK debug build: every node and leaf reference is checked
    before it is read; a bad one ends the ray and dpcs_sync reports
    DPCS_ERR_DEVICE_CHECK."""
    return open_library(_build.build(variant="_check", defines=("DPCS_CHECK",)))


def counters_library():
    """The DPCS_COUNTERS build (counts node visits, triangle tests, ...)."""
    return open_library(_build.build(variant="_counters", defines=("DPCS_COUNTERS",)))


def make_params(p) -> DpcsParams:
    o = DpcsParams()
    o.gamma_p[:] = [float(x) for x in p.gamma_p]
    o.gain_p = float(p.gain_p)
    o.gamma_c[:] = [float(x) for x in p.gamma_c]
    o.gain_c = float(p.gain_c)
    o.wb[:] = [float(x) for x in p.wb]
    o.k_proj = float(p.k_proj)
    o.ks = float(p.ks)
    o.f0 = float(p.f0)
    o.rr_start = int(p.rr_start)
    o.rr_q = float(p.rr_q)
    o.clip = float(p.clip)
    o.jitter = int(p.jitter)
    return o


def make_view(Kc, Hc, Wc, Kp, Rp, tp, Hp, Wp) -> DpcsView:
    v = DpcsView()
    v.Kc[:] = [float(x) for x in np.asarray(Kc, np.float32).ravel()]
    v.Hc, v.Wc = int(Hc), int(Wc)
    v.Kp[:] = [float(x) for x in np.asarray(Kp, np.float32).ravel()]
    v.Rp[:] = [float(x) for x in np.asarray(Rp, np.float32).ravel()]
    v.tp[:] = [float(x) for x in np.asarray(tp, np.float32).ravel()]
    v.Hp, v.Wp = int(Hp), int(Wp)
    return v


def view_of(scene) -> DpcsView:
    """DpcsView of a ``scenes.Scene``."""
    return make_view(scene.Kc, scene.Hc, scene.Wc, scene.Kp, scene.Rp, scene.tp, scene.Hp, scene.Wp)


# ---------------------------------------------------------------------------
# raw ABI wrappers (same names as the C entry points)
# ---------------------------------------------------------------------------
def dpcs_create(device: int = 0, hbm_budget_bytes: int = 0):
    h = _P()
    st = load_library().dpcs_create(int(device), int(hbm_budget_bytes), ctypes.byref(h))
    if st != DPCS_OK:
        raise DPCSError(st, "dpcs_create failed")
    return h


def dpcs_destroy(ctx):
    return load_library().dpcs_destroy(ctx)


def dpcs_last_error(ctx) -> str:
    r = load_library().dpcs_last_error(ctx)
    return r.decode() if r else ""


def dpcs_sync(ctx, stream=None):
    return load_library().dpcs_sync(ctx, stream)


def dpcs_memory_used(ctx) -> int:
    return load_library().dpcs_memory_used(ctx)


def dpcs_launch_count(ctx) -> int:
    return load_library().dpcs_launch_count(ctx)


def dpcs_scene_upload(ctx, verts, V, tris, T, uv, stream, out):
    return load_library().dpcs_scene_upload(ctx, verts, V, tris, T, uv, stream, out)


def dpcs_scene_free(ctx, scene):
    return load_library().dpcs_scene_free(ctx, scene)


def dpcs_scene_export(ctx, scene, codes, order, child, child_box):
    return load_library().dpcs_scene_export(ctx, scene, codes, order, child, child_box)


def dpcs_trace(ctx, scene, orig, dir, n, t_out, tri_out, stream):
    return load_library().dpcs_trace(ctx, scene, orig, dir, n, t_out, tri_out, stream)


def dpcs_render(ctx, scene, albedo, rough, Ht, Wt, Ip, view, params, spp, bounces, seed, Ic, Ec, stream):
    return load_library().dpcs_render(ctx, scene, albedo, rough, Ht, Wt, Ip, ctypes.byref(view),
                                      ctypes.byref(params), spp, bounces, seed, Ic, Ec, stream)


def dpcs_render_noalloc(ctx, scene, albedo, rough, Ht, Wt, Ip, view, params, spp, bounces, seed, Ic, Ec, stream):
    return load_library().dpcs_render_noalloc(ctx, scene, albedo, rough, Ht, Wt, Ip, ctypes.byref(view),
                                              ctypes.byref(params), spp, bounces, seed, Ic, Ec, stream)


def dpcs_render_backward(ctx, scene, albedo, rough, Ht, Wt, Ip, view, params, spp, bounces, seed, Ec, Ic, dIc,
                         dIp, dAlbedo, dRough, dParams, stream):
    return load_library().dpcs_render_backward(ctx, scene, albedo, rough, Ht, Wt, Ip, ctypes.byref(view),
                                               ctypes.byref(params), spp, bounces, seed, Ec, Ic, dIc, dIp, dAlbedo,
                                               dRough, dParams, stream)


def dpcs_pose_backward(ctx, scene, albedo, rough, Ht, Wt, Ip, view, params, spp, bounces, seed, Ec, Ic, dIc,
                       edge_spp, sil_spp, wrench, stream):
    return load_library().dpcs_pose_backward(ctx, scene, albedo, rough, Ht, Wt, Ip, ctypes.byref(view),
                                             ctypes.byref(params), spp, bounces, seed, Ec, Ic, dIc, edge_spp, sil_spp,
                                             wrench, stream)


def dpcs_render_loss_backward(ctx, scene, albedo, rough, Ht, Wt, Ip, view, params, spp, bounces, seed, target,
                              loss_kind, scale, Ic, Ec, loss, dIp, dAlbedo, dRough, dParams, stream):
    return load_library().dpcs_render_loss_backward(ctx, scene, albedo, rough, Ht, Wt, Ip, ctypes.byref(view),
                                                    ctypes.byref(params), spp, bounces, seed, target, loss_kind, scale,
                                                    Ic, Ec, loss, dIp, dAlbedo, dRough, dParams, stream)


def dpcs_render_keep(ctx, scene, albedo, rough, Ht, Wt, Ip, view, params, spp, bounces, seed, Ic, Ec, stream):
    return load_library().dpcs_render_keep(ctx, scene, albedo, rough, Ht, Wt, Ip, ctypes.byref(view),
                                           ctypes.byref(params), spp, bounces, seed, Ic, Ec, stream)


def dpcs_render_backward_kept(ctx, scene, albedo, rough, Ht, Wt, Ip, view, params, spp, bounces, seed, Ec, Ic, dIc,
                              dIp, dAlbedo, dRough, dParams, stream):
    return load_library().dpcs_render_backward_kept(ctx, scene, albedo, rough, Ht, Wt, Ip, ctypes.byref(view),
                                                    ctypes.byref(params), spp, bounces, seed, Ec, Ic, dIc, dIp,
                                                    dAlbedo, dRough, dParams, stream)


def dpcs_set_grad_accum(ctx, mode):
    return load_library().dpcs_set_grad_accum(ctx, int(mode))


def dpcs_set_render_path(ctx, path, chunk):
    return load_library().dpcs_set_render_path(ctx, int(path), int(chunk))


def dpcs_timing_enable(ctx, on):
    return load_library().dpcs_timing_enable(ctx, int(on))


def dpcs_timing_read(ctx, kernel, total_ms, launches):
    return load_library().dpcs_timing_read(ctx, int(kernel), total_ms, launches)


def dpcs_counters_read(ctx, out, reset):
    return load_library().dpcs_counters_read(ctx, out, int(reset))


def dpcs_gbuffer(ctx, scene, albedo, rough, Ht, Wt, view, guide, stream):
    return load_library().dpcs_gbuffer(ctx, scene, albedo, rough, Ht, Wt, ctypes.byref(view), guide, stream)


def dpcs_denoise(ctx, Ic, guide, Hc, Wc, params, out, wsum, stream):
    return load_library().dpcs_denoise(ctx, Ic, guide, Hc, Wc, ctypes.byref(params), out, wsum, stream)


def dpcs_denoise_backward(ctx, dOut, guide, wsum, Hc, Wc, params, dIc, stream):
    return load_library().dpcs_denoise_backward(ctx, dOut, guide, wsum, Hc, Wc, ctypes.byref(params), dIc, stream)


def dpcs_l2_loss(ctx, Ic, target, n, dIc, loss, stream):
    return load_library().dpcs_l2_loss(ctx, Ic, target, n, dIc, loss, stream)


def dpcs_scene_update(ctx, scene, verts, V, stream):
    return load_library().dpcs_scene_update(ctx, scene, verts, V, stream)


def dpcs_l1_loss(ctx, Ic, target, n, scale, dIc, loss, stream):
    return load_library().dpcs_l1_loss(ctx, Ic, target, n, scale, dIc, loss, stream)


def dpcs_tv_loss(ctx, tex, H, W, C, weight, grad, loss, stream):
    return load_library().dpcs_tv_loss(ctx, tex, H, W, C, weight, grad, loss, stream)


def dpcs_adam(ctx, p, g, m, v, n, lr, beta1, beta2, eps, step, lo, hi, stream):
    return load_library().dpcs_adam(ctx, p, g, m, v, n, lr, beta1, beta2, eps, step, lo, hi, stream)


# ---------------------------------------------------------------------------
# torch-facing context
# ---------------------------------------------------------------------------
def _ptr(t, name, shape=None, dtype=None, device=None, allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    import torch

    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if device is not None and t.device != device:
        raise ValueError(f"{name}: expected device {device}, got {t.device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr()) if t.numel() else None


def _stream(stream):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """A libdpcs context on one CUDA device, driven with torch tensors."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, lib=None):
        import torch

        self._moves = {}  # scene -> how many updates and transforms this object has applied
        self._ntris = {}  # scene -> triangle count, to size the host arrays export() hands to the library
        self.lib = lib if lib is not None else load_library()
        self.device = torch.device("cuda", device)
        h = _P()
        st = self.lib.dpcs_create(int(device), int(hbm_budget_bytes), ctypes.byref(h))
        if st != DPCS_OK:
            raise DPCSError(st, "dpcs_create failed")
        self.handle = h

    # -- measurement -------------------------------------------------------------
    def timing(self, on: bool):
        self.check(self.lib.dpcs_timing_enable(self.handle, 1 if on else 0), "timing_enable")

    def set_visit_cap(self, cap: int):
        """Failure-path testing: cap BVH traversal steps per ray (0 = default)."""
        self.check(self.lib.dpcs_debug_set_visit_cap(self.handle, int(cap)), "debug_set_visit_cap")

    def set_grad_accum(self, mode: int):
        """Adjoint accumulation: DPCS_ACCUM_F32 (float4 atomics, default) or
        DPCS_ACCUM_F64 (FP64 atomics; sums independent of the add order up to
        FP64 rounding)."""
        self.check(self.lib.dpcs_set_grad_accum(self.handle, int(mode)), "set_grad_accum")

    def set_bvh_builder(self, builder: int):
        """Tree topology of later uploads: DPCS_BVH_PLOC (default) or DPCS_BVH_LBVH."""
        self.check(self.lib.dpcs_set_bvh_builder(self.handle, int(builder)), "set_bvh_builder")

    def set_render_path(self, path: int, chunk: int = 0):
        """dpcs_render's kernels: DPCS_PATH_MEGAKERNEL (one kernel) or
        DPCS_PATH_WAVEFRONT (trace and shade passes over path queues, in chunks
        of ``chunk`` paths; 0 keeps the current size)."""
        self.check(self.lib.dpcs_set_render_path(self.handle, int(path), int(chunk)), "set_render_path")

    def counters(self, reset: bool = True):
        """Work counters (counters build only): dict of totals."""
        out = (ctypes.c_uint64 * 10)()
        self.check(self.lib.dpcs_counters_read(self.handle, out, 1 if reset else 0), "counters_read")
        keys = ("node_visits", "tri_tests", "rays", "shadow_rays", "vertices", "lit", "continuations", "paths",
                "trav_warp_iters", "path_warp_iters")
        return dict(zip(keys, [int(x) for x in out]))

    def kernel_time(self, kernel: int):
        """(total ms, launches) of kernel 0 = render, 1 = replay since timing(True)."""
        ms, n = ctypes.c_double(), ctypes.c_int64()
        self.check(self.lib.dpcs_timing_read(self.handle, kernel, ctypes.byref(ms), ctypes.byref(n)), "timing_read")
        return ms.value, n.value

    def close(self):
        if getattr(self, "handle", None):
            self.lib.dpcs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, status: int, what: str):
        if status != DPCS_OK:
            msg = self.lib.dpcs_last_error(self.handle)
            raise DPCSError(status, f"{what}: {msg.decode() if msg else ''}")

    # -- bookkeeping ---------------------------------------------------------
    def sync(self, stream=None):
        self.check(self.lib.dpcs_sync(self.handle, _stream(stream)), "sync")

    @property
    def memory_used(self) -> int:
        return int(self.lib.dpcs_memory_used(self.handle))

    @property
    def launch_count(self) -> int:
        return self.lib.dpcs_launch_count(self.handle)

    # -- scenes ----------------------------------------------------------------
    def upload(self, verts, tris, uv, stream=None) -> int:
        """verts (V, 3), tris (T, 3) vertex indices, uv (V, 2).  The library
        reads V x 3, T x 3 and V x 2 values from these host arrays, so their
        shapes are checked here."""
        verts = np.ascontiguousarray(verts, np.float32)
        tris = np.ascontiguousarray(tris, np.int32)
        uv = np.ascontiguousarray(uv, np.float32)
        if verts.ndim != 2 or verts.shape[1] != 3 or tris.ndim != 2 or tris.shape[1] != 3 or \
                uv.shape != (verts.shape[0], 2):
            raise ValueError(f"upload: expected verts (V, 3), tris (T, 3) and uv (V, 2), got {verts.shape}, "
                             f"{tris.shape} and {uv.shape}")
        out = ctypes.c_uint64()
        st = self.lib.dpcs_scene_upload(self.handle, verts.ctypes.data_as(_P), len(verts), tris.ctypes.data_as(_P),
                               len(tris), uv.ctypes.data_as(_P), _stream(stream), ctypes.byref(out))
        self.check(st, "scene_upload")
        self._ntris[out.value] = len(tris)
        return out.value

    def update(self, scene: int, verts, stream=None):
        """New positions for the scene's vertices (same count); refits the tree."""
        verts = np.ascontiguousarray(verts, np.float32)
        if verts.ndim != 2 or verts.shape[1] != 3:
            raise ValueError(f"update: expected verts (V, 3), got {verts.shape}")
        st = self.lib.dpcs_scene_update(self.handle, scene, verts.ctypes.data_as(_P), len(verts), _stream(stream))
        self.check(st, "scene_update")
        self._moves[scene] = self._moves.get(scene, 0) + 1

    def transform(self, scene: int, R, t, stream=None):
        """dpcs_scene_transform: the scene's stored vertex positions mapped by
        v -> R v + t (3 x 3 and 3-vector, rounded to float32), tree refitted."""
        Rf = np.ascontiguousarray(np.asarray(R, np.float64).reshape(3, 3), np.float32)
        tf = np.ascontiguousarray(np.asarray(t, np.float64).reshape(3), np.float32)
        st = self.lib.dpcs_scene_transform(self.handle, scene, Rf.ctypes.data_as(_P), tf.ctypes.data_as(_P),
                                           _stream(stream))
        self.check(st, "scene_transform")
        self._moves[scene] = self._moves.get(scene, 0) + 1

    def scene_moves(self, scene: int) -> int:
        """How many times update() or transform() has moved the scene's
        vertices through this object.  A path replay re-traces the scene as it
        is when the replay runs, so the autograd wrapper checks that this count
        is the same at a render and at its backward."""
        return self._moves.get(scene, 0)

    def free(self, scene: int):
        self.check(self.lib.dpcs_scene_free(self.handle, scene), "scene_free")
        self._ntris.pop(scene, None)
        self._moves.pop(scene, None)

    def export(self, scene: int, T: int):
        """The scene's tree in host arrays sized for T triangles.  The library
        fills them for the scene's own triangle count, so T must be that count
        (checked against the upload)."""
        known = self._ntris.get(scene)
        if known is not None and int(T) != known:
            raise ValueError(f"export: scene {scene} has {known} triangles, not {T}")
        codes = np.zeros(T, np.uint32)
        order = np.zeros(T, np.int32)
        child = np.zeros((max(T - 1, 0), 2), np.int32)
        box = np.zeros((max(T - 1, 0), 2, 6), np.float32)
        st = self.lib.dpcs_scene_export(self.handle, scene, codes.ctypes.data_as(_P), order.ctypes.data_as(_P),
                               child.ctypes.data_as(_P), box.ctypes.data_as(_P))
        self.check(st, "scene_export")
        return codes, order, child, box

    def trace(self, scene: int, orig, dir, stream=None):
        import torch

        n = orig.shape[0]
        t = torch.empty(n, dtype=torch.float32, device=self.device)
        tri = torch.empty(n, dtype=torch.int32, device=self.device)
        st = self.lib.dpcs_trace(self.handle, scene, _ptr(orig, "orig", (n, 3), torch.float32, self.device),
                        _ptr(dir, "dir", (n, 3), torch.float32, self.device), n, _ptr(t, "t"), _ptr(tri, "tri"),
                        _stream(stream))
        self.check(st, "trace")
        return t, tri

    # -- rendering -------------------------------------------------------------
    def render(self, scene: int, albedo, rough, Ip, view: DpcsView, params: DpcsParams, spp: int, bounces: int,
               seed: int, Ic=None, Ec=None, stream=None, keep: bool = False):
        import torch

        Ht, Wt = albedo.shape[0], albedo.shape[1]
        f32 = torch.float32
        if Ic is None:
            Ic = torch.empty((view.Hc, view.Wc, 3), dtype=f32, device=self.device)
        fn = self.lib.dpcs_render_keep if keep else self.lib.dpcs_render  # keep: path records for render_backward(kept=True)
        st = fn(self.handle, scene, _ptr(albedo, "albedo", (Ht, Wt, 3), f32, self.device),
                         _ptr(rough, "rough", (Ht, Wt), f32, self.device), Ht, Wt,
                         _ptr(Ip, "Ip", (view.Hp, view.Wp, 3), f32, self.device), ctypes.byref(view),
                         ctypes.byref(params), int(spp),
                         int(bounces), int(seed) & (2**64 - 1),
                         _ptr(Ic, "Ic", (view.Hc, view.Wc, 3), f32, self.device),
                         _ptr(Ec, "Ec", (view.Hc, view.Wc, 3), f32, self.device, allow_none=True), _stream(stream))
        self.check(st, "render")
        return Ic, Ec

    def render_backward(self, scene: int, albedo, rough, Ip, view: DpcsView, params: DpcsParams, spp: int,
                        bounces: int, seed: int, Ec, Ic, dIc, dIp=None, dAlbedo=None, dRough=None, dParams=None,
                        stream=None, kept: bool = False):
        import torch

        Ht, Wt = albedo.shape[0], albedo.shape[1]
        f32 = torch.float32
        img = (view.Hc, view.Wc, 3)
        fn = self.lib.dpcs_render_backward_kept if kept else self.lib.dpcs_render_backward  # kept: no re-trace
        st = fn(
            self.handle, scene, _ptr(albedo, "albedo", (Ht, Wt, 3), f32, self.device),
            _ptr(rough, "rough", (Ht, Wt), f32, self.device), Ht, Wt,
            _ptr(Ip, "Ip", (view.Hp, view.Wp, 3), f32, self.device), ctypes.byref(view),
                         ctypes.byref(params), int(spp), int(bounces),
            int(seed) & (2**64 - 1), _ptr(Ec, "Ec", img, f32, self.device), _ptr(Ic, "Ic", img, f32, self.device),
            _ptr(dIc, "dIc", img, f32, self.device),
            _ptr(dIp, "dIp", (view.Hp, view.Wp, 3), f32, self.device, allow_none=True),
            _ptr(dAlbedo, "dAlbedo", (Ht, Wt, 3), f32, self.device, allow_none=True),
            _ptr(dRough, "dRough", (Ht, Wt), f32, self.device, allow_none=True),
            _ptr(dParams, "dParams", (11,), f32, self.device, allow_none=True), _stream(stream))
        self.check(st, "render_backward")

    def pose_backward(self, scene: int, albedo, rough, Ip, view: DpcsView, params: DpcsParams, spp: int,
                      bounces: int, seed: int, Ec, Ic, dIc, edge_spp: int, sil_spp: int, wrench=None, stream=None):
        """dLoss/d(a, b) of a rigid motion of the scene in the camera frame
        (``dpcs_pose_backward``): returns ``wrench`` (3, 6) float64 on the
        device, the interior, pixel-edge and silhouette terms, ADDED to the
        tensor passed in (zeros when none is)."""
        import torch

        Ht, Wt = albedo.shape[0], albedo.shape[1]
        f32 = torch.float32
        img = (view.Hc, view.Wc, 3)
        if wrench is None:
            wrench = torch.zeros((3, 6), dtype=torch.float64, device=self.device)
        st = self.lib.dpcs_pose_backward(
            self.handle, scene, _ptr(albedo, "albedo", (Ht, Wt, 3), f32, self.device),
            _ptr(rough, "rough", (Ht, Wt), f32, self.device), Ht, Wt,
            _ptr(Ip, "Ip", (view.Hp, view.Wp, 3), f32, self.device), ctypes.byref(view), ctypes.byref(params),
            int(spp), int(bounces), int(seed) & (2**64 - 1), _ptr(Ec, "Ec", img, f32, self.device),
            _ptr(Ic, "Ic", img, f32, self.device), _ptr(dIc, "dIc", img, f32, self.device), int(edge_spp),
            int(sil_spp), _ptr(wrench, "wrench", (3, 6), torch.float64, self.device), _stream(stream))
        self.check(st, "pose_backward")
        return wrench

    def pose_backward_principled(self, scene: int, albedo, rough, metallic, normal, Ip, view: DpcsView,
                                 params: DpcsParams, spp: int, bounces: int, seed: int, Ec, Ic, dIc, edge_spp: int,
                                 sil_spp: int, wrench=None, stream=None):
        """``pose_backward`` with the principled material
        (``dpcs_pose_backward_principled``); metallic / normal may be None."""
        import torch

        f32 = torch.float32
        img = (view.Hc, view.Wc, 3)
        if wrench is None:
            wrench = torch.zeros((3, 6), dtype=torch.float64, device=self.device)
        m = self._material(albedo, rough, metallic, normal)
        st = self.lib.dpcs_pose_backward_principled(
            self.handle, scene, ctypes.byref(m), _ptr(Ip, "Ip", (view.Hp, view.Wp, 3), f32, self.device),
            ctypes.byref(view), ctypes.byref(params), int(spp), int(bounces), int(seed) & (2**64 - 1),
            _ptr(Ec, "Ec", img, f32, self.device), _ptr(Ic, "Ic", img, f32, self.device),
            _ptr(dIc, "dIc", img, f32, self.device), int(edge_spp), int(sil_spp),
            _ptr(wrench, "wrench", (3, 6), torch.float64, self.device), _stream(stream))
        self.check(st, "pose_backward_principled")
        return wrench

    # -- principled material (metallic and normal maps) --------------------------
    def _material(self, albedo, rough, metallic, normal):
        import torch

        Ht, Wt = albedo.shape[0], albedo.shape[1]
        f32 = torch.float32
        m = DpcsMaterial()
        m.albedo = _ptr(albedo, "albedo", (Ht, Wt, 3), f32, self.device)
        m.rough = _ptr(rough, "rough", (Ht, Wt), f32, self.device)
        m.metallic = _ptr(metallic, "metallic", (Ht, Wt), f32, self.device, allow_none=True)
        m.normal = _ptr(normal, "normal", (Ht, Wt, 3), f32, self.device, allow_none=True)
        m.Ht, m.Wt = Ht, Wt
        return m

    def render_principled(self, scene: int, albedo, rough, metallic, normal, Ip, view: DpcsView,
                          params: DpcsParams, spp: int, bounces: int, seed: int, Ic=None, Ec=None, stream=None,
                          keep: bool = False):
        """dpcs_render_principled: render with metallic (Ht, Wt) and normal (Ht, Wt, 3) maps (either None);
        keep=True keeps the path records for render_backward_principled(kept=True)."""
        import torch

        f32 = torch.float32
        mat = self._material(albedo, rough, metallic, normal)
        if Ic is None:
            Ic = torch.empty((view.Hc, view.Wc, 3), dtype=f32, device=self.device)
        fn = self.lib.dpcs_render_keep_principled if keep else self.lib.dpcs_render_principled
        st = fn(
            self.handle, scene, ctypes.byref(mat), _ptr(Ip, "Ip", (view.Hp, view.Wp, 3), f32, self.device),
            ctypes.byref(view), ctypes.byref(params), int(spp), int(bounces), int(seed) & (2**64 - 1),
            _ptr(Ic, "Ic", (view.Hc, view.Wc, 3), f32, self.device),
            _ptr(Ec, "Ec", (view.Hc, view.Wc, 3), f32, self.device, allow_none=True), _stream(stream))
        self.check(st, "render_principled")
        return Ic, Ec

    def render_backward_principled(self, scene: int, albedo, rough, metallic, normal, Ip, view: DpcsView,
                                   params: DpcsParams, spp: int, bounces: int, seed: int, Ec, Ic, dIc, dIp=None,
                                   dAlbedo=None, dRough=None, dMetallic=None, dNormal=None, dParams=None,
                                   stream=None, kept: bool = False):
        """dpcs_render_backward_principled: the adjoint, accumulating into the given gradient buffers;
        kept=True sweeps the records of the last keep=True render instead of re-tracing."""
        import torch

        f32 = torch.float32
        mat = self._material(albedo, rough, metallic, normal)
        Ht, Wt = mat.Ht, mat.Wt
        img = (view.Hc, view.Wc, 3)
        fn = self.lib.dpcs_render_backward_kept_principled if kept else self.lib.dpcs_render_backward_principled
        st = fn(
            self.handle, scene, ctypes.byref(mat), _ptr(Ip, "Ip", (view.Hp, view.Wp, 3), f32, self.device),
            ctypes.byref(view), ctypes.byref(params), int(spp), int(bounces), int(seed) & (2**64 - 1),
            _ptr(Ec, "Ec", img, f32, self.device), _ptr(Ic, "Ic", img, f32, self.device),
            _ptr(dIc, "dIc", img, f32, self.device),
            _ptr(dIp, "dIp", (view.Hp, view.Wp, 3), f32, self.device, allow_none=True),
            _ptr(dAlbedo, "dAlbedo", (Ht, Wt, 3), f32, self.device, allow_none=True),
            _ptr(dRough, "dRough", (Ht, Wt), f32, self.device, allow_none=True),
            _ptr(dMetallic, "dMetallic", (Ht, Wt), f32, self.device, allow_none=True),
            _ptr(dNormal, "dNormal", (Ht, Wt, 3), f32, self.device, allow_none=True),
            _ptr(dParams, "dParams", (11,), f32, self.device, allow_none=True), _stream(stream))
        self.check(st, "render_backward_principled")

    def gbuffer(self, scene: int, albedo, rough, view: DpcsView, guide=None, stream=None):
        """Guide features (Hc, Wc, 8) of the first hit through each pixel centre."""
        import torch

        Ht, Wt = albedo.shape[0], albedo.shape[1]
        f32 = torch.float32
        if guide is None:
            guide = torch.empty((view.Hc, view.Wc, 8), dtype=f32, device=self.device)
        st = self.lib.dpcs_gbuffer(self.handle, scene, _ptr(albedo, "albedo", (Ht, Wt, 3), f32, self.device),
                                   _ptr(rough, "rough", (Ht, Wt), f32, self.device), Ht, Wt, ctypes.byref(view),
                                   _ptr(guide, "guide", (view.Hc, view.Wc, 8), f32, self.device), _stream(stream))
        self.check(st, "gbuffer")
        return guide

    def denoise(self, Ic, guide, params: DpcsDenoiseParams, out=None, wsum=None, stream=None):
        """Eq. 11: out = D(Ic); also returns the weight sums the adjoint needs."""
        import torch

        Hc, Wc = Ic.shape[0], Ic.shape[1]
        f32 = torch.float32
        if out is None:
            out = torch.empty_like(Ic)
        if wsum is None:
            wsum = torch.empty((Hc, Wc), dtype=f32, device=self.device)
        st = self.lib.dpcs_denoise(self.handle, _ptr(Ic, "Ic", (Hc, Wc, 3), f32, self.device),
                                   _ptr(guide, "guide", (Hc, Wc, 8), f32, self.device), Hc, Wc, ctypes.byref(params),
                                   _ptr(out, "out", (Hc, Wc, 3), f32, self.device),
                                   _ptr(wsum, "wsum", (Hc, Wc), f32, self.device), _stream(stream))
        self.check(st, "denoise")
        return out, wsum

    def denoise_backward(self, dOut, guide, wsum, params: DpcsDenoiseParams, dIc=None, stream=None):
        """dIc += D^T(dOut) (dIc is zero-initialised when not given)."""
        import torch

        Hc, Wc = dOut.shape[0], dOut.shape[1]
        f32 = torch.float32
        if dIc is None:
            dIc = torch.zeros_like(dOut)
        st = self.lib.dpcs_denoise_backward(self.handle, _ptr(dOut, "dOut", (Hc, Wc, 3), f32, self.device),
                                            _ptr(guide, "guide", (Hc, Wc, 8), f32, self.device),
                                            _ptr(wsum, "wsum", (Hc, Wc), f32, self.device), Hc, Wc,
                                            ctypes.byref(params), _ptr(dIc, "dIc", (Hc, Wc, 3), f32, self.device),
                                            _stream(stream))
        self.check(st, "denoise_backward")
        return dIc

    def render_loss_backward(self, scene: int, albedo, rough, Ip, view: DpcsView, params: DpcsParams, spp: int,
                             bounces: int, seed: int, target, loss, loss_kind: int = 0, scale: float = 1.0, Ic=None,
                             Ec=None, dIp=None, dAlbedo=None, dRough=None, dParams=None, stream=None):
        """Render, per-pixel loss (0 = L2, 1 = L1) and adjoint in one call;
        returns Ic.  Gradient outputs accumulate."""
        import torch

        Ht, Wt = albedo.shape[0], albedo.shape[1]
        f32 = torch.float32
        img = (view.Hc, view.Wc, 3)
        if Ic is None:
            Ic = torch.empty(img, dtype=f32, device=self.device)
        st = self.lib.dpcs_render_loss_backward(
            self.handle, scene, _ptr(albedo, "albedo", (Ht, Wt, 3), f32, self.device),
            _ptr(rough, "rough", (Ht, Wt), f32, self.device), Ht, Wt,
            _ptr(Ip, "Ip", (view.Hp, view.Wp, 3), f32, self.device), ctypes.byref(view), ctypes.byref(params),
            int(spp), int(bounces), int(seed) & (2**64 - 1), _ptr(target, "target", img, f32, self.device),
            int(loss_kind), float(scale), _ptr(Ic, "Ic", img, f32, self.device),
            _ptr(Ec, "Ec", img, f32, self.device, allow_none=True), _ptr(loss, "loss", (1,), f32, self.device),
            _ptr(dIp, "dIp", (view.Hp, view.Wp, 3), f32, self.device, allow_none=True),
            _ptr(dAlbedo, "dAlbedo", (Ht, Wt, 3), f32, self.device, allow_none=True),
            _ptr(dRough, "dRough", (Ht, Wt), f32, self.device, allow_none=True),
            _ptr(dParams, "dParams", (11,), f32, self.device, allow_none=True), _stream(stream))
        self.check(st, "render_loss_backward")
        return Ic

    def render_loss_backward_principled(self, scene: int, albedo, rough, metallic, normal, Ip, view: DpcsView,
                                        params: DpcsParams, spp: int, bounces: int, seed: int, target, loss,
                                        loss_kind: int = 0, scale: float = 1.0, Ic=None, Ec=None, dIp=None,
                                        dAlbedo=None, dRough=None, dMetallic=None, dNormal=None, dParams=None,
                                        stream=None):
        """render_loss_backward with the principled material (metallic / normal maps, either None); returns Ic."""
        import torch

        f32 = torch.float32
        mat = self._material(albedo, rough, metallic, normal)
        Ht, Wt = mat.Ht, mat.Wt
        img = (view.Hc, view.Wc, 3)
        if Ic is None:
            Ic = torch.empty(img, dtype=f32, device=self.device)
        st = self.lib.dpcs_render_loss_backward_principled(
            self.handle, scene, ctypes.byref(mat), _ptr(Ip, "Ip", (view.Hp, view.Wp, 3), f32, self.device),
            ctypes.byref(view), ctypes.byref(params), int(spp), int(bounces), int(seed) & (2**64 - 1),
            _ptr(target, "target", img, f32, self.device), int(loss_kind), float(scale),
            _ptr(Ic, "Ic", img, f32, self.device), _ptr(Ec, "Ec", img, f32, self.device, allow_none=True),
            _ptr(loss, "loss", (1,), f32, self.device),
            _ptr(dIp, "dIp", (view.Hp, view.Wp, 3), f32, self.device, allow_none=True),
            _ptr(dAlbedo, "dAlbedo", (Ht, Wt, 3), f32, self.device, allow_none=True),
            _ptr(dRough, "dRough", (Ht, Wt), f32, self.device, allow_none=True),
            _ptr(dMetallic, "dMetallic", (Ht, Wt), f32, self.device, allow_none=True),
            _ptr(dNormal, "dNormal", (Ht, Wt, 3), f32, self.device, allow_none=True),
            _ptr(dParams, "dParams", (11,), f32, self.device, allow_none=True), _stream(stream))
        self.check(st, "render_loss_backward_principled")
        return Ic

    def l1_loss(self, Ic, target, dIc, loss, scale: float = 1.0, stream=None):
        """Eq. 9 data term: dIc = scale sign(Ic - target), loss = scale sum |Ic - target|."""
        import torch

        f32 = torch.float32
        st = self.lib.dpcs_l1_loss(self.handle, _ptr(Ic, "Ic", None, f32, self.device),
                                   _ptr(target, "target", tuple(Ic.shape), f32, self.device), Ic.numel(),
                                   float(scale), _ptr(dIc, "dIc", tuple(Ic.shape), f32, self.device),
                                   _ptr(loss, "loss", (1,), f32, self.device), _stream(stream))
        self.check(st, "l1_loss")

    def tv_loss(self, tex, grad, loss, weight: float, stream=None):
        """Eq. 9 regulariser: loss = weight TV(tex); grad += its derivative.
        tex is (H, W) or (H, W, C)."""
        import torch

        f32 = torch.float32
        H, W = tex.shape[0], tex.shape[1]
        C = 1 if tex.dim() == 2 else tex.shape[2]
        st = self.lib.dpcs_tv_loss(self.handle, _ptr(tex, "tex", None, f32, self.device), H, W, C, float(weight),
                                   _ptr(grad, "grad", tuple(tex.shape), f32, self.device),
                                   _ptr(loss, "loss", (1,), f32, self.device), _stream(stream))
        self.check(st, "tv_loss")

    def l2_loss(self, Ic, target, dIc, loss, stream=None):
        import torch

        f32 = torch.float32
        n = Ic.numel()
        st = self.lib.dpcs_l2_loss(self.handle, _ptr(Ic, "Ic", None, f32, self.device),
                          _ptr(target, "target", tuple(Ic.shape), f32, self.device), n,
                          _ptr(dIc, "dIc", tuple(Ic.shape), f32, self.device),
                          _ptr(loss, "loss", (1,), f32, self.device), _stream(stream))
        self.check(st, "l2_loss")

    def adam(self, p, g, m, v, step: int, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8, lo=0.0, hi=1.0, stream=None):
        import torch

        f32 = torch.float32
        shp = tuple(p.shape)
        st = self.lib.dpcs_adam(self.handle, _ptr(p, "p", None, f32, self.device), _ptr(g, "g", shp, f32, self.device),
                       _ptr(m, "m", shp, f32, self.device), _ptr(v, "v", shp, f32, self.device), p.numel(),
                       float(lr), float(beta1), float(beta2), float(eps), int(step), float(lo), float(hi),
                       _stream(stream))
        self.check(st, "adam")


class Server:
    """Continuous-batching server (dpcs_serve_*) on a Context.  Host buffers
    handed to submit() are kept alive here until the request is done."""

    def __init__(self, ctx: Context, hbm_budget_bytes: int = 0, max_active: int = 64, max_inflight: int = 2,
                 samples_per_iteration: int = 48 << 20, quantum_samples: int = 2 << 20,
                 policy: int = DPCS_SERVE_FIXED_SHARE, relight_slack: float = 4.0, compensation_slack: float = 1.0,
                 est_samples_per_s: float = 2e9, compensation_share: float = 0.5):
        self.ctx = ctx
        self.lib = ctx.lib
        cfg = DpcsServeConfig(int(hbm_budget_bytes), int(max_active), int(max_inflight), int(samples_per_iteration),
                              int(quantum_samples), int(policy), 0, float(relight_slack), float(compensation_slack),
                              float(est_samples_per_s), float(compensation_share))
        h = _P()
        ctx.check(self.lib.dpcs_serve_create(ctx.handle, ctypes.byref(cfg), ctypes.byref(h)), "serve_create")
        self.handle = h
        self._keep = {}
        self._proj = {}  # scene slot -> projector size (Hp, Wp), to check the host buffers of requests

    def close(self):
        if getattr(self, "handle", None):
            self.lib.dpcs_serve_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_scene(self, scene: int, albedo, rough, view: DpcsView, params: DpcsParams, bounces: int) -> int:
        import torch

        Ht, Wt = albedo.shape[0], albedo.shape[1]
        slot = ctypes.c_int32()
        st = self.lib.dpcs_serve_add_scene(self.handle, scene,
                                           _ptr(albedo, "albedo", (Ht, Wt, 3), torch.float32, self.ctx.device),
                                           _ptr(rough, "rough", (Ht, Wt), torch.float32, self.ctx.device), Ht, Wt,
                                           ctypes.byref(view), ctypes.byref(params), int(bounces), ctypes.byref(slot))
        self.ctx.check(st, "serve_add_scene")
        self._keep[("scene", slot.value)] = (albedo, rough)
        self._proj[slot.value] = (int(view.Hp), int(view.Wp))
        return slot.value

    def submit(self, kind: int, scene: int, Hc: int, Wc: int, spp: int, seed: int, Ip, Ic_out, target=None,
               Ip_out=None, steps: int = 0, lr: float = 1e-2) -> int:
        """Ip, target, Ic_out, Ip_out: contiguous float32 host arrays (pinned
        memory keeps the server's copies asynchronous).  The server copies
        whole images to and from these addresses, which the library cannot
        check, so their sizes are checked here (ValueError): Ic_out and target
        Hc x Wc x 3, Ip and Ip_out the scene's projector size x 3.  Requests
        whose sizes or scene the library itself refuses are passed on for it to
        refuse (DPCSError)."""
        def hp(a, name, n):
            if a is None:
                return None
            if hasattr(a, "data_ptr"):  # torch tensor
                import torch

                ok = (a.device.type == "cpu" and a.dtype == torch.float32 and a.is_contiguous()
                      and (n is None or a.numel() == n))
                ptr = a.data_ptr()
            elif isinstance(a, np.ndarray):
                ok = a.dtype == np.float32 and a.flags.c_contiguous and (n is None or a.size == n)
                ptr = a.ctypes.data
            else:
                ok, ptr = False, None
            if not ok:
                raise ValueError(f"serve_submit: {name} must be a contiguous float32 host array"
                                 + ("" if n is None else f" of {n} elements"))
            return ctypes.c_void_p(ptr)

        img = int(Hc) * int(Wc) * 3 if int(Hc) > 0 and int(Wc) > 0 else None
        proj = self._proj.get(int(scene))
        npj = None if proj is None else proj[0] * proj[1] * 3

        req = DpcsRequest(int(kind), int(scene), int(Hc), int(Wc), int(spp), int(seed) & (2**64 - 1), int(steps),
                          float(lr), hp(Ip, "Ip", npj), hp(target, "target", img), hp(Ic_out, "Ic_out", img),
                          hp(Ip_out, "Ip_out", npj))
        rid = ctypes.c_uint64()
        self.ctx.check(self.lib.dpcs_serve_submit(self.handle, ctypes.byref(req), ctypes.byref(rid)), "serve_submit")
        self._keep[rid.value] = (Ip, target, Ic_out, Ip_out)
        return rid.value

    def step(self) -> int:
        n = ctypes.c_int32()
        self.ctx.check(self.lib.dpcs_serve_step(self.handle, ctypes.byref(n)), "serve_step")
        return n.value

    def query(self, rid: int):
        st, lat = ctypes.c_int32(), ctypes.c_double()
        self.ctx.check(self.lib.dpcs_serve_query(self.handle, rid, ctypes.byref(st), ctypes.byref(lat)), "serve_query")
        if st.value in (DPCS_REQ_DONE, DPCS_REQ_FAILED):
            self._keep.pop(rid, None)
        return st.value, lat.value

    def drain(self, timeout_s: float = 600.0):
        self.ctx.check(self.lib.dpcs_serve_drain(self.handle, float(timeout_s)), "serve_drain")

    def stats(self) -> dict:
        o = DpcsServeStats()
        self.ctx.check(self.lib.dpcs_serve_stats_get(self.handle, ctypes.byref(o)), "serve_stats")
        return {k: getattr(o, k) for k, _ in DpcsServeStats._fields_}
