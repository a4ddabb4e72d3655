"""ctypes binding of the FP64 oracle (``dpcs_oracle.c``) -- test infrastructure.

Inputs are the seeded arrays of ``paper_2503_12174_gb300.scenes``; every
differentiable input (textures, projector image, parameters) is widened to
float64 before it reaches the C code.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dpcs_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "libdpcs_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, OpenMP, no FP contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class OrParams(ctypes.Structure):
    _fields_ = [("gamma_p", ctypes.c_double * 3), ("gain_p", ctypes.c_double),
                ("gamma_c", ctypes.c_double * 3), ("gain_c", ctypes.c_double),
                ("wb", ctypes.c_double * 3), ("k_proj", ctypes.c_double),
                ("ks", ctypes.c_double), ("f0", ctypes.c_double),
                ("rr_start", ctypes.c_int32), ("rr_q", ctypes.c_double),
                ("clip", ctypes.c_double), ("jitter", ctypes.c_int32)]


class OrView(ctypes.Structure):
    _fields_ = [("Kc", ctypes.c_double * 9), ("Hc", ctypes.c_int32), ("Wc", ctypes.c_int32),
                ("Kp", ctypes.c_double * 9), ("Rp", ctypes.c_double * 9), ("tp", ctypes.c_double * 3),
                ("Hp", ctypes.c_int32), ("Wp", ctypes.c_int32)]


def load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        _lib.or_render.restype = ctypes.c_int
        _lib.or_render_backward.restype = ctypes.c_int
        _lib.or_ggx_D.restype = ctypes.c_double
        _lib.or_ggx_D.argtypes = [ctypes.c_double, ctypes.c_double]
        _lib.or_bsdf_pdf.restype = ctypes.c_double
        _lib.or_bsdf_pdf.argtypes = [P, P, P, ctypes.c_double, ctypes.c_double]
        _lib.or_bsdf_sample.restype = ctypes.c_int
        _lib.or_bsdf_sample.argtypes = [P, P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, P]
        _lib.or_bsdf_eval.argtypes = [P, P, P, P, ctypes.c_double, ctypes.c_double, ctypes.c_double, P, P]
        _lib.or_pbr_eval.argtypes = [P, P, P, P, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     P, P, P, P, P]
        _lib.or_render_m.restype = ctypes.c_int
        _lib.or_render_backward_m.restype = ctypes.c_int
        _lib.or_pose_backward.restype = ctypes.c_int
        _lib.or_pose_backward_m.restype = ctypes.c_int
        _lib.or_gbuffer.restype = ctypes.c_int
        _lib.or_num_threads.restype = ctypes.c_int
        _lib.or_num_threads.argtypes = [ctypes.c_int]
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads(n: int = 0) -> int:
    return load().or_num_threads(int(n))


def make_params(p) -> OrParams:
    o = OrParams()
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


def make_view(sc) -> OrView:
    v = OrView()
    v.Kc[:] = [float(x) for x in np.asarray(sc.Kc, np.float64).ravel()]
    v.Hc, v.Wc = int(sc.Hc), int(sc.Wc)
    v.Kp[:] = [float(x) for x in np.asarray(sc.Kp, np.float64).ravel()]
    v.Rp[:] = [float(x) for x in np.asarray(sc.Rp, np.float64).ravel()]
    v.tp[:] = [float(x) for x in np.asarray(sc.tp, np.float64).ravel()]
    v.Hp, v.Wp = int(sc.Ip.shape[0]), int(sc.Ip.shape[1])
    return v


# ---------------------------------------------------------------------------
def philox(ctr: np.ndarray, seed: int) -> np.ndarray:
    """Philox4x32-10 blocks for counters ``ctr`` (n, 4) uint32 under key ``seed``."""
    ctr = _c(ctr, np.uint32).reshape(-1, 4)
    out = np.empty_like(ctr)
    load().or_philox(_p(ctr), ctypes.c_int64(len(ctr)), ctypes.c_uint64(seed), _p(out))
    return out


def morton(verts, tris) -> np.ndarray:
    verts, tris = _c(verts, np.float32), _c(tris, np.int32)
    out = np.empty(len(tris), np.uint32)
    load().or_morton(_p(verts), _p(tris), ctypes.c_int32(len(tris)), _p(out))
    return out


def lbvh(verts, tris):
    """(sorted codes, sorted triangle order, child refs (T-1, 2), child boxes (T-1, 2, 6))."""
    verts, tris = _c(verts, np.float32), _c(tris, np.int32)
    T = len(tris)
    codes = np.empty(T, np.uint32)
    order = np.empty(T, np.int32)
    child = np.zeros((max(T - 1, 0), 2), np.int32)
    box = np.zeros((max(T - 1, 0), 2, 6), np.float32)
    load().or_lbvh(_p(verts), _p(tris), ctypes.c_int32(T), _p(codes), _p(order), _p(child), _p(box))
    return codes, order, child, box


def closest(verts, tris, o, d, accel: bool = False):
    """FP64 closest hit (t, triangle) of each ray; brute force, or the BVH of
    the timing mode (``accel``)."""
    verts, tris = _c(verts, np.float32), _c(tris, np.int32)
    o, d = _c(o, np.float64).reshape(-1, 3), _c(d, np.float64).reshape(-1, 3)
    n = len(o)
    t = np.empty(n, np.float64)
    tri = np.empty(n, np.int32)
    uv = np.zeros((max(len(verts), 1), 2), np.float32)
    with _Accel(accel):
        load().or_closest(_p(verts), ctypes.c_int32(len(verts)), _p(tris), ctypes.c_int32(len(tris)), _p(uv),
                          _p(o), _p(d), ctypes.c_int64(n), _p(t), _p(tri))
    return t, tri


def ggx_D(cos_h: float, alpha: float) -> float:
    return load().or_ggx_D(float(cos_h), float(alpha))


def bsdf_eval(n, wo, wi, rho, r, ks, f0):
    n, wo, wi, rho = (_c(x, np.float64) for x in (n, wo, wi, rho))
    f = np.zeros(3)
    dfdr = np.zeros(1)
    load().or_bsdf_eval(_p(n), _p(wo), _p(wi), _p(rho), float(r), float(ks), float(f0), _p(f), _p(dfdr))
    return f, float(dfdr[0])


def pbr_eval(n, wo, wi, rho, r, m, ks, f0):
    """Principled BRDF with metallic ``m``: dict(f, dr, drho, dm (3,) and dn (3, 3), row = channel)."""
    n, wo, wi, rho = (_c(x, np.float64) for x in (n, wo, wi, rho))
    out = {k: np.zeros(3) for k in ("f", "dr", "drho", "dm")}
    out["dn"] = np.zeros((3, 3))
    load().or_pbr_eval(_p(n), _p(wo), _p(wi), _p(rho), float(r), float(m), float(ks), float(f0), _p(out["f"]),
                       _p(out["dr"]), _p(out["drho"]), _p(out["dm"]), _p(out["dn"]))
    return out


def bsdf_pdf(n, wo, wi, r, ks) -> float:
    n, wo, wi = (_c(x, np.float64) for x in (n, wo, wi))
    return load().or_bsdf_pdf(_p(n), _p(wo), _p(wi), float(r), float(ks))


def bsdf_sample(n, wo, r, ks, u0, u1, u2):
    n, wo = _c(n, np.float64), _c(wo, np.float64)
    wi = np.zeros(3)
    ok = load().or_bsdf_sample(_p(n), _p(wo), float(r), float(ks), float(u0), float(u1), float(u2), _p(wi))
    return bool(ok), wi


def prf(Ip, params) -> np.ndarray:
    Ip = _c(Ip, np.float64)
    out = np.empty_like(Ip)
    P = make_params(params)
    load().or_prf(_p(Ip), ctypes.c_int64(Ip.size // 3), ctypes.byref(P), _p(out))
    return out


def _scene_args(sc, albedo, rough, Ip):
    verts, tris, uv = _c(sc.verts, np.float32), _c(sc.tris, np.int32), _c(sc.uv, np.float32)
    albedo = _c(sc.albedo if albedo is None else albedo, np.float64)
    rough = _c(sc.rough if rough is None else rough, np.float64)
    Ip = _c(sc.Ip if Ip is None else Ip, np.float64)
    return verts, tris, uv, albedo, rough, Ip


_SCENE = object()  # default: take the map from the scene (None there = not used)


def _maps(sc, metallic, normal, Ht, Wt):
    """The principled maps as float64 arrays (or None); checked against the albedo's size."""
    m = getattr(sc, "metallic", None) if metallic is _SCENE else metallic
    nm = getattr(sc, "normal", None) if normal is _SCENE else normal
    m = None if m is None else _c(m, np.float64)
    nm = None if nm is None else _c(nm, np.float64)
    if m is not None and m.shape != (Ht, Wt):
        raise ValueError(f"metallic map {m.shape} != {(Ht, Wt)}")
    if nm is not None and nm.shape != (Ht, Wt, 3):
        raise ValueError(f"normal map {nm.shape} != {(Ht, Wt, 3)}")
    return m, nm


class _Accel:
    """Timing mode for the duration of one call: the C oracle tests only the
    triangles a median-split BVH cannot cull (same hits as brute force)."""

    def __init__(self, on: bool):
        self.on = bool(on)

    def __enter__(self):
        load().or_set_accel(ctypes.c_int(1 if self.on else 0))

    def __exit__(self, *exc):
        load().or_set_accel(ctypes.c_int(0))


def render(sc, pixels=None, *, albedo=None, rough=None, Ip=None, params=None, spp=None, bounces=None,
           seed=None, nthreads: int = 0, metallic=_SCENE, normal=_SCENE, accel: bool = False):
    """FP64 forward render.  Returns (Ec, Ic), each (npix, 3) for a pixel list
    or (Hc, Wc, 3) for the full image.  ``metallic`` (Ht, Wt) and ``normal``
    (Ht, Wt, 3) default to the scene's maps; None = metallic 0 / no normal map.
    ``accel`` = timing mode (BVH; identical results)."""
    verts, tris, uv, albedo, rough, Ip = _scene_args(sc, albedo, rough, Ip)
    m, nm = _maps(sc, metallic, normal, albedo.shape[0], albedo.shape[1])
    P = make_params(params or sc.params)
    V = make_view(sc)
    full = pixels is None
    px = None if full else _c(pixels, np.int64)
    n = sc.Hc * sc.Wc if full else len(px)
    Ec = np.zeros((n, 3))
    Ic = np.zeros((n, 3))
    with _Accel(accel):
        rc = load().or_render_m(_p(verts), _p(tris), ctypes.c_int32(len(tris)), _p(uv), _p(albedo), _p(rough),
                                None if m is None else _p(m), None if nm is None else _p(nm),
                                ctypes.c_int32(albedo.shape[0]), ctypes.c_int32(albedo.shape[1]), _p(Ip),
                                ctypes.byref(V), ctypes.byref(P), ctypes.c_int32(spp or sc.spp),
                                ctypes.c_int32(sc.bounces if bounces is None else bounces),
                                ctypes.c_uint64(sc.seed if seed is None else seed),
                                None if full else _p(px), ctypes.c_int64(n), _p(Ec), _p(Ic), ctypes.c_int32(nthreads))
    if rc != 0:
        raise ValueError("oracle render: invalid arguments")
    if full:
        return Ec.reshape(sc.Hc, sc.Wc, 3), Ic.reshape(sc.Hc, sc.Wc, 3)
    return Ec, Ic


def render_backward(sc, dIc, pixels=None, *, albedo=None, rough=None, Ip=None, params=None, spp=None,
                    bounces=None, seed=None, nthreads: int = 0, metallic=_SCENE, normal=_SCENE, accel: bool = False,
                    unit_taps: bool = False):
    """FP64 adjoint.  ``dIc`` is (npix, 3) for a pixel list or (Hc, Wc, 3).
    Returns dict(dIp, dalbedo, drough, dparams[11]) plus dmetallic / dnormal
    where those maps are used (see ``render``).  ``accel`` = timing mode.
    ``unit_taps`` (a diagnostic, not the adjoint): projector and albedo
    contributions reach each of their four bilinear taps with weight 1."""
    verts, tris, uv, albedo, rough, Ip = _scene_args(sc, albedo, rough, Ip)
    m, nm = _maps(sc, metallic, normal, albedo.shape[0], albedo.shape[1])
    P = make_params(params or sc.params)
    V = make_view(sc)
    full = pixels is None
    px = None if full else _c(pixels, np.int64)
    n = sc.Hc * sc.Wc if full else len(px)
    dIc = _c(dIc, np.float64).reshape(n, 3)
    dIp = np.zeros(Ip.shape)
    dA = np.zeros(albedo.shape)
    dR = np.zeros(rough.shape)
    dM = None if m is None else np.zeros(m.shape)
    dN = None if nm is None else np.zeros(nm.shape)
    dP = np.zeros(11)
    load().or_set_unit_taps(ctypes.c_int(1 if unit_taps else 0))
    try:
        with _Accel(accel):
            rc = load().or_render_backward_m(
                _p(verts), _p(tris), ctypes.c_int32(len(tris)), _p(uv), _p(albedo), _p(rough),
                None if m is None else _p(m), None if nm is None else _p(nm),
                ctypes.c_int32(albedo.shape[0]), ctypes.c_int32(albedo.shape[1]), _p(Ip), ctypes.byref(V),
                ctypes.byref(P), ctypes.c_int32(spp or sc.spp), ctypes.c_int32(sc.bounces if bounces is None else bounces),
                ctypes.c_uint64(sc.seed if seed is None else seed), None if full else _p(px), ctypes.c_int64(n), _p(dIc),
                _p(dIp), _p(dA), _p(dR), None if dM is None else _p(dM), None if dN is None else _p(dN), _p(dP),
                ctypes.c_int32(nthreads))
    finally:
        load().or_set_unit_taps(ctypes.c_int(0))
    if rc != 0:
        raise ValueError("oracle render_backward: invalid arguments")
    out = {"dIp": dIp, "dalbedo": dA, "drough": dR, "dparams": dP}
    if dM is not None:
        out["dmetallic"] = dM
    if dN is not None:
        out["dnormal"] = dN
    return out


def crf_grad(Ec, params):
    """dIc/dEc of Eq. 5, Ic_j = (Gc w_j Ec_j)^gamma_c,j (0 where Gc w_j Ec_j <= 0),
    per pixel and channel; Ec is (..., 3)."""
    Ec = np.asarray(Ec, np.float64)
    gam = np.asarray(params.gamma_c, np.float64)
    a = float(params.gain_c) * np.asarray(params.wb, np.float64)
    x = a * Ec
    return np.where(x > 0.0, gam * a * np.power(np.maximum(x, 1e-300), gam - 1.0), 0.0)


def pose_backward(sc, dEc, twists, edge_spp, sil_spp, *, albedo=None, rough=None, Ip=None, params=None, spp=None,
                  bounces=None, seed=None, nthreads: int = 0, accel: bool = False, metallic=None, normal=None):
    """FP64 gradient of a loss with dLoss/dEc = ``dEc`` (Hc, Wc, 3) with
    respect to camera-pose parameters, each given by the twist (a, b) of the
    scene's motion in the camera frame (a point y moves with a x y + b);
    ``twists`` is (K, 6).  Returns (3, K): the interior, pixel-edge and
    silhouette terms (their sum is the gradient).  ``metallic`` (Ht, Wt) and
    ``normal`` (Ht, Wt, 3) select the principled material (default: none)."""
    verts, tris, uv, albedo, rough, Ip = _scene_args(sc, albedo, rough, Ip)
    m, nm = _maps(sc, metallic, normal, albedo.shape[0], albedo.shape[1])
    P = make_params(params or sc.params)
    V = make_view(sc)
    dEc = _c(dEc, np.float64).reshape(sc.Hc * sc.Wc, 3)
    tw = _c(twists, np.float64).reshape(-1, 6)
    out = np.zeros(3 * len(tw))
    with _Accel(accel):
        rc = load().or_pose_backward_m(
            _p(verts), _p(tris), ctypes.c_int32(len(tris)), _p(uv), _p(albedo), _p(rough),
            None if m is None else _p(m), None if nm is None else _p(nm),
            ctypes.c_int32(albedo.shape[0]), ctypes.c_int32(albedo.shape[1]), _p(Ip), ctypes.byref(V), ctypes.byref(P),
            ctypes.c_int32(spp or sc.spp), ctypes.c_int32(sc.bounces if bounces is None else bounces),
            ctypes.c_uint64(sc.seed if seed is None else seed), _p(dEc), ctypes.c_int32(len(tw)), _p(tw),
            ctypes.c_int32(edge_spp), ctypes.c_int32(sil_spp), _p(out), ctypes.c_int32(nthreads))
    if rc != 0:
        raise ValueError("oracle pose_backward: invalid arguments")
    return out.reshape(3, len(tw))


def adam_step(p, g, m, v, step, lr=1e-2, b1=0.9, b2=0.999, eps=1e-8, lo=0.0, hi=1.0):
    """Adam (Kingma & Ba 2015) with bias correction, then clamp to [lo, hi];
    in place on float64 arrays."""
    m *= b1
    m += (1.0 - b1) * g
    v *= b2
    v += (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    p -= lr * mh / (np.sqrt(vh) + eps)
    np.clip(p, lo, hi, out=p)
    return p


# ---------------------------------------------------------------------------
# Eq. 11: Ic' = D(Ic), a cross-bilateral filter.  The paper names the filter
# (a differentiable cross-bilateral filter) but not its guide, window or
# widths; the reading taken here:
#   D(I)(p) = sum_q w(p,q) I(q) / W(p),  W(p) = sum_q w(p,q),
#   w(p,q)  = exp(-|p-q|^2 / (2 s_s^2) - sum_f |g_f(p) - g_f(q)|^2 / (2 s_f^2)),
# q over the (2r+1)^2 window around p that lies inside the image, g_f the
# guide features of gbuffer() (albedo, normal, depth); a width <= 0 drops
# its feature.  The weights depend on the guide only, so D is linear in I and
# its adjoint is dI(q) = sum_p w(p,q) dD(p) / W(p).
# ---------------------------------------------------------------------------
def gbuffer(sc, albedo=None, nthreads: int = 0):
    """First-hit guide through each camera pixel centre: (Hc, Wc, 8) =
    albedo rgb, normal xyz (towards the camera), hit distance, hit flag."""
    verts, tris, uv = _c(sc.verts, np.float32), _c(sc.tris, np.int32), _c(sc.uv, np.float32)
    albedo = _c(sc.albedo if albedo is None else albedo, np.float64)
    V = make_view(sc)
    g = np.zeros((sc.Hc, sc.Wc, 8))
    rc = load().or_gbuffer(_p(verts), _p(tris), ctypes.c_int32(len(tris)), _p(uv), _p(albedo),
                           ctypes.c_int32(albedo.shape[0]), ctypes.c_int32(albedo.shape[1]), ctypes.byref(V), _p(g),
                           ctypes.c_int32(nthreads))
    if rc != 0:
        raise ValueError("oracle gbuffer: invalid arguments")
    return g


_FEATURES = (("sigma_albedo", slice(0, 3)), ("sigma_normal", slice(3, 6)), ("sigma_depth", slice(6, 7)))


def _bilateral_weight(guide, p_sl, q_sl, dy, dx, prm):
    """w(p, q) for every p in the window slice p_sl with q = p + (dy, dx)."""
    e = (dx * dx + dy * dy) / (2.0 * prm["sigma_s"] ** 2)
    for name, fs in _FEATURES:
        s = prm[name]
        if s > 0.0:
            diff = guide[p_sl][..., fs] - guide[q_sl][..., fs]
            e = e + np.sum(diff * diff, axis=-1) / (2.0 * s * s)
    return np.exp(-e)


def _offsets(H, W, r):
    """(dy, dx, p-slices, q-slices) of every window offset, q = p + (dy, dx)."""
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            if abs(dy) >= H or abs(dx) >= W:
                continue  # no pixel pair this far apart inside the image
            py = slice(max(0, -dy), min(H, H - dy))
            px = slice(max(0, -dx), min(W, W - dx))
            qy = slice(py.start + dy, py.stop + dy)
            qx = slice(px.start + dx, px.stop + dx)
            yield dy, dx, (py, px), (qy, qx)


def denoise(I, guide, prm):
    """FP64 cross-bilateral filter of Eq. 11.  I (H, W, 3), guide (H, W, 8),
    prm dict(radius, sigma_s, sigma_albedo, sigma_normal, sigma_depth).
    Returns (D(I), W) with W the per-pixel weight sum."""
    I = np.asarray(I, np.float64)
    guide = np.asarray(guide, np.float64)
    H, W = I.shape[:2]
    num = np.zeros((H, W, 3))
    den = np.zeros((H, W))
    for dy, dx, ps, qs in _offsets(H, W, int(prm["radius"])):
        w = _bilateral_weight(guide, ps, qs, dy, dx, prm)
        num[ps] += w[..., None] * I[qs]
        den[ps] += w
    return num / den[..., None], den


def denoise_backward(dout, guide, prm):
    """Adjoint of denoise(): dI(q) = sum_p w(p,q) dout(p) / W(p), scattered
    from every output pixel p to the inputs q it read."""
    dout = np.asarray(dout, np.float64)
    guide = np.asarray(guide, np.float64)
    H, W = dout.shape[:2]
    den = np.zeros((H, W))
    for dy, dx, ps, qs in _offsets(H, W, int(prm["radius"])):
        den[ps] += _bilateral_weight(guide, ps, qs, dy, dx, prm)
    g = dout / den[..., None]
    dI = np.zeros((H, W, 3))
    for dy, dx, ps, qs in _offsets(H, W, int(prm["radius"])):
        w = _bilateral_weight(guide, ps, qs, dy, dx, prm)
        dI[qs] += w[..., None] * g[ps]
    return dI


# ---------------------------------------------------------------------------
# Eq. 9: theta* = argmin (1/K) sum_i |R(Ip_i, theta) - Ic_i| + lambda L(m).
# Readings: |.| is the L1 norm (scaled by the caller, e.g. 1/(K n) for a
# mean), L(m) the anisotropic total variation of a BRDF map over right and
# down neighbours.  sign(0) = 0 in both subgradients.
# ---------------------------------------------------------------------------
def l1_loss(I, target, scale=1.0):
    """(scale * sum |I - target|, scale * sign(I - target))."""
    d = np.asarray(I, np.float64) - np.asarray(target, np.float64)
    return scale * float(np.sum(np.abs(d))), scale * np.sign(d)


def tv_loss(m, weight=1.0):
    """(weight * sum |m(x+1,y) - m(x,y)| + |m(x,y+1) - m(x,y)|, its
    subgradient) for m of shape (H, W) or (H, W, C).  The subgradient is
    scattered difference by difference: each difference d = m(q) - m(p) adds
    sign(d) to q and subtracts it from p."""
    m = np.asarray(m, np.float64)
    dx = m[:, 1:] - m[:, :-1]
    dy = m[1:, :] - m[:-1, :]
    loss = weight * (float(np.sum(np.abs(dx))) + float(np.sum(np.abs(dy))))
    g = np.zeros_like(m)
    g[:, 1:] += np.sign(dx)
    g[:, :-1] -= np.sign(dx)
    g[1:, :] += np.sign(dy)
    g[:-1, :] -= np.sign(dy)
    return loss, weight * g
