"""Seeded synthetic inputs for the DPCS path tracer.

This module only builds inputs: triangle meshes with per-vertex UVs, albedo and
roughness textures, projector images, camera/projector intrinsics and
extrinsics, and parameter sets.  It holds none of the rendering arithmetic, so
both the CUDA library and the FP64 oracle can consume exactly the same arrays.

The paper (arxiv 2503.12174, Sec. 4) renders Poisson-reconstructed meshes of
real scenes captured with an 800x600 projector and a 640x360 camera.  Those
captures are not available; the scenes here stand in for them:

* ``plane``       -- one quad (2 triangles) at z = 1 facing a pinhole camera and
                     projector 0.3 apart, direct light only (Eqs. 1-6).
* ``corner``      -- three orthogonal 1 m planes (13x13 quad grids) plus an
                     occluding box, T = 1026, Lambert+GGX with smooth noise
                     textures; exercises interreflection (Eq. 3).
* ``heightfield`` -- a 317x317-vertex displaced surface, T = 199,712.
* ``sphere``      -- a closed icosphere around camera and projector, used for
                     the integrating-sphere closed form.

All randomness comes from ``numpy.random.default_rng(seed)``.  Camera
convention: pinhole at the world origin, OpenCV axes (+z forward, +y down),
pixel (i, j) spans [i, i+1) x [j, j+1).  Matrices are row-major float32.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Params:
    """Response, BRDF and sampling parameters (mirror of the C ``dpcs_params``)."""

    gamma_p: tuple = (2.2, 2.2, 2.2)   # Eq. 1 projector gamma per channel
    gain_p: float = 1.0                # Eq. 1 projector gain Gp
    gamma_c: tuple = (1.0, 1.0, 1.0)   # Eq. 5 camera gamma per channel
    gain_c: float = 1.0                # Eq. 5 camera exposure Gc
    wb: tuple = (1.0, 1.0, 1.0)        # Eq. 5 white balance w
    k_proj: float = 1.0                # Eq. 2 / Eq. 12 projector intensity scale k
    ks: float = 0.0                    # GGX lobe weight
    f0: float = 0.04                   # Schlick F0
    rr_start: int = 0                  # first vertex subject to Russian roulette (0 = off)
    rr_q: float = 1.0                  # RR survival probability
    clip: float = 0.0                  # Eq. 12 radiance clip (0 = off)
    jitter: int = 1                    # 1 = box-filter jitter, 0 = pixel centre


@dataclasses.dataclass
class Scene:
    """A complete render input."""

    verts: np.ndarray      # (V, 3) float32
    tris: np.ndarray       # (T, 3) int32
    uv: np.ndarray         # (V, 2) float32, u along texture x, v along texture y (down)
    albedo: np.ndarray     # (Ht, Wt, 3) float32
    rough: np.ndarray      # (Ht, Wt) float32
    Ip: np.ndarray         # (Hp, Wp, 3) float32 projector input image
    Kc: np.ndarray         # (3, 3) float32
    Hc: int
    Wc: int
    Kp: np.ndarray         # (3, 3) float32
    Rp: np.ndarray         # (3, 3) float32, world -> projector rotation
    tp: np.ndarray         # (3,) float32, world -> projector translation
    params: Params
    spp: int
    bounces: int
    seed: int
    name: str = ""
    metallic: np.ndarray | None = None  # (Ht, Wt) float32 in [0, 1]; None = 0 everywhere
    normal: np.ndarray | None = None    # (Ht, Wt, 3) float32 normal map in [0, 1]^3; None = unperturbed

    @property
    def Hp(self) -> int:
        return int(self.Ip.shape[0])

    @property
    def Wp(self) -> int:
        return int(self.Ip.shape[1])

    @property
    def Ht(self) -> int:
        return int(self.albedo.shape[0])

    @property
    def Wt(self) -> int:
        return int(self.albedo.shape[1])

    @property
    def T(self) -> int:
        return int(self.tris.shape[0])

    @property
    def n_samples(self) -> int:
        return self.Hc * self.Wc * self.spp

    def replace(self, **kw) -> "Scene":
        return dataclasses.replace(self, **kw)


# ---------------------------------------------------------------------------
# intrinsics / extrinsics
# ---------------------------------------------------------------------------
def intrinsics(W: int, H: int, hfov_deg: float) -> np.ndarray:
    """Pinhole K with square pixels, horizontal field of view, centred principal point."""
    f = (W / 2.0) / math.tan(math.radians(hfov_deg) / 2.0)
    return np.array([[f, 0.0, W / 2.0], [0.0, f, H / 2.0], [0.0, 0.0, 1.0]], np.float32)


def look_at(centre, target, up=(0.0, -1.0, 0.0)):
    """World -> device rotation R and translation t (x_dev = R x_world + t) for a
    device at ``centre`` whose +z axis points at ``target`` (OpenCV: +y down)."""
    c = np.asarray(centre, np.float64)
    z = np.asarray(target, np.float64) - c
    z /= np.linalg.norm(z)
    u = np.asarray(up, np.float64)
    x = np.cross(-u, z)  # +x to the right when +y is down
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    t = -R @ c
    return R.astype(np.float32), t.astype(np.float32)


# ---------------------------------------------------------------------------
# textures and projector images
# ---------------------------------------------------------------------------
def smooth_noise(rng, H: int, W: int, octaves: int = 4, base: int = 4) -> np.ndarray:
    """Perlin-style smooth noise in [0, 1]: octaves of bicubically smoothed
    value noise on coarse lattices, summed with halving amplitude."""
    out = np.zeros((H, W), np.float64)
    amp, total = 1.0, 0.0
    ys = (np.arange(H) + 0.5) / H
    xs = (np.arange(W) + 0.5) / W
    for o in range(octaves):
        n = base * (2 ** o)
        lat = rng.random((n + 3, n + 3))
        gy = ys * n
        gx = xs * n
        iy = np.floor(gy).astype(int)
        ix = np.floor(gx).astype(int)
        fy = gy - iy
        fx = gx - ix
        sy = fy * fy * (3 - 2 * fy)  # smoothstep fade
        sx = fx * fx * (3 - 2 * fx)
        a = lat[iy[:, None], ix[None, :]]
        b = lat[iy[:, None], ix[None, :] + 1]
        c = lat[iy[:, None] + 1, ix[None, :]]
        d = lat[iy[:, None] + 1, ix[None, :] + 1]
        top = a + (b - a) * sx[None, :]
        bot = c + (d - c) * sx[None, :]
        out += amp * (top + (bot - top) * sy[:, None])
        total += amp
        amp *= 0.5
    out /= total
    lo, hi = out.min(), out.max()
    return (out - lo) / max(hi - lo, 1e-12)


def blob_image(rng, H: int, W: int, n_blobs: int = 8) -> np.ndarray:
    """Projector image of random smooth coloured Gaussian blobs, rescaled to [0, 1]."""
    yy, xx = np.meshgrid((np.arange(H) + 0.5) / H, (np.arange(W) + 0.5) / W, indexing="ij")
    img = np.zeros((H, W, 3), np.float64)
    for _ in range(n_blobs):
        cx, cy = rng.random(2)
        s = 0.05 + 0.25 * rng.random()
        col = rng.random(3)
        g = np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * s * s))
        img += g[..., None] * col[None, None, :]
    for j in range(3):
        ch = img[..., j]
        img[..., j] = (ch - ch.min()) / max(ch.max() - ch.min(), 1e-12)
    return img.astype(np.float32)


# ---------------------------------------------------------------------------
# meshes
# ---------------------------------------------------------------------------
def _grid(p0, du, dv, n: int, uv0, uv_size):
    """n x n quad grid spanning p0 + s du + t dv, s, t in [0, 1]; UVs map into
    the atlas rectangle uv0 + (s, t) * uv_size."""
    s = np.linspace(0.0, 1.0, n + 1)
    S, Tt = np.meshgrid(s, s, indexing="xy")
    P = (np.asarray(p0)[None, None, :] + S[..., None] * np.asarray(du)[None, None, :]
         + Tt[..., None] * np.asarray(dv)[None, None, :])
    verts = P.reshape(-1, 3)
    uv = np.stack([uv0[0] + S * uv_size[0], uv0[1] + Tt * uv_size[1]], -1).reshape(-1, 2)
    tris = []
    for j in range(n):
        for i in range(n):
            a = j * (n + 1) + i
            b, c, d = a + 1, a + n + 2, a + n + 1
            tris.append((a, b, c))
            tris.append((a, c, d))
    return verts, np.asarray(tris, np.int64), uv


def _merge(parts):
    verts, tris, uvs, off = [], [], [], 0
    for v, t, u in parts:
        verts.append(v)
        tris.append(t + off)
        uvs.append(u)
        off += len(v)
    return (np.concatenate(verts).astype(np.float32), np.concatenate(tris).astype(np.int32),
            np.concatenate(uvs).astype(np.float32))


def _box(centre, half, yaw_deg, uv0, uv_size):
    """Box with 12 triangles, rotated about the y axis; every face maps to the
    same atlas rectangle."""
    c = np.asarray(centre, np.float64)
    a = math.radians(yaw_deg)
    R = np.array([[math.cos(a), 0, math.sin(a)], [0, 1, 0], [-math.sin(a), 0, math.cos(a)]])
    h = np.asarray(half, np.float64)
    faces = []
    for axis in range(3):
        for sgn in (-1.0, 1.0):
            u_ax, v_ax = [k for k in range(3) if k != axis]
            p0 = np.zeros(3); p0[axis] = sgn * h[axis]; p0[u_ax] = -h[u_ax]; p0[v_ax] = -h[v_ax]
            du = np.zeros(3); du[u_ax] = 2 * h[u_ax]
            dv = np.zeros(3); dv[v_ax] = 2 * h[v_ax]
            v, t, u = _grid(p0, du, dv, 1, uv0, uv_size)
            v = (R @ v.T).T + c
            faces.append((v, t, u))
    return _merge(faces)


def icosphere(subdiv: int, radius: float = 1.0):
    """Icosahedron subdivided ``subdiv`` times and projected to the sphere."""
    t = (1.0 + 5 ** 0.5) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
         (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11),
         (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.asarray(p, np.float64) / np.linalg.norm(p) for p in v]
    faces = list(f)
    for _ in range(subdiv):
        cache, nf = {}, []

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.asarray(verts) * radius
    uv = np.zeros((len(V), 2))
    uv[:, 0] = 0.5 + np.arctan2(V[:, 0], V[:, 2]) / (2 * math.pi)
    uv[:, 1] = np.arccos(np.clip(V[:, 1] / radius, -1, 1)) / math.pi
    return V.astype(np.float32), np.asarray(faces, np.int32), uv.astype(np.float32)


def heightfield_mesh(rng, n_vert: int = 317, half: float = 1.0, z0: float = 1.5, amp: float = 0.1):
    """Displaced surface z = z0 + h(x, y): four seeded sinusoids plus a
    5-octave fBm, scaled so max |h| = amp."""
    s = np.linspace(-half, half, n_vert)
    X, Y = np.meshgrid(s, s, indexing="xy")
    h = np.zeros_like(X)
    for _ in range(4):
        kx, ky = rng.uniform(1.0, 6.0, 2) * rng.choice([-1, 1], 2)
        ph = rng.uniform(0, 2 * math.pi)
        h += rng.uniform(0.3, 1.0) * np.sin(kx * X + ky * Y + ph)
    fbm = smooth_noise(rng, n_vert, n_vert, octaves=5, base=6) * 2.0 - 1.0
    h += 1.5 * fbm
    h *= amp / np.abs(h).max()
    verts = np.stack([X, Y, z0 + h], -1).reshape(-1, 3)
    uv = np.stack([(X + half) / (2 * half), (Y + half) / (2 * half)], -1).reshape(-1, 2)
    n = n_vert - 1
    idx = np.arange(n_vert * n_vert).reshape(n_vert, n_vert)
    a = idx[:n, :n].ravel()
    b = idx[:n, 1:].ravel()
    c = idx[1:, 1:].ravel()
    d = idx[1:, :n].ravel()
    tris = np.stack([np.stack([a, b, c], -1), np.stack([a, c, d], -1)], 1).reshape(-1, 3)
    return verts.astype(np.float32), tris.astype(np.int32), uv.astype(np.float32)


# ---------------------------------------------------------------------------
# the workloads
# ---------------------------------------------------------------------------
def plane(res: int = 64, spp: int = 4, seed: int = 0, ip_seed: int = 0) -> Scene:
    """Direct light on one quad: 2 triangles at z = 1, camera at the origin,
    projector at (0.3, 0, 0) with Rp = I; 40 degree field of view; albedo 0.5;
    Ip uniform random in [0, 1]; gamma_p 2.2, linear CRF, white balance 1;
    1 bounce, ``spp`` samples, Philox seed ``seed``."""
    rng = np.random.default_rng(ip_seed)
    verts = np.array([[-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], np.float32)
    tris = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    uv = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], np.float32)
    K = intrinsics(res, res, 40.0)
    return Scene(verts=verts, tris=tris, uv=uv,
                 albedo=np.full((64, 64, 3), 0.5, np.float32), rough=np.full((64, 64), 0.5, np.float32),
                 Ip=rng.random((res, res, 3), dtype=np.float32), Kc=K, Hc=res, Wc=res, Kp=K.copy(),
                 Rp=np.eye(3, dtype=np.float32), tp=np.array([-0.3, 0, 0], np.float32),
                 params=Params(gamma_p=(2.2, 2.2, 2.2)), spp=spp, bounces=1, seed=seed, name=f"plane{res}")


def corner_mesh():
    back = _grid((-0.5, -0.5, 1.6), (1.0, 0, 0), (0, 1.0, 0), 13, (0.0, 0.0), (0.5, 0.5))
    floor = _grid((-0.5, 0.5, 1.6), (1.0, 0, 0), (0, 0, -1.0), 13, (0.5, 0.0), (0.5, 0.5))
    left = _grid((-0.5, -0.5, 0.6), (0, 0, 1.0), (0, 1.0, 0), 13, (0.0, 0.5), (0.5, 0.5))
    box = _box((0.08, 0.3745, 1.15), (0.125, 0.125, 0.125), 30.0, (0.5, 0.5), (0.5, 0.5))
    return _merge([back, floor, left, box])


def corner(res: int = 256, tex: int | None = None, spp: int = 64, bounces: int = 3, seed: int = 0,
           scene_seed: int = 1) -> Scene:
    """Interreflection corner: three orthogonal 1 m planes (13x13 quads each,
    338 triangles) and a 12-triangle occluding box, T = 1026.  Albedo
    textures in [0.2, 0.9] and roughness in [0.1, 0.8] from smooth noise;
    Ip = 8 random Gaussian blobs in [0, 1]; Lambert + GGX."""
    tex = tex or res
    rng = np.random.default_rng(scene_seed)
    verts, tris, uv = corner_mesh()
    albedo = np.stack([0.2 + 0.7 * smooth_noise(rng, tex, tex) for _ in range(3)], -1).astype(np.float32)
    rough = (0.1 + 0.7 * smooth_noise(rng, tex, tex)).astype(np.float32)
    Ip = blob_image(rng, res, res)
    Kc = intrinsics(res, res, 40.0)
    Rp, tp = look_at((0.25, -0.15, 0.0), (-0.05, 0.1, 1.3))
    params = Params(gamma_p=(2.2, 2.4, 2.0), gain_p=1.0, gamma_c=(0.45, 0.5, 0.55), gain_c=4.0,
                    wb=(1.1, 1.0, 0.9), k_proj=4.0, ks=1.0, f0=0.04)
    return Scene(verts=verts, tris=tris, uv=uv, albedo=albedo, rough=rough, Ip=Ip, Kc=Kc, Hc=res, Wc=res,
                 Kp=intrinsics(res, res, 45.0), Rp=Rp, tp=tp, params=params, spp=spp, bounces=bounces,
                 seed=seed, name=f"corner{res}")


def compensation(res: int = 512, spp: int = 16, seed: int = 0) -> Scene:
    """Projector compensation workload: the corner scene at ``res`` for camera,
    projector and textures, 16 spp, 3 bounces."""
    return corner(res=res, tex=res, spp=spp, bounces=3, seed=seed).replace(name=f"compensation{res}")


def heightfield(spp: int = 256, seed: int = 0, scene_seed: int = 4, cam: int = 1024, proj=(768, 1024),
                tex: int = 512, n_vert: int = 317) -> Scene:
    """Large displaced surface: 317x317 vertices (T = 199,712), amplitude 0.1;
    projector 1024x768, camera 1024x1024, textures 512x512; 4 bounces with
    Russian roulette after vertex 2 (q = 0.75)."""
    rng = np.random.default_rng(scene_seed)
    verts, tris, uv = heightfield_mesh(rng, n_vert=n_vert)
    albedo = np.stack([0.2 + 0.7 * smooth_noise(rng, tex, tex) for _ in range(3)], -1).astype(np.float32)
    rough = (0.1 + 0.7 * smooth_noise(rng, tex, tex)).astype(np.float32)
    Hp, Wp = proj
    Ip = blob_image(rng, Hp, Wp)
    Rp, tp = look_at((0.3, -0.2, 0.0), (0.0, 0.0, 1.5))
    params = Params(gamma_p=(2.2, 2.4, 2.0), gamma_c=(0.45, 0.5, 0.55), gain_c=3.0, wb=(1.1, 1.0, 0.9),
                    k_proj=4.0, ks=1.0, f0=0.04, rr_start=2, rr_q=0.75)
    return Scene(verts=verts, tris=tris, uv=uv, albedo=albedo, rough=rough, Ip=Ip,
                 Kc=intrinsics(cam, cam, 62.0), Hc=cam, Wc=cam, Kp=intrinsics(Wp, Hp, 50.0), Rp=Rp, tp=tp,
                 params=params, spp=spp, bounces=4, seed=seed, name=f"heightfield{cam}")


def sphere(subdiv: int = 4, res: int = 32, spp: int = 64, bounces: int = 3, albedo: float = 0.5,
           ip_value: float = 0.8, seed: int = 0) -> Scene:
    """Integrating sphere: camera at the centre of a closed unit icosphere,
    projector at (0.2, 0, 0) looking along +z, uniform Lambertian albedo,
    uniform Ip, gamma_p = 1, linear CRF."""
    verts, tris, uv = icosphere(subdiv)
    K = intrinsics(res, res, 40.0)
    return Scene(verts=verts, tris=tris, uv=uv, albedo=np.full((8, 8, 3), albedo, np.float32),
                 rough=np.full((8, 8), 0.5, np.float32), Ip=np.full((res, res, 3), ip_value, np.float32),
                 Kc=K, Hc=res, Wc=res, Kp=K.copy(), Rp=np.eye(3, dtype=np.float32),
                 tp=np.array([-0.2, 0.0, 0.0], np.float32),
                 params=Params(gamma_p=(1.0, 1.0, 1.0), ks=0.0), spp=spp, bounces=bounces, seed=seed,
                 name=f"sphere{subdiv}")


CONFIGS = {
    "plane": plane,
    "corner": corner,
    "compensation": compensation,
    "heightfield": heightfield,
}


def principled_maps(rng, Ht: int, Wt: int, metal_max: float = 0.8, bump: float = 0.35):
    """Seeded maps of the principled material (Sec. 3.2, Sec. 4.3): metallic
    in [0, metal_max] from smooth noise, and a normal map from the slopes of
    a smooth bump field h (tangent-space normal (-bump dh/du, -bump dh/dv, 1)
    normalised, stored as (n + 1) / 2 in [0, 1]^3)."""
    metallic = (metal_max * smooth_noise(rng, Ht, Wt)).astype(np.float32)
    h = smooth_noise(rng, Ht, Wt)
    dhdv, dhdu = np.gradient(h)
    n = np.stack([-bump * dhdu * Wt / 8.0, -bump * dhdv * Ht / 8.0, np.ones_like(h)], -1)
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    return metallic, ((n + 1.0) * 0.5).astype(np.float32)


def with_principled(sc: Scene, seed: int = 21, **kw) -> Scene:
    """``sc`` with seeded metallic and normal maps of its texture size."""
    metallic, normal = principled_maps(np.random.default_rng(seed), sc.Ht, sc.Wt, **kw)
    return sc.replace(metallic=metallic, normal=normal)
