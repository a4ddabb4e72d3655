"""Pins of the oracle's camera-pose gradient (Sec. 3.2 counts the pose Rc, tc
among the scene parameters theta).  ``oracle.pose_backward`` splits the
derivative of the box-filtered pixel means (Eq. 4) into an interior term, a
pixel-edge term and a silhouette term; these tests hold the sum to values
fixed outside that split:
  - the motion ``pose.twists`` hands it equals the derivative of the posed
    points (central differences of pose_of);
  - on a glossy plane that fills the view, lit everywhere by a wide
    projector (no discontinuity in the image), the gradient equals the
    derivative of the closed-form direct light integrated over each pixel by
    Gauss-Legendre quadrature, within the Monte Carlo error of the estimate;
  - where a nearer quad hides a farther one, the gradient equals the
    derivative of the oracle's own rendered image taken by central
    differences with common random numbers (which sees the silhouette's
    motion as samples that change sides), and the silhouette term is
    needed for that agreement;
  - a rotation about the camera centre moves both sides of a silhouette
    alike, so the silhouette term vanishes."""
import math

import numpy as np
import pytest

from paper_2503_12174_gb300 import pose, scenes


def test_twists_are_the_motion_of_the_posed_points():
    rng = np.random.default_rng(0)
    R0, t0 = pose.rotation([0.1, -0.2, 0.3]), np.array([0.1, 0.2, -0.3])
    for xi in [rng.normal(size=6) * 0.3, np.zeros(6), np.array([1e-7, 0.0, 2e-7, 0.1, 0.0, 0.0])]:
        tw = pose.twists(xi, R0, t0)
        for x in rng.normal(size=(4, 3)):
            def y(z):
                R, t = pose.pose_of(z, R0, t0)
                return R @ x + t
            for k in range(6):
                e = np.zeros(6)
                e[k] = 1e-6
                fd = (y(xi + e) - y(xi - e)) / 2e-6
                np.testing.assert_allclose(np.cross(tw[k, :3], y(xi)) + tw[k, 3:], fd, atol=1e-8)


def _ggx_brdf(n, wo, wi, rho, r, ks, f0):
    """Lambert + GGX (alpha = r^2, separable Smith masking, Schlick Fresnel)."""
    co, ci = np.sum(n * wo, -1), np.sum(n * wi, -1)
    a = min(max(r, 0.01), 1.0) ** 2
    h = wo + wi
    h = h / np.linalg.norm(h, axis=-1, keepdims=True)
    ch = np.sum(n * h, -1)
    D = a * a / (math.pi * (ch * ch * (a * a - 1.0) + 1.0) ** 2)

    def G1(c):
        return 2.0 * c / (c + np.sqrt(a * a + (1.0 - a * a) * c * c))
    F = f0 + (1.0 - f0) * np.clip(1.0 - np.sum(wo * h, -1), 0.0, None) ** 5
    spec = ks * D * G1(ci) * G1(co) * F / (4.0 * ci * co)
    return rho / math.pi + np.where((co > 0) & (ci > 0), spec, 0.0)


def _plane_radiance(sc, R, t, pts, c, gamma, k, gain, rho, r, ks, f0):
    """Direct light reaching image points pts (N, 2) from the plane z = 1 of
    ``sc`` seen from a camera at pose (R, t), constant projector input c."""
    Kinv = np.linalg.inv(np.asarray(sc.Kc, np.float64))
    d = np.concatenate([pts, np.ones((len(pts), 1))], -1) @ Kinv.T
    d = d / np.linalg.norm(d, axis=-1, keepdims=True)
    n = R @ np.array([0.0, 0.0, 1.0])
    p0 = R @ np.array([0.0, 0.0, 1.0]) + t
    x = d * ((p0 @ n) / (d @ n))[:, None]
    Rp = np.asarray(sc.Rp, np.float64)
    cp = R @ (-Rp.T @ np.asarray(sc.tp, np.float64)) + t
    axis = R @ (Rp.T @ np.array([0.0, 0.0, 1.0]))
    v = cp - x
    dist = np.linalg.norm(v, axis=-1)
    wp = v / dist[:, None]
    nf = np.where(((d @ n) > 0)[:, None], -n, n)
    cos_s = np.sum(nf * wp, -1)
    cos_p = ((x - cp) @ axis) / dist
    return _ggx_brdf(nf, -d, wp, rho, r, ks, f0) * k * gain * c ** gamma * cos_p * cos_s / dist ** 2


def _posed(sc, xi, R0, t0):
    R, t = pose.pose_of(xi, R0, t0)
    Rp2, tp2 = pose.posed_extrinsics(sc.Rp, sc.tp, R, t)
    return sc.replace(verts=(sc.verts.astype(np.float64) @ R.T + t).astype(np.float32), Rp=Rp2.astype(np.float32),
                      tp=tp2.astype(np.float32))


def test_plane_pose_gradient_equals_the_closed_form_pixel_integrals(orc):
    res = 16
    f32 = lambda v: float(np.float32(v))  # noqa: E731  (the oracle reads the float32 inputs)
    sc = scenes.plane(res=res)
    sc = sc.replace(Ip=np.full((res, res, 3), 0.6, np.float32), albedo=np.full((8, 8, 3), 0.5, np.float32),
                    rough=np.full((8, 8), 0.3, np.float32), Kp=scenes.intrinsics(res, res, 80.0),
                    params=scenes.Params(gamma_p=(2.2,) * 3, gain_p=1.1, k_proj=1.3, ks=0.8, f0=0.04, jitter=1))
    W = np.random.default_rng(3).uniform(0.5, 1.5, (res, res, 3))
    R0, t0 = pose.rotation([0.02, -0.03, 0.1]), np.array([0.01, 0.02, 0.05])
    xi = np.array([0.01, 0.0, -0.02, 0.005, 0.0, 0.01])
    # Gauss-Legendre 6 x 6 over each pixel's square
    gx, gw = np.polynomial.legendre.leggauss(6)
    gx, gw = 0.5 * (gx + 1.0), 0.5 * gw
    ys, xs = np.mgrid[0:res, 0:res]
    sub = np.stack(np.meshgrid(gx, gx, indexing="xy"), -1)
    pts = (np.stack([xs, ys], -1)[:, :, None, None, :] + sub[None, None]).reshape(-1, 2)
    wts = (gw[None, :] * gw[:, None]).ravel()

    def psi(x):
        R, t = pose.pose_of(x, R0, t0)
        L = _plane_radiance(sc, R, t, pts, f32(0.6), 2.2, 1.3, f32(1.1), f32(0.5), f32(0.3), 0.8, 0.04)
        return float(np.sum(W * (L.reshape(res, res, -1) * wts).sum(-1)[..., None]))

    truth = pose.central_differences(psi, xi, 1e-4)
    psc = _posed(sc, xi, R0, t0)
    tw = pose.twists(xi, R0, t0)
    est = np.array([orc.pose_backward(psc, W, tw, 64, 0, spp=256, seed=s).sum(0) for s in range(8)])
    mean, se = est.mean(0), est.std(0, ddof=1) / math.sqrt(len(est))
    scale = np.abs(truth).max()
    assert scale > 1.0
    assert np.all(np.abs(mean - truth) <= 5.0 * se + 2e-4 * scale), (mean, truth, se)


def _quad(c, half, z, rot_deg):
    cs, sn = math.cos(math.radians(rot_deg)), math.sin(math.radians(rot_deg))
    return np.array([[c[0] + cs * half * u - sn * half * v, c[1] + sn * half * u + cs * half * v, z]
                     for u, v in [(-1, -1), (1, -1), (1, 1), (-1, 1)]], np.float32)


def _occluder_scene(res=24):
    """A quad at z = 1.2 (turned 20 degrees) in front of a wide quad at z = 2,
    both lit directly by a wide projector; Lambert, one bounce."""
    verts = np.concatenate([_quad((0.0, 0.0), 2.0, 2.0, 0.0), _quad((0.05, -0.03), 0.18, 1.2, 20.0)])
    tris = np.array([[0, 1, 2], [0, 2, 3], [4, 5, 6], [4, 6, 7]], np.int32)
    uv = np.array([[0, 0], [1, 0], [1, 1], [0, 1]] * 2, np.float32)
    return scenes.Scene(verts=verts, tris=tris, uv=uv, albedo=np.full((8, 8, 3), 0.6, np.float32),
                        rough=np.full((8, 8), 0.4, np.float32), Ip=np.full((16, 16, 3), 0.7, np.float32),
                        Kc=scenes.intrinsics(res, res, 40.0), Hc=res, Wc=res, Kp=scenes.intrinsics(16, 16, 80.0),
                        Rp=np.eye(3, dtype=np.float32), tp=np.array([-0.3, 0.1, 0.0], np.float32),
                        params=scenes.Params(gamma_p=(2.2,) * 3, k_proj=2.0, ks=0.0, jitter=1), spp=64, bounces=1,
                        seed=0, name="occluder")


def test_silhouette_term_matches_common_random_number_differences(orc):
    sc = _occluder_scene()
    W = np.random.default_rng(5).uniform(0.5, 1.5, (sc.Hc, sc.Wc, 3))
    R0, t0 = pose.rotation([0.01, -0.02, 0.05]), np.array([0.01, -0.02, 0.03])
    # h small enough that the differences' O(h^2) bias stays well inside the
    # noise (the silhouette moves by about a tenth of a pixel)
    xi, ks, h, spp, nseed = np.zeros(6), [3, 5], 4e-3, 16384, 6
    tw = pose.twists(xi, R0, t0)[ks]
    fd, est = [], []
    for seed in range(nseed):
        row = []
        for k in ks:
            e = np.zeros(6)
            e[k] = h
            Ep, _ = orc.render(_posed(sc, xi + e, R0, t0), spp=spp, seed=seed)
            Em, _ = orc.render(_posed(sc, xi - e, R0, t0), spp=spp, seed=seed)
            row.append(np.sum(W * (Ep - Em)) / (2.0 * h))
        fd.append(row)
        est.append(orc.pose_backward(_posed(sc, xi, R0, t0), W, tw, 64, 64, spp=256, seed=seed))
    fd, est = np.array(fd), np.array(est)
    se = (fd.std(0, ddof=1) + est.sum(1).std(0, ddof=1)) / math.sqrt(nseed)
    tol = 5.0 * se
    full, no_sil = est.sum(1).mean(0), est[:, :2].sum(1).mean(0)
    assert np.all(np.abs(full - fd.mean(0)) <= tol), (full, fd.mean(0), tol)
    # the silhouette term carries a visible share of the translation along y
    assert abs(no_sil[0] - fd.mean(0)[0]) > 2.0 * tol[0], (no_sil, fd.mean(0), tol)


def test_rotation_about_the_camera_centre_has_no_silhouette_term(orc):
    sc = _occluder_scene(res=16)
    W = np.random.default_rng(6).uniform(0.5, 1.5, (16, 16, 3))
    tw = np.zeros((3, 6))
    tw[:, :3] = np.eye(3)
    out = orc.pose_backward(sc, W, tw, 0, 64, spp=4, seed=0)
    assert np.abs(out[2]).max() <= 1e-6 * np.abs(out[0]).max()
    assert np.abs(out[0]).max() > 0.0


def _principled_plane():
    res = 16
    sc = scenes.plane(res=res)
    return sc.replace(Ip=np.full((res, res, 3), 0.6, np.float32), albedo=np.full((8, 8, 3), 0.5, np.float32),
                      rough=np.full((8, 8), 0.3, np.float32), Kp=scenes.intrinsics(res, res, 80.0),
                      params=scenes.Params(gamma_p=(2.2,) * 3, gain_p=1.1, k_proj=1.3, ks=0.8, f0=0.04, jitter=1))


def test_flat_principled_maps_reproduce_the_plain_pose_gradient(orc):
    """Metallic 0 and the normal map (0.5, 0.5, 1) are the plain material:
    the same gradient up to rounding."""
    sc = _posed(_principled_plane(), np.array([0.01, 0.0, -0.02, 0.005, 0.0, 0.01]), np.eye(3), np.zeros(3))
    W = np.random.default_rng(4).uniform(0.5, 1.5, (sc.Hc, sc.Wc, 3))
    tw = pose.twists(np.zeros(6))
    plain = orc.pose_backward(sc, W, tw, 16, 16, spp=16, seed=3)
    flat = orc.pose_backward(sc, W, tw, 16, 16, spp=16, seed=3, metallic=np.zeros((8, 8)),
                             normal=np.tile([0.5, 0.5, 1.0], (8, 8, 1)))
    np.testing.assert_allclose(flat, plain, rtol=1e-9, atol=1e-12 * np.abs(plain).max())


def test_principled_pose_gradient_matches_common_random_number_differences(orc):
    """With a metallic map and a tilted normal map the first vertex's BRDF
    and its turn with the camera change; the gradient still equals the
    central differences of the oracle's renders at the same keys (the
    posed plane has no silhouette in view, so the differences are smooth)."""
    base = _principled_plane()
    m = np.full((8, 8), 0.6)
    nm = np.tile([0.62, 0.42, 0.9], (8, 8, 1))
    W = np.random.default_rng(5).uniform(0.5, 1.5, (base.Hc, base.Wc, 3))
    R0, t0 = pose.rotation([0.02, -0.03, 0.1]), np.array([0.01, 0.02, 0.05])
    xi, h, spp, nseed = np.zeros(6), 2e-3, 4096, 4
    tw = pose.twists(xi, R0, t0)
    fd, est = [], []
    for seed in range(nseed):
        row = []
        for k in range(6):
            e = np.zeros(6)
            e[k] = h
            Ep, _ = orc.render(_posed(base, xi + e, R0, t0), spp=spp, seed=seed, metallic=m, normal=nm)
            Em, _ = orc.render(_posed(base, xi - e, R0, t0), spp=spp, seed=seed, metallic=m, normal=nm)
            row.append(np.sum(W * (Ep - Em)) / (2.0 * h))
        fd.append(row)
        est.append(orc.pose_backward(_posed(base, xi, R0, t0), W, tw, 64, 0, spp=256, seed=seed, metallic=m,
                                     normal=nm).sum(0))
    fd, est = np.array(fd), np.array(est)
    se = (fd.std(0, ddof=1) + est.std(0, ddof=1)) / math.sqrt(nseed)
    scale = np.abs(fd.mean(0)).max()
    assert scale > 1.0
    assert np.all(np.abs(est.mean(0) - fd.mean(0)) <= 5.0 * se + 2e-3 * scale), (est.mean(0), fd.mean(0), se)
