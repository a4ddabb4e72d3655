"""Pins of the oracle's principled material (Sec. 3.2's m with a metallic
map, and the normal map Vn) against closed forms, special cases that reduce
to the already pinned Lambert + GGX renderer, exact invariants, and central
finite differences of the FP64 forward.

* metallic 0 and a flat normal map reproduce the plain renderer;
* at normal incidence the GGX lobe has the closed form ks F0 / (4 pi a^2)
  with F0 = (1 - m) f0 + m rho, and a full metal has no diffuse part;
* direct light on a plane through a constant tilted normal map is
  (rho / pi) k Gp c^gamma cos(theta_p) max(ns . wp, 0) / r^2 with ns the
  tilted normal in the plane's tangent frame;
* one bounce is affine in the metallic map, and a metal of albedo f0 is the
  specular lobe alone;
* the adjoint's metallic, albedo, roughness and normal-map gradients match
  central differences wherever those parameters do not move sampled paths;
* the sampler's mean weight f cos / pdf equals the quadrature of f cos
  with metallic on, and stays <= 1;
* without the specular lobe, the albedo and metallic adjoints satisfy the
  homogeneity identities of Euler's theorem exactly, per seed.
"""
import math

import numpy as np
import pytest

from paper_2503_12174_gb300 import scenes


def _unit(rng, n=1):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _upper(rng, n_, k):
    """k random unit directions in the hemisphere of n_."""
    out = []
    while len(out) < k:
        w = _unit(rng)[0]
        if w @ n_ > 0.05:
            out.append(w)
    return out


def test_metallic_zero_is_the_plain_brdf(orc):
    rng = np.random.default_rng(0)
    for _ in range(200):
        n = _unit(rng)[0]
        wo, wi = _upper(rng, n, 2)
        rho = rng.uniform(0.1, 0.9, 3)
        r = rng.uniform(0.05, 1.0)
        f, dfdr = orc.bsdf_eval(n, wo, wi, rho, r, 1.0, 0.04)
        p = orc.pbr_eval(n, wo, wi, rho, r, 0.0, 1.0, 0.04)
        np.testing.assert_allclose(p["f"], f, rtol=1e-13)
        np.testing.assert_allclose(p["dr"], dfdr, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(p["drho"], 1.0 / math.pi, rtol=1e-15)


def test_principled_reciprocity(orc):
    rng = np.random.default_rng(1)
    for _ in range(200):
        n = _unit(rng)[0]
        wo, wi = _upper(rng, n, 2)
        rho = rng.uniform(0.1, 0.9, 3)
        r, m = rng.uniform(0.05, 1.0), rng.uniform(0.0, 1.0)
        a = orc.pbr_eval(n, wo, wi, rho, r, m, 1.0, 0.04)["f"]
        b = orc.pbr_eval(n, wi, wo, rho, r, m, 1.0, 0.04)["f"]
        np.testing.assert_allclose(a, b, rtol=1e-12)


@pytest.mark.parametrize("m", [0.0, 0.3, 1.0])
def test_normal_incidence_closed_form(orc, m):
    """wo = wi = n: h = n, so D = 1 / (pi a^2), G1 = 1, Schlick F = F0."""
    n = np.array([0.2, -0.3, 0.9])
    n /= np.linalg.norm(n)
    rho = np.array([0.7, 0.4, 0.15])
    r, ks, f0 = 0.6, 0.8, 0.04
    a = r * r
    F0 = (1.0 - m) * f0 + m * rho
    expect = (1.0 - m) * rho / math.pi + ks * F0 / (4.0 * math.pi * a * a)
    got = orc.pbr_eval(n, n, n, rho, r, m, ks, f0)["f"]
    np.testing.assert_allclose(got, expect, rtol=1e-13)
    if m == 1.0:  # a full metal has no diffuse lobe
        np.testing.assert_array_equal(orc.pbr_eval(n, n, n, rho, r, 1.0, 0.0, f0)["f"], 0.0)


def test_principled_partial_derivatives_fd(orc):
    rng = np.random.default_rng(2)
    h = 1e-6
    for _ in range(40):
        n = _unit(rng)[0]
        wo, wi = _upper(rng, n, 2)
        rho = rng.uniform(0.1, 0.9, 3)
        r, m = rng.uniform(0.1, 0.9), rng.uniform(0.05, 0.95)
        p = orc.pbr_eval(n, wo, wi, rho, r, m, 1.0, 0.04)

        def f(**kw):
            args = dict(n=n, wo=wo, wi=wi, rho=rho, r=r, m=m, ks=1.0, f0=0.04)
            args.update(kw)
            return orc.pbr_eval(**args)["f"]

        scale = np.abs(p["f"]).max()
        fd = (f(r=r + h) - f(r=r - h)) / (2 * h)
        np.testing.assert_allclose(p["dr"], fd, atol=1e-6 * scale, rtol=1e-6)
        fd = (f(m=m + h) - f(m=m - h)) / (2 * h)
        np.testing.assert_allclose(p["dm"], fd, atol=1e-6 * scale, rtol=1e-6)
        for j in range(3):
            e = np.zeros(3); e[j] = h
            fd = (f(rho=rho + e) - f(rho=rho - e)) / (2 * h)
            assert abs(fd[j] - p["drho"][j]) <= 1e-6 * scale, (j, fd, p["drho"])
            fd = (f(n=n + e) - f(n=n - e)) / (2 * h)  # n enters only through dot products
            np.testing.assert_allclose(p["dn"][:, j], fd, atol=1e-6 * scale, rtol=1e-6)


def _flat_maps(sc):
    normal = np.zeros((sc.Ht, sc.Wt, 3), np.float32)
    normal[..., :2] = 0.5
    normal[..., 2] = 1.0
    return np.zeros((sc.Ht, sc.Wt), np.float32), normal


def test_flat_maps_reproduce_the_plain_renderer(orc):
    sc = scenes.corner(res=12, tex=16, spp=3, bounces=3, seed=4)
    m, nm = _flat_maps(sc)
    Ec0, Ic0 = orc.render(sc)
    Ec1, Ic1 = orc.render(sc, metallic=m, normal=nm)
    np.testing.assert_allclose(Ec1, Ec0, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(Ic1, Ic0, rtol=1e-12, atol=1e-15)
    W = np.random.default_rng(3).normal(size=Ic0.shape)
    g0 = orc.render_backward(sc, W)
    g1 = orc.render_backward(sc, W, metallic=m, normal=nm)
    for k in ("dIp", "dalbedo", "drough", "dparams"):
        np.testing.assert_allclose(g1[k], g0[k], rtol=1e-10, atol=1e-12 * np.abs(g0[k]).max(), err_msg=k)
    assert g1["dmetallic"].shape == m.shape and g1["dnormal"].shape == nm.shape


@pytest.mark.parametrize("theta,phi", [(0.4, 0.0), (0.3, 2.0), (0.6, -1.2)])
def test_tilted_normal_map_direct_light_closed_form(orc, theta, phi):
    """The plane z = 1 with u along +x: tangent T = +x, normal N = -z towards
    the camera, B = N x T = -y.  A constant normal map tilts the shading
    normal to ns = v_x T + v_y B + v_z N (v decoded and normalised)."""
    c, gamma, k, gain, rho = 0.6, 2.2, 1.5, 1.2, 0.55
    sc = scenes.plane(res=40)
    v = np.array([math.sin(theta) * math.cos(phi), math.sin(theta) * math.sin(phi), math.cos(theta)])
    enc = ((v + 1.0) * 0.5).astype(np.float32)
    sc = sc.replace(Ip=np.full((40, 40, 3), c, np.float32), albedo=np.full((8, 8, 3), rho, np.float32),
                    params=scenes.Params(gamma_p=(gamma,) * 3, gain_p=gain, k_proj=k, ks=0.0, jitter=0),
                    normal=np.broadcast_to(enc, (8, 8, 3)).copy())
    Ec, _ = orc.render(sc)
    vd = 2.0 * enc.astype(np.float64) - 1.0
    vd /= np.linalg.norm(vd)
    T, N = np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.0, -1.0])
    B = np.cross(N, T)
    ns = vd[0] * T + vd[1] * B + vd[2] * N
    Kinv = np.linalg.inv(np.asarray(sc.Kc, np.float64))
    ys, xs = np.mgrid[0:sc.Hc, 0:sc.Wc]
    d = np.stack([xs + 0.5, ys + 0.5, np.ones_like(xs, dtype=np.float64)], -1) @ Kinv.T
    x = d / d[..., 2:3]
    cp = -np.asarray(sc.tp, np.float64)
    wv = cp - x
    r = np.linalg.norm(wv, axis=-1)
    wp = wv / r[..., None]
    cos_s = np.maximum(wp @ ns, 0.0)
    cos_p = (x - cp)[..., 2] / r
    q = (x - cp) @ np.asarray(sc.Kp, np.float64).T
    u, vv = q[..., 0] / q[..., 2], q[..., 1] / q[..., 2]
    inside = (u >= 0) & (u < sc.Wp) & (vv >= 0) & (vv < sc.Hp)
    cf, rf = float(np.float32(c)), float(np.float32(rho))
    expect = np.where(inside, rf / math.pi * k * gain * cf ** gamma * cos_p * cos_s / r ** 2, 0.0)
    assert (expect > 0).sum() > 0.4 * expect.size
    np.testing.assert_allclose(Ec[..., 0], expect, rtol=1e-12, atol=1e-15)


def test_one_bounce_is_affine_in_metallic_and_a_metal_of_albedo_f0_is_the_specular_lobe(orc):
    sc = scenes.corner(res=14, tex=16, spp=2, bounces=1, seed=8)
    ones = np.ones((sc.Ht, sc.Wt), np.float32)
    E0, _ = orc.render(sc, metallic=0.0 * ones)
    E1, _ = orc.render(sc, metallic=ones)
    Eh, _ = orc.render(sc, metallic=0.5 * ones)
    np.testing.assert_allclose(Eh, 0.5 * (E0 + E1), rtol=1e-12, atol=1e-15)
    assert np.abs(E1 - E0).max() > 1e-3 * np.abs(E0).max()
    f0 = sc.params.f0
    alb = np.full(sc.albedo.shape, f0, np.float32)
    Emetal, _ = orc.render(sc, metallic=ones, albedo=alb)
    Espec, _ = orc.render(sc, albedo=np.zeros_like(alb))
    np.testing.assert_allclose(Emetal, Espec, rtol=1e-6, atol=1e-12)  # f0 enters as float32 through the albedo


def _principled_scene(bounces, spp=3, res=12):
    sc = scenes.with_principled(scenes.corner(res=res, tex=16, spp=spp, bounces=bounces, seed=5))
    p = sc.params
    return sc.replace(params=scenes.Params(gamma_p=p.gamma_p, gain_p=1.3, gamma_c=p.gamma_c, gain_c=p.gain_c,
                                           wb=p.wb, k_proj=p.k_proj, ks=p.ks, f0=p.f0))


def _fd(orc, sc, W, name, idx, h):
    base = {"albedo": sc.albedo, "rough": sc.rough, "metallic": sc.metallic, "normal": sc.normal}[name]
    base = base.astype(np.float64)
    out = []
    for s in (h, -h):
        x = base.copy()
        x.flat[idx] += s
        out.append(float((W * orc.render(sc, **{name: x})[1]).sum()))
    return (out[0] - out[1]) / (2 * h)


def _check(orc, sc, W, g, name, key, rng):
    G = g[key].ravel()
    scale = np.abs(G).max()
    assert scale > 0, key
    for i in list(np.argsort(-np.abs(G))[:6]) + list(rng.integers(0, G.size, 4)):
        fd = _fd(orc, sc, W, name, i, 1e-6)
        assert abs(fd - G[i]) <= 1e-6 * scale + 1e-5 * abs(G[i]), (key, i, fd, G[i])


def test_adjoint_metallic_and_albedo_fd_multi_bounce(orc):
    """Metallic and albedo move no sampled direction: per-seed FD holds at 3 bounces."""
    sc = _principled_scene(bounces=3)
    rng = np.random.default_rng(6)
    W = rng.normal(size=(sc.Hc, sc.Wc, 3))
    g = orc.render_backward(sc, W)
    _check(orc, sc, W, g, "metallic", "dmetallic", rng)
    _check(orc, sc, W, g, "albedo", "dalbedo", rng)


def test_adjoint_normal_map_and_roughness_fd_direct_only(orc):
    """The normal map and roughness move sampled directions; with direct light
    only (one vertex, no sampling) per-seed FD holds."""
    sc = _principled_scene(bounces=1)
    rng = np.random.default_rng(7)
    W = rng.normal(size=(sc.Hc, sc.Wc, 3))
    g = orc.render_backward(sc, W)
    _check(orc, sc, W, g, "normal", "dnormal", rng)
    _check(orc, sc, W, g, "rough", "drough", rng)
    _check(orc, sc, W, g, "metallic", "dmetallic", rng)


@pytest.mark.parametrize("m", [0.5, 1.0])
def test_principled_mean_weight_is_directional_albedo(orc, m):
    """E[f cos / pdf] over the sampler's directions equals the quadrature of
    f cos over the hemisphere (the sampler and pdf are the plain BRDF's; f
    carries the metallic Fresnel), and a metal of albedo <= 0.9 reflects no
    more than it receives."""
    rng = np.random.default_rng(8)
    n = np.array([0.0, 0.0, 1.0])
    wo = np.array([0.4, -0.2, 0.85])
    wo /= np.linalg.norm(wo)
    rho, r = np.array([0.9, 0.6, 0.3]), 0.45
    nt, nph = 300, 600
    th = (np.arange(nt) + 0.5) * np.pi / nt
    ph = (np.arange(nph) + 0.5) * 2 * np.pi / nph
    T, P = np.meshgrid(th, ph, indexing="ij")
    d = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)
    w = (np.sin(T) * (np.pi / nt) * (2 * np.pi / nph)).ravel()
    fq = np.array([orc.pbr_eval(n, wo, di, rho, r, m, 1.0, 0.04)["f"] for di in d])
    albedo = (fq * np.maximum(d[:, 2], 0)[:, None] * w[:, None]).sum(0)
    N = 20000
    u = rng.random((N, 3))
    acc = np.zeros((N, 3))
    for i in range(N):
        ok, wi = orc.bsdf_sample(n, wo, r, 1.0, *u[i])
        if ok:
            acc[i] = orc.pbr_eval(n, wo, wi, rho, r, m, 1.0, 0.04)["f"] * wi[2] / orc.bsdf_pdf(n, wo, wi, r, 1.0)
    se = acc.std(0) / np.sqrt(N)
    assert np.all(np.abs(acc.mean(0) - albedo) < 4 * se + 1e-3), (acc.mean(0), albedo)
    assert np.all(albedo <= 1.0)


def test_adjoint_albedo_and_metallic_homogeneity_without_the_specular_lobe(orc):
    """With ks = 0 the principled BRDF is (1 - m) rho / pi at the shading
    normal and each vertex's sampling weight is (1 - m) rho, so vertex b's
    contribution is homogeneous of degree b in the albedo texels of its
    channel and in the texels of 1 - m (bilinear weights sum to 1).  Renders
    with 1..B vertices share their first vertices, so E_b, vertex b's part of
    Ec, is a difference of renders, and Euler's theorem gives per seed, with
    the normal map on and exactly up to rounding,
        sum rho dL/drho = -sum (1 - m) dL/dm = sum W g'(Ec) sum_b b E_b
    (per channel for the albedo, over the channels for m; g' = gamma_c Ic / Ec)."""
    import dataclasses

    sc = _principled_scene(bounces=3)
    sc = sc.replace(params=dataclasses.replace(sc.params, ks=0.0))
    assert sc.metallic.max() > 0.2 and np.abs(sc.normal - [0.5, 0.5, 1.0]).max() > 0.05
    W = np.random.default_rng(13).normal(size=(sc.Hc, sc.Wc, 3))
    E = [np.zeros((sc.Hc, sc.Wc, 3))] + [orc.render(sc, bounces=b)[0] for b in (1, 2, 3)]
    Ec, Ic = orc.render(sc)
    np.testing.assert_array_equal(Ec, E[3])
    gc = np.asarray(sc.params.gamma_c, np.float64)
    gprime = np.where(Ec > 0, gc * Ic / np.where(Ec > 0, Ec, 1.0), 0.0)
    expect = (W * gprime * sum(b * (E[b] - E[b - 1]) for b in (1, 2, 3))).sum(axis=(0, 1))
    g = orc.render_backward(sc, W)
    rho_side = (sc.albedo.astype(np.float64) * g["dalbedo"]).sum(axis=(0, 1))
    np.testing.assert_allclose(rho_side, expect, rtol=1e-10)
    m_side = -((1.0 - sc.metallic.astype(np.float64)) * g["dmetallic"]).sum()
    np.testing.assert_allclose(m_side, expect.sum(), rtol=1e-10)
