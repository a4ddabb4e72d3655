"""Pins for the oracle's forward estimator against closed forms and invariants.

* direct light on a Lambertian plane from a uniform pinhole projector:
  Ec = (rho/pi) k Gp c^gamma_p cos(theta_p) cos(theta_s) / r^2 (Eqs. 1-3, 6);
* integrating sphere: inside a closed sphere with Lambertian albedo a, every
  point receives the same indirect irradiance Phi / A * sum_n a^n, Phi the
  projector's power (form factor of a sphere);
* white furnace: the same sphere with albedo 1 and no specular lobe absorbs
  nothing, so every further path vertex adds the same Phi / (pi A);
* linearity in Ep before the CRF; monotonicity in the bounce count;
  dark projector, empty scene, projector behind the surface.
"""
import math

import numpy as np
import pytest

from paper_2503_12174_gb300 import scenes


def _pixel_centre_dirs(sc):
    Kinv = np.linalg.inv(np.asarray(sc.Kc, np.float64))
    ys, xs = np.mgrid[0:sc.Hc, 0:sc.Wc]
    p = np.stack([xs + 0.5, ys + 0.5, np.ones_like(xs, dtype=np.float64)], -1)
    return p @ Kinv.T


@pytest.mark.parametrize("c,gamma,k,gain,rho", [(0.7, 2.2, 1.0, 1.0, 0.5), (0.35, 2.6, 3.0, 1.7, 0.8)])
def test_direct_light_closed_form(orc, c, gamma, k, gain, rho):
    sc = scenes.plane(res=48)
    sc = sc.replace(Ip=np.full((48, 48, 3), c, np.float32), albedo=np.full((8, 8, 3), rho, np.float32),
                    params=scenes.Params(gamma_p=(gamma,) * 3, gain_p=gain, k_proj=k, jitter=0))
    Ec, _ = orc.render(sc)
    c, rho = float(np.float32(c)), float(np.float32(rho))   # the inputs are float32 arrays
    d = _pixel_centre_dirs(sc)
    x = d / d[..., 2:3]                       # hit point on z = 1
    cp = -np.asarray(sc.tp, np.float64)       # projector centre -Rp^T tp with Rp = I
    v = cp - x
    r = np.linalg.norm(v, axis=-1)
    cos_s = (v @ np.array([0.0, 0.0, -1.0])) / r   # normal faces the camera
    cos_p = (x - cp)[..., 2] / r                   # projector looks along +z
    Kp = np.asarray(sc.Kp, np.float64)
    q = (x - cp) @ Kp.T
    u, vv = q[..., 0] / q[..., 2], q[..., 1] / q[..., 2]
    inside = (u >= 0) & (u < sc.Wp) & (vv >= 0) & (vv < sc.Hp)
    expect = rho / math.pi * k * gain * c ** gamma * cos_p * cos_s / r ** 2
    expect = np.where(inside, expect, 0.0)
    assert inside.sum() > 0.5 * inside.size and (~inside).sum() > 0
    np.testing.assert_allclose(Ec[..., 0], expect, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(Ec[..., 1], expect, rtol=1e-12, atol=1e-15)


def _projector_power(sc, k, Ep, n=8):
    """Phi = k Ep * integral over the image of cos(theta_p) d omega, with
    d omega = du dv / (f^2 rho^3) and cos = 1 / rho (rho = |(u-cx)/f, (v-cy)/f, 1|)."""
    f = float(sc.Kp[0, 0])
    cx, cy = float(sc.Kp[0, 2]), float(sc.Kp[1, 2])
    s = (np.arange(sc.Wp * n) + 0.5) / n
    t = (np.arange(sc.Hp * n) + 0.5) / n
    U, V = np.meshgrid(s, t, indexing="xy")
    rho = np.sqrt(((U - cx) / f) ** 2 + ((V - cy) / f) ** 2 + 1.0)
    return k * Ep * np.sum(1.0 / (f * f * rho ** 4)) / (n * n)


@pytest.mark.slow
def test_integrating_sphere(orc):
    a, c = 0.6, 0.8
    sc = scenes.sphere(subdiv=3, res=32, spp=96, bounces=3, albedo=a, ip_value=c)
    K = scenes.intrinsics(32, 32, 110.0)  # wide projector: a large lit patch keeps MC noise low
    sc = sc.replace(Kp=K)
    E3, _ = orc.render(sc)
    E1, _ = orc.render(sc.replace(bounces=1))
    ind = (E3 - E1)[..., 0].ravel()            # same seed: the indirect part of every pixel
    V = sc.verts.astype(np.float64)[sc.tris]
    A = 0.5 * np.linalg.norm(np.cross(V[:, 1] - V[:, 0], V[:, 2] - V[:, 0]), axis=1).sum()
    Phi = _projector_power(sc, 1.0, c)          # gamma_p = 1, Gp = k = 1
    expect = a / math.pi * Phi / A * (a + a * a)
    # pixels are independent estimates of the same value
    se = ind.std() / math.sqrt(ind.size)
    assert abs(ind.mean() - expect) < 4 * se + 0.015 * expect, (ind.mean(), expect, se)


@pytest.mark.slow
def test_white_furnace(orc):
    """Albedo 1, Lambert only: after the first bounce the light is spread
    uniformly over the sphere and nothing is absorbed, so vertex b >= 2 of
    every path adds Phi / (pi A) to the pixel's mean radiance.  Renders with
    B and B + 1 vertices share their first B vertices (the Philox counters
    are per vertex), so their difference is vertex B + 1's contribution alone."""
    sc = scenes.sphere(subdiv=3, res=32, spp=96, bounces=4, albedo=1.0, ip_value=0.8)
    sc = sc.replace(Kp=scenes.intrinsics(32, 32, 110.0))
    E = [orc.render(sc.replace(bounces=b))[0][..., 0].ravel() for b in (1, 2, 3, 4)]
    V = sc.verts.astype(np.float64)[sc.tris]
    A = 0.5 * np.linalg.norm(np.cross(V[:, 1] - V[:, 0], V[:, 2] - V[:, 0]), axis=1).sum()
    expect = _projector_power(sc, 1.0, 0.8) / (math.pi * A)
    for b in range(1, 4):
        inc = E[b] - E[b - 1]
        assert np.all(inc >= 0.0)
        se = inc.std() / math.sqrt(inc.size)
        assert abs(inc.mean() - expect) < 4 * se + 0.015 * expect, (b + 1, inc.mean(), expect, se)


def test_linear_in_projector_image(orc):
    sc = scenes.corner(res=24, spp=4, bounces=3)
    p = sc.params
    sc = sc.replace(params=scenes.Params(gamma_p=(1.0, 1.0, 1.0), gain_p=1.0, gamma_c=p.gamma_c, gain_c=p.gain_c,
                                         wb=p.wb, k_proj=p.k_proj, ks=p.ks, f0=p.f0))
    rng = np.random.default_rng(0)
    I1 = rng.random(sc.Ip.shape)
    I2 = rng.random(sc.Ip.shape)
    E1, _ = orc.render(sc, Ip=I1)
    E2, _ = orc.render(sc, Ip=I2)
    E12, _ = orc.render(sc, Ip=0.3 * I1 + 1.7 * I2)
    np.testing.assert_allclose(E12, 0.3 * E1 + 1.7 * E2, rtol=1e-12, atol=1e-15)


def test_monotone_in_bounces(orc):
    sc = scenes.corner(res=20, spp=4, bounces=1)
    prev = None
    for B in (1, 2, 3, 4):
        E, _ = orc.render(sc, bounces=B)
        if prev is not None:
            assert np.all(E >= prev - 1e-15)
        prev = E
    assert prev.sum() > 0


def test_degenerate_cases(orc):
    sc = scenes.corner(res=16, spp=2)
    E, I = orc.render(sc, Ip=np.zeros_like(sc.Ip))
    assert not E.any() and not I.any()
    empty = sc.replace(verts=np.zeros((0, 3), np.float32), tris=np.zeros((0, 3), np.int32),
                       uv=np.zeros((0, 2), np.float32))
    E, I = orc.render(empty)
    assert not E.any()
    # projector turned around (looking along -z): nothing is lit
    sc2 = scenes.plane(res=16).replace(Rp=np.diag([-1.0, 1.0, -1.0]).astype(np.float32),
                                         tp=np.array([0.3, 0, 0], np.float32))
    E, _ = orc.render(sc2)
    assert not E.any()
    E, _ = orc.render(sc, bounces=0)
    assert not E.any()


def test_pixel_list_matches_full_image(orc):
    sc = scenes.corner(res=20, spp=3)
    Ef, If = orc.render(sc)
    px = np.array([0, 7, 133, 399, 250])
    Ep, Ipx = orc.render(sc, pixels=px)
    np.testing.assert_array_equal(Ep, Ef.reshape(-1, 3)[px])
    np.testing.assert_array_equal(Ipx, If.reshape(-1, 3)[px])


def _with(p, **kw):
    d = {f: getattr(p, f) for f in p.__dataclass_fields__}
    d.update(kw)
    return scenes.Params(**d)


def test_russian_roulette_is_unbiased(orc):
    """Russian roulette from vertex 2 with survival q: survivors carry 1/q,
    so q = 1 is exactly the renderer without roulette, and q = 0.75 has the
    same expectation (image mean within 4 standard errors over 64 x 128
    paths, in a closed sphere where every path would continue)."""
    sc = scenes.sphere(subdiv=2, res=8, spp=128, bounces=5, seed=2)
    E0, _ = orc.render(sc)
    E1, _ = orc.render(sc.replace(params=_with(sc.params, rr_start=2, rr_q=1.0)))
    np.testing.assert_array_equal(E1, E0)
    Eq, _ = orc.render(sc.replace(params=_with(sc.params, rr_start=2, rr_q=0.75)))
    assert np.abs(Eq - E0).max() > 0  # roulette changed individual paths
    # per-pixel differences are independent across pixels: compare the image means
    d = (Eq - E0).mean(axis=-1).ravel()
    se = d.std(ddof=1) / np.sqrt(d.size)
    assert abs(d.mean()) < 4 * se + 1e-12, (d.mean(), se)


def test_radiance_clipping_bounds(orc):
    """Eq. 12 clamps each per-vertex contribution per channel: a clip above
    every contribution changes nothing, clipping never brightens a pixel, and
    a pixel's mean over samples is at most (vertices per path) x clip."""
    sc = scenes.corner(res=16, tex=16, spp=8, bounces=3, seed=6)
    E0, _ = orc.render(sc)
    Ebig, _ = orc.render(sc.replace(params=_with(sc.params, clip=1e6)))
    np.testing.assert_array_equal(Ebig, E0)
    for clip in (0.05, 0.005):
        Ec, _ = orc.render(sc.replace(params=_with(sc.params, clip=clip)))
        assert np.all(Ec <= E0 + 1e-15)
        assert np.all(Ec <= sc.bounces * clip * (1 + 1e-12))
        assert (Ec < E0 - 1e-9).any()  # the clip was active somewhere
