"""Pins for the oracle's adjoint (path-replay gradient with detached sampling).

The loss is the linear functional L = sum(W * Ic) with random weights W, so
dL/dIc = W.  Parameters that do not move sampled paths (projector image,
albedo, PRF/CRF/white-balance scalars, and roughness when only direct light
is traced) give a per-seed deterministic forward, so central finite
differences of the FP64 forward must match the adjoint closely.
"""
import numpy as np
import pytest

from paper_2503_12174_gb300 import scenes


def _scene(res=12, spp=3, bounces=3, clip=0.0):
    sc = scenes.corner(res=res, tex=16, spp=spp, bounces=bounces, seed=5)
    p = sc.params
    return sc.replace(params=scenes.Params(gamma_p=p.gamma_p, gain_p=1.3, gamma_c=p.gamma_c, gain_c=p.gain_c,
                                           wb=p.wb, k_proj=p.k_proj, ks=p.ks, f0=p.f0, clip=clip))


def _loss(orc, sc, W, **kw):
    _, Ic = orc.render(sc, **kw)
    return float((W * Ic).sum())


def _fd(orc, sc, W, name, idx, h, **kw):
    base = {"Ip": sc.Ip, "albedo": sc.albedo, "rough": sc.rough}[name].astype(np.float64)
    p = base.copy(); p.flat[idx] += h
    m = base.copy(); m.flat[idx] -= h
    return (_loss(orc, sc, W, **{name: p}, **kw) - _loss(orc, sc, W, **{name: m}, **kw)) / (2 * h)


@pytest.mark.parametrize("clip", [0.0, 0.02])
def test_adjoint_textures_and_projector_fd(orc, clip):
    sc = _scene(clip=clip)
    rng = np.random.default_rng(0)
    W = rng.normal(size=(sc.Hc, sc.Wc, 3))
    g = orc.render_backward(sc, W)
    # pick elements with non-negligible gradient plus a few random ones
    for name, key in (("Ip", "dIp"), ("albedo", "dalbedo")):
        G = g[key].ravel()
        idx = list(np.argsort(-np.abs(G))[:6]) + list(rng.integers(0, G.size, 4))
        scale = np.abs(G).max()
        assert scale > 0
        for i in idx:
            fd = _fd(orc, sc, W, name, i, 1e-6)
            assert abs(fd - G[i]) <= 1e-6 * scale + 1e-5 * abs(G[i]), (name, i, fd, G[i])


def test_adjoint_roughness_fd_direct_only(orc):
    sc = _scene(bounces=1)
    rng = np.random.default_rng(1)
    W = rng.normal(size=(sc.Hc, sc.Wc, 3))
    g = orc.render_backward(sc, W)
    G = g["drough"].ravel()
    scale = np.abs(G).max()
    assert scale > 0
    for i in list(np.argsort(-np.abs(G))[:6]) + list(rng.integers(0, G.size, 4)):
        fd = _fd(orc, sc, W, "rough", i, 1e-6)
        assert abs(fd - G[i]) <= 1e-6 * scale + 1e-5 * abs(G[i]), (i, fd, G[i])


def _with(p, **kw):
    d = {f: getattr(p, f) for f in p.__dataclass_fields__}
    d.update(kw)
    return scenes.Params(**d)


def test_adjoint_response_parameters_fd(orc):
    sc = _scene()
    rng = np.random.default_rng(2)
    W = rng.normal(size=(sc.Hc, sc.Wc, 3))
    g = orc.render_backward(sc, W)["dparams"]
    p = sc.params
    h = 1e-6
    checks = []
    for j in range(3):
        checks.append((j, "gamma_p", j))
        checks.append((4 + j, "gamma_c", j))
        checks.append((8 + j, "wb", j))
    checks += [(3, "gain_p", None), (7, "gain_c", None)]
    for slot, field, j in checks:
        def at(delta):
            if j is None:
                return _with(p, **{field: getattr(p, field) + delta})
            v = list(getattr(p, field)); v[j] += delta
            return _with(p, **{field: tuple(v)})
        fd = (_loss(orc, sc, W, params=at(h)) - _loss(orc, sc, W, params=at(-h))) / (2 * h)
        assert abs(fd - g[slot]) <= 1e-6 * max(1.0, abs(g[slot])), (field, j, fd, g[slot])


def test_adjoint_pixel_list_consistency(orc):
    sc = _scene(res=10, spp=2)
    rng = np.random.default_rng(3)
    W = rng.normal(size=(sc.Hc, sc.Wc, 3))
    px = np.array([3, 17, 42, 99, 64])
    Wl = np.zeros_like(W).reshape(-1, 3)
    Wl[px] = W.reshape(-1, 3)[px]
    full = orc.render_backward(sc, Wl.reshape(W.shape))
    part = orc.render_backward(sc, W.reshape(-1, 3)[px], pixels=px)
    for k in full:
        np.testing.assert_allclose(part[k], full[k], rtol=1e-12, atol=1e-18)


@pytest.mark.slow
def test_adjoint_roughness_unbiased_multi_bounce(orc):
    """With two and three bounces, GGX-sampled directions move with roughness,
    so the detached-sampling gradient equals the finite difference only in
    expectation.  Averaged over seeds, for a loss linear in Ec (linear CRF),
    both must agree within their combined standard error.  The dropped
    continuation term would shift the adjoint by about 10x the tolerance."""
    sc = _scene(res=8, spp=4, bounces=3)
    sc = sc.replace(rough=np.full_like(sc.rough, 0.3), albedo=np.full_like(sc.albedo, 0.6),
                    params=_with(sc.params, gamma_c=(1.0, 1.0, 1.0)))
    W = np.ones((sc.Hc, sc.Wc, 3))  # total image brightness
    h, n = 0.05, 1200
    nt = 2  # 64 pixels per call: more threads cost more to start than they save
    for B in (2, 3):
        s2 = sc.replace(bounces=B)
        adj, fd = np.zeros(n), np.zeros(n)
        for k in range(n):
            seed = 5000 + k
            adj[k] = orc.render_backward(s2, W, seed=seed, nthreads=nt)["drough"].sum()  # d/d(uniform roughness)
            lp = float((W * orc.render(s2, rough=s2.rough + h, seed=seed, nthreads=nt)[1]).sum())
            lm = float((W * orc.render(s2, rough=s2.rough - h, seed=seed, nthreads=nt)[1]).sum())
            adj[k], fd[k] = adj[k], (lp - lm) / (2 * h)
        se = np.sqrt(adj.var() / n + fd.var() / n)
        assert abs(adj.mean()) > 10 * se  # the gradient is resolved, not noise
        assert abs(adj.mean() - fd.mean()) < 4 * se, (B, adj.mean(), fd.mean(), se)


def test_unit_tap_diagnostic_counts_each_contribution_once_per_tap(orc):
    """The unit-tap diagnostic (used to bound how far FP32 rounding of a hit
    point's texel position can move a texel's gradient): with dLoss/dIc >= 0
    every projector and albedo contribution is nonnegative; each reaches its
    four bilinear taps with weight 1 instead of weights that sum to 1, so the
    totals are exactly four times the adjoint's, and no texel gets less than
    its share under the real weights."""
    import numpy as np

    from paper_2503_12174_gb300 import scenes

    sc = scenes.corner(res=20, tex=16, spp=3, bounces=3, seed=5)
    p = sc.params
    sc = sc.replace(params=scenes.Params(gamma_p=(1.0, 1.0, 1.0), gain_p=1.0, gamma_c=p.gamma_c, gain_c=p.gain_c,
                                         wb=p.wb, k_proj=p.k_proj, ks=p.ks, f0=p.f0))
    W = np.random.default_rng(8).uniform(0.1, 1.0, size=(sc.Hc, sc.Wc, 3))
    g = orc.render_backward(sc, W)
    u = orc.render_backward(sc, W, unit_taps=True)
    for k in ("dIp", "dalbedo"):
        assert g[k].min() >= 0.0 and g[k].sum() > 0
        np.testing.assert_allclose(u[k].sum(), 4.0 * g[k].sum(), rtol=1e-12)
        assert np.all(u[k] >= g[k] * (1 - 1e-12))
    # the diagnostic is off again for the next call
    g2 = orc.render_backward(sc, W)
    np.testing.assert_allclose(g2["dIp"], g["dIp"], rtol=1e-12)


def test_adjoint_projector_and_gains_euler_identities(orc):
    """Homogeneity, checked without finite differences.  With no clipping,
    channel j of Ic is homogeneous of degree gamma_p,j * gamma_c,j in channel
    j of the projector image (Ep = Gp Ip^gamma_p per texel, Eq. 1; the paths
    do not depend on Ip; Ic = (Gc w Ec)^gamma_c, Eq. 5), and of degree
    gamma_c,j in Gp, in Gc and in w_j.  Euler's theorem then fixes, per seed
    and exactly up to rounding, sum_k Ip_kj dL/dIp_kj = gamma_p,j gamma_c,j L_j
    and Gp dL/dGp = Gc dL/dGc = sum_j gamma_c,j L_j, w_j dL/dw_j =
    gamma_c,j L_j, for L = sum W Ic and L_j its channel-j part.  A wrong
    exponent or a dropped factor in the PRF or CRF adjoint breaks one of them."""
    sc = _scene(bounces=3)
    p = sc.params
    W = np.random.default_rng(11).normal(size=(sc.Hc, sc.Wc, 3))
    _, Ic = orc.render(sc)
    Lj = (W * Ic).sum(axis=(0, 1))
    g = orc.render_backward(sc, W)
    gp, gc = np.asarray(p.gamma_p, np.float64), np.asarray(p.gamma_c, np.float64)
    Ip = sc.Ip.astype(np.float64)
    lhs = (Ip * g["dIp"]).sum(axis=(0, 1))
    np.testing.assert_allclose(lhs, gp * gc * Lj, rtol=1e-10)
    dP = g["dparams"]
    total = float((gc * Lj).sum())
    assert abs(total) > 1e-3 * np.abs(Lj).sum()
    np.testing.assert_allclose(p.gain_p * dP[3], total, rtol=1e-10)
    np.testing.assert_allclose(p.gain_c * dP[7], total, rtol=1e-10)
    np.testing.assert_allclose(np.asarray(p.wb) * dP[8:11], gc * Lj, rtol=1e-10)


def test_adjoint_albedo_euler_identity(orc):
    """With the Lambert lobe alone (ks = 0) each path's throughput is the
    product of the albedos at its vertices (the cosine-sampling weight is
    rho), so the contribution of vertex b is homogeneous of degree b in the
    albedo texels of its channel.  Renders with 1..B vertices share their
    first vertices (per-vertex Philox counters), so E_b, vertex b's part of
    Ec, is the difference of two renders.  Euler's theorem then gives, per
    seed and exactly up to rounding,
        sum_k rho_kj dL/drho_kj = sum_pixels W_j g'(Ec_j) sum_b b E_b,j
    with g' = gamma_c Ic / Ec the derivative of Eq. 5.  Dropping the
    continuation term of the albedo adjoint turns b into 1 and fails it."""
    sc = _scene(bounces=3)
    sc = sc.replace(params=_with(sc.params, ks=0.0))
    W = np.random.default_rng(12).normal(size=(sc.Hc, sc.Wc, 3))
    E = [np.zeros((sc.Hc, sc.Wc, 3))] + [orc.render(sc, bounces=b)[0] for b in (1, 2, 3)]
    Ec, Ic = orc.render(sc)
    np.testing.assert_array_equal(Ec, E[3])
    weighted = sum(b * (E[b] - E[b - 1]) for b in (1, 2, 3))
    gc = np.asarray(sc.params.gamma_c, np.float64)
    gprime = np.where(Ec > 0, gc * Ic / np.where(Ec > 0, Ec, 1.0), 0.0)
    expect = (W * gprime * weighted).sum(axis=(0, 1))
    g = orc.render_backward(sc, W)
    lhs = (sc.albedo.astype(np.float64) * g["dalbedo"]).sum(axis=(0, 1))
    assert np.all(np.abs(expect) > 0)
    np.testing.assert_allclose(lhs, expect, rtol=1e-10)
    # the identity separates the vertices: the undifferentiated sum is far off
    plain = (W * gprime * E[3]).sum(axis=(0, 1))
    assert np.all(np.abs(plain - expect) > 1e-3 * np.abs(expect))
