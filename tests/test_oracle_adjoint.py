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
    for B in (2, 3):
        s2 = sc.replace(bounces=B)
        adj, fd = np.zeros(n), np.zeros(n)
        for k in range(n):
            seed = 5000 + k
            adj[k] = orc.render_backward(s2, W, seed=seed)["drough"].sum()  # d/d(uniform roughness)
            lp = float((W * orc.render(s2, rough=s2.rough + h, seed=seed)[1]).sum())
            lm = float((W * orc.render(s2, rough=s2.rough - h, seed=seed)[1]).sum())
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
