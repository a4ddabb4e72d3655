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
