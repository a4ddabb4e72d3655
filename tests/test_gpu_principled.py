"""Principled material on the GPU (Sec. 3.2's metallic map and normal map
Vn): dpcs_render_principled against the oracle's render with the same maps,
the plain material as its special case, and dpcs_render_backward_principled
against the oracle's adjoint (metallic and normal-map gradients included)."""
import numpy as np
import pytest

from paper_2503_12174_gb300 import dpcs, scenes
from gpu_util import GpuScene, crf_atol, need_cuda, pixel_parity

pytestmark = pytest.mark.gpu


def _grad_close(g, r, rtol, scale_tol):
    g, r = np.asarray(g, np.float64).ravel(), np.asarray(r, np.float64).ravel()
    scale = np.abs(r).max()
    err = np.abs(g - r) - (rtol * np.abs(r) + scale_tol * scale)
    return bool(np.all(err <= 0)), float(np.max(np.abs(g - r) / (np.abs(r) + 1e-30))), scale


def _maps(g, sc):
    torch = need_cuda()
    dev = g.ctx.device
    m = None if sc.metallic is None else torch.from_numpy(np.ascontiguousarray(sc.metallic)).to(dev)
    n = None if sc.normal is None else torch.from_numpy(np.ascontiguousarray(sc.normal)).to(dev)
    return m, n


def _render(g, sc, m, n):
    torch = need_cuda()
    Ec = torch.empty((sc.Hc, sc.Wc, 3), dtype=torch.float32, device=g.ctx.device)
    Ic, _ = g.ctx.render_principled(g.handle, g.albedo, g.rough, m, n, g.Ip, g.view, g.params, sc.spp, sc.bounces,
                                    sc.seed, Ec=Ec)
    g.ctx.sync()
    return Ec, Ic


def _cases():
    yield "corner", scenes.with_principled(scenes.corner(res=32, tex=16, spp=4, bounces=3, seed=2))
    p = scenes.corner(res=29, tex=24, spp=5, bounces=2, seed=7)
    q = p.params
    yield "corner-ragged-clip", scenes.with_principled(p.replace(params=scenes.Params(
        gamma_p=q.gamma_p, gain_p=q.gain_p, gamma_c=q.gamma_c, gain_c=q.gain_c, wb=q.wb, k_proj=q.k_proj, ks=q.ks,
        f0=q.f0, clip=0.05)), seed=3)
    h = scenes.heightfield(spp=4, cam=48, proj=(40, 56), tex=32, n_vert=41)
    yield "heightfield-rr", scenes.with_principled(h, seed=4)
    yield "metal-only", scenes.with_principled(scenes.corner(res=24, tex=16, spp=4, bounces=3, seed=5),
                                               seed=6).replace(normal=None)
    yield "normal-only", scenes.with_principled(scenes.corner(res=24, tex=16, spp=4, bounces=3, seed=6),
                                                seed=7).replace(metallic=None)


@pytest.mark.parametrize("case", range(5))
def test_principled_render_matches_oracle(orc, case):
    need_cuda()
    name, sc = list(_cases())[case]
    g = GpuScene(sc)
    try:
        m, n = _maps(g, sc)
        Ec, Ic = _render(g, sc, m, n)
        Ec, Ic = Ec.cpu().numpy(), Ic.cpu().numpy()
    finally:
        g.close()
    rEc, rIc = orc.render(sc)
    assert rEc.max() > 0
    ok, info = pixel_parity(Ec, rEc)
    assert ok, (name, info)
    ok, info = pixel_parity(Ic, rIc, atol=crf_atol(sc, rEc))
    assert ok, (name, info)


def test_plain_maps_are_the_plain_material(orc):
    """No maps, and metallic 0 with the flat normal map (0.5, 0.5, 1): both
    render what dpcs_render renders (to FP32 rounding of the extra frame)."""
    torch = need_cuda()
    sc = scenes.corner(res=32, tex=16, spp=4, bounces=3, seed=8)
    g = GpuScene(sc)
    try:
        E0, _ = g.render()
        E1, _ = _render(g, sc, None, None)
        zeros = torch.zeros_like(g.rough)
        flat = torch.zeros((sc.Ht, sc.Wt, 3), dtype=torch.float32, device=g.ctx.device)
        flat[..., :2] = 0.5
        flat[..., 2] = 1.0
        E2, _ = _render(g, sc, zeros, flat)
        E0, E1, E2 = (x.cpu().numpy() for x in (E0, E1, E2))
    finally:
        g.close()
    for E in (E1, E2):
        ok, info = pixel_parity(E, E0, rtol=1e-5, atol=1e-8)
        assert ok, info


@pytest.mark.parametrize("case", [0, 1, 2, 3])
def test_principled_backward_matches_oracle(orc, case):
    torch = need_cuda()
    name, sc = list(_cases())[case]
    p = sc.params
    sc = sc.replace(params=scenes.Params(gamma_p=p.gamma_p, gain_p=1.2, gamma_c=p.gamma_c, gain_c=p.gain_c, wb=p.wb,
                                         k_proj=p.k_proj, ks=p.ks, f0=p.f0, clip=p.clip, rr_start=p.rr_start,
                                         rr_q=p.rr_q))
    rng = np.random.default_rng(case)
    W = rng.normal(size=(sc.Hc, sc.Wc, 3)).astype(np.float32)
    g = GpuScene(sc)
    try:
        m, n = _maps(g, sc)
        Ec, Ic = _render(g, sc, m, n)
        dev = g.ctx.device
        gr = {"dIp": torch.zeros_like(g.Ip), "dalbedo": torch.zeros_like(g.albedo),
              "drough": torch.zeros_like(g.rough), "dparams": torch.zeros(11, dtype=torch.float32, device=dev)}
        if m is not None:
            gr["dmetallic"] = torch.zeros_like(m)
        if n is not None:
            gr["dnormal"] = torch.zeros_like(n)
        g.ctx.render_backward_principled(g.handle, g.albedo, g.rough, m, n, g.Ip, g.view, g.params, sc.spp,
                                         sc.bounces, sc.seed, Ec, Ic, torch.from_numpy(W).to(dev), gr["dIp"],
                                         gr["dalbedo"], gr["drough"], gr.get("dmetallic"), gr.get("dnormal"),
                                         gr["dparams"])
        g.ctx.sync()
        gr = {k: v.cpu().numpy().astype(np.float64) for k, v in gr.items()}
    finally:
        g.close()
    ref = orc.render_backward(sc, W.astype(np.float64))
    for k in ("dIp", "dalbedo", "drough", "dmetallic", "dnormal"):
        if k not in gr:
            continue
        ok, mx, scale = _grad_close(gr[k], ref[k], 1e-3, 2e-5)
        assert scale > 0 and ok, (name, k, mx, scale)
    ok, mx, _ = _grad_close(gr["dparams"], ref["dparams"], 1e-3, 1e-6)
    assert ok, (name, "dparams", gr["dparams"], ref["dparams"])


def test_principled_backward_refuses_a_gradient_without_its_map():
    torch = need_cuda()
    sc = scenes.corner(res=16, tex=16, spp=2, bounces=2, seed=1)
    g = GpuScene(sc)
    try:
        Ec, Ic = _render(g, sc, None, None)
        dM = torch.zeros_like(g.rough)
        with pytest.raises(dpcs.DPCSError) as e:
            g.ctx.render_backward_principled(g.handle, g.albedo, g.rough, None, None, g.Ip, g.view, g.params, 2, 2,
                                             sc.seed, Ec, Ic, torch.ones_like(Ic), dMetallic=dM)
        assert e.value.status == dpcs.DPCS_ERR_INVALID_ARG
        with pytest.raises(dpcs.DPCSError) as e:
            g.ctx.render_backward_principled(g.handle, g.albedo, g.rough, None, None, g.Ip, g.view, g.params, 2, 2,
                                             sc.seed, Ec, Ic, torch.ones_like(Ic),
                                             dNormal=torch.zeros((sc.Ht, sc.Wt, 3), device=g.ctx.device))
        assert e.value.status == dpcs.DPCS_ERR_INVALID_ARG
        g.ctx.sync()
    finally:
        g.close()


def test_principled_full_size_sampled_pixels(orc):
    """The forward workload's size and launch shape (corner 256^2, 64 spp,
    3 bounces, 32 lanes per pixel) with both maps: 300 random pixels against
    the oracle run on those pixels alone."""
    torch = need_cuda()
    sc = scenes.with_principled(scenes.corner(res=256, spp=64, bounces=3, seed=1000), seed=4000)
    g = GpuScene(sc)
    try:
        m, n = _maps(g, sc)
        Ec, Ic = _render(g, sc, m, n)
        Ec, Ic = Ec.cpu().numpy().reshape(-1, 3), Ic.cpu().numpy().reshape(-1, 3)
    finally:
        g.close()
    px = np.random.default_rng(11).choice(sc.Hc * sc.Wc, 300, replace=False)
    rEc, rIc = orc.render(sc, pixels=px)
    assert rEc.max() > 0
    ok, info = pixel_parity(Ec[px], rEc)
    assert ok, info
    ok, info = pixel_parity(Ic[px], rIc, atol=crf_atol(sc, rEc))
    assert ok, info


def test_principled_degenerate_inputs(orc):
    """No bounces, a dark projector, an empty scene and a one-pixel camera
    with one sample: the principled calls return what the oracle returns
    (zeros where nothing is lit) and their adjoints stay finite."""
    torch = need_cuda()
    sc = scenes.with_principled(scenes.corner(res=16, tex=16, spp=3, bounces=2, seed=4), seed=2)
    g = GpuScene(sc)
    try:
        m, n = _maps(g, sc)
        Ec, Ic = g.ctx.render_principled(g.handle, g.albedo, g.rough, m, n, g.Ip, g.view, g.params, 3, 0, 1,
                                         Ec=torch.empty((sc.Hc, sc.Wc, 3), device=g.ctx.device))
        g.ctx.sync()
        assert not Ec.any() and not Ic.any()
        Ec, Ic = g.ctx.render_principled(g.handle, g.albedo, g.rough, m, n, torch.zeros_like(g.Ip), g.view,
                                         g.params, 3, 2, 1, Ec=torch.empty((sc.Hc, sc.Wc, 3), device=g.ctx.device))
        dM, dN = torch.zeros_like(m), torch.zeros_like(n)
        g.ctx.render_backward_principled(g.handle, g.albedo, g.rough, m, n, torch.zeros_like(g.Ip), g.view,
                                         g.params, 3, 2, 1, Ec, Ic, torch.ones_like(Ic), dMetallic=dM, dNormal=dN)
        g.ctx.sync()
        assert not Ec.any() and not dM.any() and not dN.any()
    finally:
        g.close()
    one = sc.replace(Hc=1, Wc=1, Kc=scenes.intrinsics(1, 1, 40.0), spp=1)
    g = GpuScene(one)
    try:
        m, n = _maps(g, one)
        Ec, Ic = _render(g, one, m, n)
        rE, _ = orc.render(one)
        np.testing.assert_allclose(Ec.cpu().numpy(), rE, rtol=1e-4, atol=1e-7)
    finally:
        g.close()
    empty = sc.replace(verts=np.zeros((0, 3), np.float32), tris=np.zeros((0, 3), np.int32),
                       uv=np.zeros((0, 2), np.float32))
    g = GpuScene(empty)
    try:
        m, n = _maps(g, empty)
        Ec, Ic = _render(g, empty, m, n)
        assert not Ec.any()
    finally:
        g.close()


@pytest.mark.parametrize("spp,bounces", [(16, 3), (64, 2)])
def test_principled_kept_records_equal_the_replay(spp, bounces):
    """dpcs_render_keep_principled renders what dpcs_render_principled
    renders, bit for bit, and the adjoint from its records equals the
    re-tracing replay (every material gradient) to atomic rounding, twice
    from the same records; a kept plain render does not serve the principled
    adjoint."""
    torch = need_cuda()
    sc = scenes.with_principled(scenes.corner(res=24, tex=16, spp=spp, bounces=bounces, seed=6), seed=8)
    g = GpuScene(sc)
    try:
        c = g.ctx
        m, n = torch.from_numpy(sc.metallic).cuda(), torch.from_numpy(sc.normal).cuda()
        W = torch.from_numpy(np.random.default_rng(spp).normal(size=(sc.Hc, sc.Wc, 3)).astype(np.float32)).cuda()
        args = (g.handle, g.albedo, g.rough, m, n, g.Ip, g.view, g.params, sc.spp, sc.bounces, sc.seed)

        def grads():
            return {"dIp": torch.zeros_like(g.Ip), "dA": torch.zeros_like(g.albedo), "dR": torch.zeros_like(g.rough),
                    "dM": torch.zeros_like(m), "dN": torch.zeros_like(n), "dP": torch.zeros(11, device="cuda")}

        def backward(Ec, Ic, gr, kept):
            c.render_backward_principled(*args, Ec, Ic, W, dIp=gr["dIp"], dAlbedo=gr["dA"], dRough=gr["dR"],
                                         dMetallic=gr["dM"], dNormal=gr["dN"], dParams=gr["dP"], kept=kept)

        E0 = torch.empty_like(W)
        I0, _ = c.render_principled(*args, Ec=E0)
        g0 = grads()
        backward(E0, I0, g0, False)
        E1 = torch.empty_like(W)
        I1, _ = c.render_principled(*args, Ec=E1, keep=True)
        g1, g2 = grads(), grads()
        backward(E1, I1, g1, True)
        backward(E1, I1, g2, True)
        c.sync()
        assert torch.equal(E0, E1) and torch.equal(I0, I1)
        for gk in (g1, g2):
            for k in g0:
                a, b = g0[k].cpu().numpy(), gk[k].cpu().numpy()
                assert np.abs(a).max() > 0, k
                np.testing.assert_allclose(b, a, rtol=1e-4, atol=1e-6 * np.abs(a).max(), err_msg=k)
        c.render(g.handle, g.albedo, g.rough, g.Ip, g.view, g.params, sc.spp, sc.bounces, sc.seed, keep=True)
        with pytest.raises(dpcs.DPCSError) as e:
            backward(E1, I1, grads(), True)
        assert e.value.status == dpcs.DPCS_ERR_INVALID_ARG
        c.sync()
    finally:
        g.close()
