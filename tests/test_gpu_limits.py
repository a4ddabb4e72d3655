"""The largest path the library accepts (DPCS_MAX_BOUNCES vertices) inside a
closed sphere, where most paths reach that length: the render, the replay
adjoint, the one-trace loss step (8 records per lane), the kept records and
the principled material, each against the oracle or against the separate
calls on the same paths."""
import numpy as np
import pytest

from paper_2503_12174_gb300 import dpcs, scenes
from gpu_util import GpuScene, crf_atol, need_cuda, pixel_parity

pytestmark = pytest.mark.gpu


def _sphere():
    sc = scenes.sphere(subdiv=3, res=20, spp=2, bounces=dpcs.DPCS_MAX_BOUNCES, seed=3)
    p = sc.params
    # a glossy lobe and a non-linear response so every term of the adjoint is exercised
    return sc.replace(params=scenes.Params(gamma_p=(1.8, 2.0, 2.2), gain_p=1.1, gamma_c=(0.8, 0.9, 1.0),
                                           gain_c=1.2, wb=(1.0, 1.1, 0.9), k_proj=p.k_proj, ks=0.5, f0=0.04))


def _grad_close(g, r, rtol, scale_tol):
    g, r = np.asarray(g, np.float64).ravel(), np.asarray(r, np.float64).ravel()
    scale = np.abs(r).max()
    return bool(np.all(np.abs(g - r) <= rtol * np.abs(r) + scale_tol * scale)), scale


def test_longest_paths_render_and_adjoint_match_oracle(orc):
    torch = need_cuda()
    sc = _sphere()
    rng = np.random.default_rng(0)
    W = rng.normal(size=(sc.Hc, sc.Wc, 3)).astype(np.float32)
    g = GpuScene(sc)
    try:
        Ec, Ic = g.render()
        grads = g.backward(Ec, Ic, torch.from_numpy(W).cuda())
        Ec, Ic = Ec.cpu().numpy(), Ic.cpu().numpy()
    finally:
        g.close()
    rEc, rIc = orc.render(sc)
    ok, info = pixel_parity(Ec, rEc)
    assert ok, info
    ok, info = pixel_parity(Ic, rIc, atol=crf_atol(sc, rEc))
    assert ok, info
    ref = orc.render_backward(sc, W.astype(np.float64))
    for k in ("dIp", "dalbedo", "drough"):
        ok, scale = _grad_close(grads[k], ref[k], 1e-3, 2e-5)
        assert scale > 0 and ok, k
    ok, _ = _grad_close(grads["dparams"], ref["dparams"], 1e-3, 1e-6)
    assert ok, (grads["dparams"], ref["dparams"])


def test_longest_paths_one_trace_and_kept_records_equal_the_replay():
    """8 vertices per path: the one-trace step keeps 8 records per lane and
    the kept-record adjoint sweeps 8 per path; both equal the re-tracing
    replay on the same paths."""
    torch = need_cuda()
    sc = _sphere()
    g = GpuScene(sc)
    try:
        c = g.ctx
        tgt = torch.full((sc.Hc, sc.Wc, 3), 0.05, device="cuda")
        out = {}
        for mode in ("replay", "fused", "kept"):
            Ic, Ec = torch.empty_like(tgt), torch.empty_like(tgt)
            loss, dIc = torch.zeros(1, device="cuda"), torch.empty_like(tgt)
            gr = {"dIp": torch.zeros_like(g.Ip), "dA": torch.zeros_like(g.albedo), "dR": torch.zeros_like(g.rough),
                  "dP": torch.zeros(11, device="cuda")}
            if mode == "fused":
                c.render_loss_backward(g.handle, g.albedo, g.rough, g.Ip, g.view, g.params, sc.spp, sc.bounces,
                                       sc.seed, tgt, loss, loss_kind=0, Ic=Ic, Ec=Ec, dIp=gr["dIp"],
                                       dAlbedo=gr["dA"], dRough=gr["dR"], dParams=gr["dP"])
            else:
                c.render(g.handle, g.albedo, g.rough, g.Ip, g.view, g.params, sc.spp, sc.bounces, sc.seed, Ic=Ic,
                         Ec=Ec, keep=mode == "kept")
                c.l2_loss(Ic, tgt, dIc, loss)
                c.render_backward(g.handle, g.albedo, g.rough, g.Ip, g.view, g.params, sc.spp, sc.bounces, sc.seed,
                                  Ec, Ic, dIc, dIp=gr["dIp"], dAlbedo=gr["dA"], dRough=gr["dR"], dParams=gr["dP"],
                                  kept=mode == "kept")
            c.sync()
            out[mode] = (Ic.cpu().numpy(), loss.item(), {k: v.cpu().numpy().astype(np.float64) for k, v in gr.items()})
        I0, l0, g0 = out["replay"]
        for mode in ("fused", "kept"):
            I1, l1, g1 = out[mode]
            np.testing.assert_array_equal(I1, I0)
            assert abs(l1 - l0) <= 1e-5 * abs(l0)
            for k in g0:
                assert np.abs(g0[k]).max() > 0, k
                np.testing.assert_allclose(g1[k], g0[k], rtol=1e-4, atol=1e-6 * np.abs(g0[k]).max(),
                                           err_msg=f"{mode} {k}")
    finally:
        g.close()


def test_longest_paths_principled_match_oracle(orc):
    torch = need_cuda()
    sc = scenes.with_principled(_sphere(), seed=9)
    rng = np.random.default_rng(1)
    W = rng.normal(size=(sc.Hc, sc.Wc, 3)).astype(np.float32)
    g = GpuScene(sc)
    try:
        m, n = torch.from_numpy(sc.metallic).cuda(), torch.from_numpy(sc.normal).cuda()
        Ec = torch.empty((sc.Hc, sc.Wc, 3), device="cuda")
        Ic, _ = g.ctx.render_principled(g.handle, g.albedo, g.rough, m, n, g.Ip, g.view, g.params, sc.spp,
                                        sc.bounces, sc.seed, Ec=Ec)
        gr = {"dIp": torch.zeros_like(g.Ip), "dalbedo": torch.zeros_like(g.albedo),
              "drough": torch.zeros_like(g.rough), "dmetallic": torch.zeros_like(m), "dnormal": torch.zeros_like(n)}
        g.ctx.render_backward_principled(g.handle, g.albedo, g.rough, m, n, g.Ip, g.view, g.params, sc.spp,
                                         sc.bounces, sc.seed, Ec, Ic, torch.from_numpy(W).cuda(), dIp=gr["dIp"],
                                         dAlbedo=gr["dalbedo"], dRough=gr["drough"], dMetallic=gr["dmetallic"],
                                         dNormal=gr["dnormal"])
        g.ctx.sync()
        Ec = Ec.cpu().numpy()
        gr = {k: v.cpu().numpy().astype(np.float64) for k, v in gr.items()}
    finally:
        g.close()
    rEc, _ = orc.render(sc)
    ok, info = pixel_parity(Ec, rEc)
    assert ok, info
    ref = orc.render_backward(sc, W.astype(np.float64))
    for k in gr:
        ok, scale = _grad_close(gr[k], ref[k], 1e-3, 2e-5)
        assert scale > 0 and ok, k
