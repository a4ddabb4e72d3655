"""dpcs_render_keep + dpcs_render_backward_kept: a render that keeps its
path records and an adjoint that sweeps them instead of re-tracing, against
the plain render and the path replay on the same paths."""
import numpy as np
import pytest

from paper_2503_12174_gb300 import dpcs, scenes
from gpu_util import GpuScene, ctx, need_cuda

pytestmark = pytest.mark.gpu


def _backward(g, sc, Ec, Ic, dIc, spp, bounces, kept):
    torch = need_cuda()
    out = {"dIp": torch.zeros_like(g.Ip), "dalbedo": torch.zeros_like(g.albedo), "drough": torch.zeros_like(g.rough),
           "dparams": torch.zeros(11, device="cuda")}
    g.ctx.render_backward(g.handle, g.albedo, g.rough, g.Ip, g.view, g.params, spp, bounces, sc.seed, Ec, Ic, dIc,
                          dIp=out["dIp"], dAlbedo=out["dalbedo"], dRough=out["drough"], dParams=out["dparams"],
                          kept=kept)
    return out


@pytest.mark.parametrize("accum", ["f32", "f64"])
@pytest.mark.parametrize("case", ["corner16", "corner64", "corner256", "heightfield_rr"])
def test_kept_adjoint_equals_replay(case, accum):
    torch = need_cuda()
    if case == "heightfield_rr":
        sc = scenes.heightfield(spp=8, cam=96, proj=(64, 80), tex=64, n_vert=41)
    else:
        spp = int(case[len("corner"):])
        sc = scenes.corner(res=40, tex=32, spp=spp, bounces=3, seed=2)
    g = GpuScene(sc)
    g.ctx.set_grad_accum(dpcs.DPCS_ACCUM_F64 if accum == "f64" else dpcs.DPCS_ACCUM_F32)
    try:
        Ea = torch.empty((sc.Hc, sc.Wc, 3), device="cuda")
        Ia, _ = g.ctx.render(g.handle, g.albedo, g.rough, g.Ip, g.view, g.params, sc.spp, sc.bounces, sc.seed, Ec=Ea)
        Eb = torch.empty_like(Ea)
        Ib, _ = g.ctx.render(g.handle, g.albedo, g.rough, g.Ip, g.view, g.params, sc.spp, sc.bounces, sc.seed, Ec=Eb,
                             keep=True)
        g.ctx.sync()
        assert torch.equal(Ia, Ib) and torch.equal(Ea, Eb)
        dIc = torch.from_numpy(np.random.default_rng(1).normal(size=(sc.Hc, sc.Wc, 3)).astype(np.float32)).cuda()
        ref = _backward(g, sc, Ea, Ia, dIc, sc.spp, sc.bounces, kept=False)
        got = _backward(g, sc, Eb, Ib, dIc, sc.spp, sc.bounces, kept=True)
        got2 = _backward(g, sc, Eb, Ib, dIc, sc.spp, sc.bounces, kept=True)  # the records stay for a second adjoint
        g.ctx.sync()
        for k in ref:
            a = ref[k].cpu().numpy()
            for o in (got, got2):
                np.testing.assert_allclose(o[k].cpu().numpy(), a, rtol=1e-4, atol=1e-6 * np.abs(a).max(), err_msg=k)
            if accum == "f64":  # order-independent sums: the second sweep repeats the first bit for bit
                np.testing.assert_array_equal(got2[k].cpu().numpy(), got[k].cpu().numpy(), err_msg=k)
    finally:
        g.ctx.set_grad_accum(dpcs.DPCS_ACCUM_F32)
        g.close()


def test_kept_adjoint_refuses_another_render():
    torch = need_cuda()
    sc = scenes.corner(res=16, tex=16, spp=4, bounces=2)
    c = dpcs.Context(0)  # a fresh context: nothing kept yet
    try:
        h = c.upload(sc.verts, sc.tris, sc.uv)
        alb, rough, Ip = (torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (sc.albedo, sc.rough, sc.Ip))
        view, prm = dpcs.view_of(sc), dpcs.make_params(sc.params)
        Ec = torch.empty((sc.Hc, sc.Wc, 3), device="cuda")
        Ic, _ = c.render(h, alb, rough, Ip, view, prm, 4, 2, 1, Ec=Ec)
        dIc = torch.ones_like(Ic)
        with pytest.raises(dpcs.DPCSError) as e:
            c.render_backward(h, alb, rough, Ip, view, prm, 4, 2, 1, Ec, Ic, dIc, dIp=torch.zeros_like(Ip), kept=True)
        assert e.value.status == dpcs.DPCS_ERR_INVALID_ARG
        c.render(h, alb, rough, Ip, view, prm, 4, 2, 1, Ic=Ic, Ec=Ec, keep=True)
        for spp, bounces, seed in ((8, 2, 1), (4, 3, 1), (4, 2, 2)):
            with pytest.raises(dpcs.DPCSError) as e:
                c.render_backward(h, alb, rough, Ip, view, prm, spp, bounces, seed, Ec, Ic, dIc,
                                  dIp=torch.zeros_like(Ip), kept=True)
            assert e.value.status == dpcs.DPCS_ERR_INVALID_ARG
        c.render_backward(h, alb, rough, Ip, view, prm, 4, 2, 1, Ec, Ic, dIc, dIp=torch.zeros_like(Ip), kept=True)
        c.sync()
        c.free(h)
    finally:
        c.close()
