"""dpcs_render_loss_backward: the fused render + per-pixel loss + adjoint
against the separate calls (render, loss, render_backward) on the same
paths, in both its fused and its fallback regime, and against the oracle's
chain."""
import numpy as np
import pytest

from paper_2503_12174_gb300 import dpcs, scenes
from gpu_util import GpuScene, need_cuda

pytestmark = pytest.mark.gpu


def _grads(torch, g):
    return {"dIp": torch.zeros_like(g.Ip), "dalbedo": torch.zeros_like(g.albedo), "drough": torch.zeros_like(g.rough),
            "dparams": torch.zeros(11, device="cuda")}


def _separate(g, sc, target, kind, scale, spp, bounces):
    torch = need_cuda()
    c = g.ctx
    Ic, Ec = torch.empty_like(target), torch.empty_like(target)
    c.render(g.handle, g.albedo, g.rough, g.Ip, g.view, g.params, spp, bounces, sc.seed, Ic=Ic, Ec=Ec)
    dIc, loss = torch.empty_like(target), torch.zeros(1, device="cuda")
    if kind == 0:
        c.l2_loss(Ic, target, dIc, loss)
        dIc *= scale
        loss *= scale
    else:
        c.l1_loss(Ic, target, dIc, loss, scale=scale)
    out = _grads(torch, g)
    c.render_backward(g.handle, g.albedo, g.rough, g.Ip, g.view, g.params, spp, bounces, sc.seed, Ec, Ic, dIc,
                      dIp=out["dIp"], dAlbedo=out["dalbedo"], dRough=out["drough"], dParams=out["dparams"])
    return Ic, Ec, loss, out


def _fused(g, sc, target, kind, scale, spp, bounces):
    torch = need_cuda()
    Ec, loss = torch.empty_like(target), torch.zeros(1, device="cuda")
    out = _grads(torch, g)
    Ic = g.ctx.render_loss_backward(g.handle, g.albedo, g.rough, g.Ip, g.view, g.params, spp, bounces, sc.seed,
                                    target, loss, loss_kind=kind, scale=scale, Ec=Ec, dIp=out["dIp"],
                                    dAlbedo=out["dalbedo"], dRough=out["drough"], dParams=out["dparams"])
    return Ic, Ec, loss, out


# (spp, bounces): 16/3 and 64/3 take the fused path (1 and 2 samples per
# lane); 256/3 (8 samples per lane) and 128/4 (4 x 4 vertices) fall back
@pytest.mark.parametrize("spp,bounces", [(16, 3), (64, 3), (256, 3), (128, 4)])
@pytest.mark.parametrize("kind,scale", [(0, 0.5), (1, 1e-3)])
def test_fused_equals_separate_calls(spp, bounces, kind, scale):
    torch = need_cuda()
    sc = scenes.corner(res=40, tex=32, spp=spp, bounces=bounces, seed=4)
    g = GpuScene(sc)
    rng = np.random.default_rng(spp + bounces)
    try:
        target = torch.from_numpy(rng.uniform(0.0, 1.0, (sc.Hc, sc.Wc, 3)).astype(np.float32)).cuda()
        Ia, Ea, la, ga = _separate(g, sc, target, kind, scale, spp, bounces)
        Ib, Eb, lb, gb = _fused(g, sc, target, kind, scale, spp, bounces)
        g.ctx.sync()
        # the forward is k_render's arithmetic in the same order: bit for bit
        assert torch.equal(Ia, Ib) and torch.equal(Ea, Eb)
        np.testing.assert_allclose(lb.item(), la.item(), rtol=1e-5)
        for k in ("dIp", "dalbedo", "drough", "dparams"):
            a, b = ga[k].cpu().numpy(), gb[k].cpu().numpy()
            np.testing.assert_allclose(b, a, rtol=1e-4, atol=1e-6 * np.abs(a).max(), err_msg=k)
    finally:
        g.close()


def test_fused_full_size_equals_separate_calls():
    """The benchmark's launch configuration (512 x 512, 16 spp, 3 bounces,
    the compensation step): the fused call against the separate calls."""
    torch = need_cuda()
    sc = scenes.compensation(512, 16)
    g = GpuScene(sc)
    rng = np.random.default_rng(3)
    try:
        target = torch.from_numpy(rng.uniform(0.0, 1.0, (sc.Hc, sc.Wc, 3)).astype(np.float32)).cuda()
        Ia, Ea, la, ga = _separate(g, sc, target, 0, 1.0, sc.spp, sc.bounces)
        Ib, Eb, lb, gb = _fused(g, sc, target, 0, 1.0, sc.spp, sc.bounces)
        g.ctx.sync()
        assert torch.equal(Ia, Ib) and torch.equal(Ea, Eb)
        np.testing.assert_allclose(lb.item(), la.item(), rtol=1e-5)
        for k in ("dIp", "dparams"):
            a, b = ga[k].cpu().numpy(), gb[k].cpu().numpy()
            np.testing.assert_allclose(b, a, rtol=1e-4, atol=1e-6 * np.abs(a).max(), err_msg=k)
    finally:
        g.close()


def test_fused_gradient_matches_oracle(orc):
    torch = need_cuda()
    sc = scenes.corner(res=24, tex=16, spp=8, bounces=2, seed=7)
    g = GpuScene(sc)
    rng = np.random.default_rng(1)
    _, Ic_ref = orc.render(sc)
    # targets 0.1 away from the render, so every L1 sign is the same in FP32 and FP64
    tgt = Ic_ref + 0.1 * rng.choice([-1.0, 1.0], size=Ic_ref.shape)
    scale = 1.0 / Ic_ref.size
    try:
        Ic, Ec, loss, out = _fused(g, sc, torch.from_numpy(tgt.astype(np.float32)).cuda(), 1, scale, sc.spp,
                                   sc.bounces)
        g.ctx.sync()
        got = {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}
        got_loss = loss.item()
    finally:
        g.close()
    rl, dIc = orc.l1_loss(Ic_ref, tgt, scale)
    ref = orc.render_backward(sc, dIc)
    assert got_loss == pytest.approx(rl, rel=1e-4)
    for k in ("dIp", "dalbedo", "drough"):
        r = ref[k]
        np.testing.assert_allclose(got[k], r, rtol=1e-3, atol=1e-5 * np.abs(r).max(), err_msg=k)
    np.testing.assert_allclose(got["dparams"], ref["dparams"], rtol=1e-3, atol=1e-6 * np.abs(ref["dparams"]).max())


def test_fused_refuses_bad_loss_arguments():
    torch = need_cuda()
    sc = scenes.corner(res=16, tex=16, spp=4)
    g = GpuScene(sc)
    try:
        t = torch.zeros((sc.Hc, sc.Wc, 3), device="cuda")
        loss = torch.zeros(1, device="cuda")
        for kind, scale in ((2, 1.0), (0, 0.0), (1, -1.0)):
            with pytest.raises(dpcs.DPCSError) as e:
                g.ctx.render_loss_backward(g.handle, g.albedo, g.rough, g.Ip, g.view, g.params, 4, 2, 0, t, loss,
                                           loss_kind=kind, scale=scale)
            assert e.value.status == dpcs.DPCS_ERR_INVALID_ARG
    finally:
        g.close()


@pytest.mark.parametrize("spp,bounces", [(16, 3), (256, 3)])
def test_fused_equals_separate_calls_with_fp64_accumulation(spp, bounces):
    """With FP64 accumulators both ways of computing the step sum the same
    per-vertex contributions with order-independent atomics: the fused call
    (and its fallback) agree with the separate calls far inside the FP32
    gate, and a repeat of the fused call is bit for bit the same."""
    torch = need_cuda()
    sc = scenes.corner(res=40, tex=32, spp=spp, bounces=bounces, seed=6)
    g = GpuScene(sc)
    rng = np.random.default_rng(spp)
    g.ctx.set_grad_accum(dpcs.DPCS_ACCUM_F64)
    try:
        target = torch.from_numpy(rng.uniform(0.0, 1.0, (sc.Hc, sc.Wc, 3)).astype(np.float32)).cuda()
        Ia, Ea, la, ga = _separate(g, sc, target, 0, 0.5, spp, bounces)
        Ib, Eb, lb, gb = _fused(g, sc, target, 0, 0.5, spp, bounces)
        Ic, Ec, lc, gc = _fused(g, sc, target, 0, 0.5, spp, bounces)
        g.ctx.sync()
        assert torch.equal(Ia, Ib) and torch.equal(Ea, Eb)
        for k in ("dIp", "dalbedo", "drough", "dparams"):
            a, b, c = ga[k].cpu().numpy(), gb[k].cpu().numpy(), gc[k].cpu().numpy()
            np.testing.assert_allclose(b, a, rtol=1e-5, atol=1e-7 * np.abs(a).max(), err_msg=k)
            np.testing.assert_array_equal(c, b, err_msg=k)
    finally:
        g.ctx.set_grad_accum(dpcs.DPCS_ACCUM_F32)
        g.close()
