"""Projector compensation (Eq. 13) on the GPU: the Adam trajectory follows
the FP64 oracle's own compensation loop step by step, the loss falls, and
the loop captured once as a CUDA graph reproduces the eager loop."""
import numpy as np
import pytest

from paper_2503_12174_gb300 import compensate, dpcs, scenes
from gpu_util import GpuScene, need_cuda

pytestmark = pytest.mark.gpu


def _setup(orc, res=20, steps=4):
    torch = need_cuda()
    sc = scenes.corner(res=res, tex=res, spp=4, bounces=2, seed=11)
    rng = np.random.default_rng(0)
    _, target = orc.render(sc, Ip=rng.random(sc.Ip.shape), seed=777)
    return torch, sc, target.astype(np.float32)


def test_compensation_follows_oracle(orc):
    torch, sc, target = _setup(orc)
    steps, lr = 4, 0.05
    g = GpuScene(sc)
    try:
        comp = compensate.Compensation(g.ctx, g.handle, g.albedo, g.rough, g.view, g.params, sc.spp, sc.bounces,
                                       steps, lr=lr, seed=sc.seed, graph=False)
        P, hist = comp.run(torch.full_like(g.Ip, 0.5), torch.from_numpy(target).cuda())
        g.ctx.sync()
        P, hist = P.cpu().numpy().astype(np.float64), hist.cpu().numpy().astype(np.float64)
    finally:
        g.close()
    Pr = np.full(sc.Ip.shape, 0.5)
    m, v = np.zeros_like(Pr), np.zeros_like(Pr)
    losses = []
    for k in range(steps):
        _, Ic = orc.render(sc, Ip=Pr, seed=sc.seed + k)
        dIc = Ic - target
        losses.append(0.5 * np.sum(dIc * dIc))
        grad = orc.render_backward(sc, dIc, Ip=Pr, seed=sc.seed + k)["dIp"]
        orc.adam_step(Pr, grad, m, v, k + 1, lr=lr)
    np.testing.assert_allclose(hist, losses, rtol=1e-3)
    assert losses[-1] < losses[0]
    # Adam normalises each texel's step, so texels whose gradient is at FP32
    # noise level may move differently; every other texel must agree closely
    np.testing.assert_allclose(P, Pr, rtol=0, atol=2e-3)


def test_graph_replay_matches_eager(orc):
    torch, sc, target = _setup(orc, res=24, steps=6)
    g = GpuScene(sc)
    try:
        args = (g.ctx, g.handle, g.albedo, g.rough, g.view, g.params, sc.spp, sc.bounces, 6)
        tgt = torch.from_numpy(target).cuda()
        init = torch.full_like(g.Ip, 0.5)
        eager = compensate.Compensation(*args, lr=0.05, seed=5, graph=False)
        Pe, he = eager.run(init, tgt)
        Pe, he = Pe.clone(), he.clone()
        graphed = compensate.Compensation(*args, lr=0.05, seed=5, graph=True)
        for _ in range(2):  # two replays: the graph resets its own state
            Pg, hg = graphed.run(init, tgt)
            g.ctx.sync()
            np.testing.assert_allclose(hg.cpu().numpy(), he.cpu().numpy(), rtol=1e-4)
            np.testing.assert_allclose(Pg.cpu().numpy(), Pe.cpu().numpy(), rtol=0, atol=1e-4)
        assert hg[-1].item() < hg[0].item()
    finally:
        g.close()


def test_denoised_compensation_follows_oracle(orc):
    """The loss on D(Ic) (Eq. 11 before the Eq. 13 loss), step by step against
    the oracle's loop with its own filter and adjoint; then the same loop as a
    CUDA-graph replay."""
    torch, sc, target = _setup(orc)
    steps, lr = 3, 0.05
    prm = dict(radius=3, sigma_s=1.5, sigma_albedo=0.1, sigma_normal=0.3, sigma_depth=0.1)
    guide = orc.gbuffer(sc).astype(np.float32)  # one guide for both sides
    g = GpuScene(sc)
    try:
        kw = dict(lr=lr, seed=sc.seed, denoise=dpcs.make_denoise_params(**prm), guide=torch.from_numpy(guide).cuda())
        args = (g.ctx, g.handle, g.albedo, g.rough, g.view, g.params, sc.spp, sc.bounces, steps)
        init, tgt = torch.full_like(g.Ip, 0.5), torch.from_numpy(target).cuda()
        P, hist = compensate.Compensation(*args, graph=False, **kw).run(init, tgt)
        P, hist = P.clone().cpu().numpy().astype(np.float64), hist.clone().cpu().numpy().astype(np.float64)
        Pg, hg = compensate.Compensation(*args, graph=True, **kw).run(init, tgt)
        g.ctx.sync()
        Pg, hg = Pg.cpu().numpy(), hg.cpu().numpy()
    finally:
        g.close()
    gd = guide.astype(np.float64)
    Pr = np.full(sc.Ip.shape, 0.5)
    m, v = np.zeros_like(Pr), np.zeros_like(Pr)
    losses = []
    for k in range(steps):
        _, Ic = orc.render(sc, Ip=Pr, seed=sc.seed + k)
        D, _ = orc.denoise(Ic, gd, prm)
        dD = D - target
        losses.append(0.5 * np.sum(dD * dD))
        grad = orc.render_backward(sc, orc.denoise_backward(dD, gd, prm), Ip=Pr, seed=sc.seed + k)["dIp"]
        orc.adam_step(Pr, grad, m, v, k + 1, lr=lr)
    np.testing.assert_allclose(hist, losses, rtol=1e-3)
    assert losses[-1] < losses[0]
    np.testing.assert_allclose(P, Pr, rtol=0, atol=2e-3)
    np.testing.assert_allclose(hg, hist, rtol=1e-4)
    np.testing.assert_allclose(Pg, P, rtol=0, atol=1e-4)


def test_checkpoint_and_resume(orc, tmp_path):
    """Three steps, a checkpoint, a fresh object that resumes and runs three
    more: the same trajectory as six steps in one go (up to the rounding of
    the adjoint's float atomics)."""
    torch, sc, target = _setup(orc, res=20, steps=6)
    g = GpuScene(sc)
    try:
        args = (g.ctx, g.handle, g.albedo, g.rough, g.view, g.params, sc.spp, sc.bounces, 6)
        init, tgt = torch.full_like(g.Ip, 0.5), torch.from_numpy(target).cuda()
        whole = compensate.Compensation(*args, lr=0.05, seed=7, graph=False)
        whole.start(init, tgt)
        Pw, hw = whole.advance(6)
        Pw, hw = Pw.clone(), hw.clone()
        first = compensate.Compensation(*args, lr=0.05, seed=7, graph=False)
        first.start(init, tgt)
        first.advance(3)
        path = str(tmp_path / "comp.npz")
        first.save(path)
        second = compensate.Compensation(*args, lr=0.05, seed=7, graph=False)
        second.resume(path)
        Pr, hr = second.advance(3)
        g.ctx.sync()
        np.testing.assert_allclose(hr.cpu().numpy(), hw.cpu().numpy(), rtol=1e-4)
        np.testing.assert_allclose(Pr.cpu().numpy(), Pw.cpu().numpy(), rtol=0, atol=1e-4)
        with pytest.raises(ValueError):
            compensate.Compensation(*args, lr=0.05, seed=8, graph=False).resume(path)
    finally:
        g.close()


def test_checkpoint_and_resume_is_exact_with_fp64_accumulation(orc, tmp_path):
    """With FP64 gradient accumulation the adjoint's sums do not depend on the
    order of its atomics (beyond FP64 rounding, far below the FP32 result), so
    three steps, a checkpoint and three resumed steps reproduce six steps in
    one go bit for bit."""
    from paper_2503_12174_gb300 import dpcs

    torch, sc, target = _setup(orc, res=20, steps=6)
    g = GpuScene(sc)
    g.ctx.set_grad_accum(dpcs.DPCS_ACCUM_F64)
    try:
        args = (g.ctx, g.handle, g.albedo, g.rough, g.view, g.params, sc.spp, sc.bounces, 6)
        init, tgt = torch.full_like(g.Ip, 0.5), torch.from_numpy(target).cuda()
        whole = compensate.Compensation(*args, lr=0.05, seed=7, graph=False)
        whole.start(init, tgt)
        Pw, hw = whole.advance(6)
        Pw, hw = Pw.clone(), hw.clone()
        first = compensate.Compensation(*args, lr=0.05, seed=7, graph=False)
        first.start(init, tgt)
        first.advance(3)
        path = str(tmp_path / "comp64.npz")
        first.save(path)
        second = compensate.Compensation(*args, lr=0.05, seed=7, graph=False)
        second.resume(path)
        Pr, hr = second.advance(3)
        g.ctx.sync()
        np.testing.assert_array_equal(hr.cpu().numpy(), hw.cpu().numpy())
        np.testing.assert_array_equal(Pr.cpu().numpy(), Pw.cpu().numpy())
    finally:
        g.ctx.set_grad_accum(dpcs.DPCS_ACCUM_F32)
        g.close()


@pytest.mark.parametrize("denoised", [False, True])
def test_principled_compensation_follows_oracle(orc, denoised):
    """Compensation on a surface with metallic and normal maps: the one-trace
    step (and, with the Eq. 11 filter, the separate calls) follow the
    oracle's loop with the same maps; the CUDA graph reproduces the eager
    loop."""
    torch = need_cuda()
    sc = scenes.with_principled(scenes.corner(res=20, tex=20, spp=4, bounces=2, seed=11), seed=13)
    rng = np.random.default_rng(1)
    _, target = orc.render(sc, Ip=rng.random(sc.Ip.shape), seed=777)
    target = target.astype(np.float32)
    steps, lr = 3, 0.05
    prm = dpcs.make_denoise_params(radius=2, sigma_s=1.0, sigma_albedo=0.2, sigma_normal=0.3, sigma_depth=0.2) \
        if denoised else None
    g = GpuScene(sc)
    try:
        m = torch.from_numpy(sc.metallic).cuda()
        n = torch.from_numpy(sc.normal).cuda()
        args = (g.ctx, g.handle, g.albedo, g.rough, g.view, g.params, sc.spp, sc.bounces, steps)
        comp = compensate.Compensation(*args, lr=lr, seed=sc.seed, graph=False, denoise=prm, metallic=m, normal=n)
        init, tgt = torch.full_like(g.Ip, 0.5), torch.from_numpy(target).cuda()
        P, hist = comp.run(init, tgt)
        P, hist = P.clone(), hist.clone()
        guide = comp.guide.cpu().numpy().astype(np.float64) if denoised else None
        graphed = compensate.Compensation(*args, lr=lr, seed=sc.seed, graph=True, denoise=prm, metallic=m, normal=n)
        Pg, hg = graphed.run(init, tgt)
        g.ctx.sync()
        np.testing.assert_allclose(hg.cpu().numpy(), hist.cpu().numpy(), rtol=1e-4)
        P, hist = P.cpu().numpy().astype(np.float64), hist.cpu().numpy().astype(np.float64)
    finally:
        g.close()
    dprm = None if prm is None else {"radius": 2, "sigma_s": 1.0, "sigma_albedo": 0.2, "sigma_normal": 0.3,
                                     "sigma_depth": 0.2}
    Pr = np.full(sc.Ip.shape, 0.5)
    mo, vo = np.zeros_like(Pr), np.zeros_like(Pr)
    losses = []
    for k in range(steps):
        _, Ic = orc.render(sc, Ip=Pr, seed=sc.seed + k)
        if denoised:
            D, W = orc.denoise(Ic, guide, dprm)
            dD = D - target
            losses.append(0.5 * np.sum(dD * dD))
            dIc = orc.denoise_backward(dD, guide, dprm)
        else:
            dIc = Ic - target
            losses.append(0.5 * np.sum(dIc * dIc))
        grad = orc.render_backward(sc, dIc, Ip=Pr, seed=sc.seed + k)["dIp"]
        orc.adam_step(Pr, grad, mo, vo, k + 1, lr=lr)
    np.testing.assert_allclose(hist, losses, rtol=1e-3)
    np.testing.assert_allclose(P, Pr, rtol=0, atol=2e-3)


def test_principled_fused_step_equals_separate_calls():
    """render_loss_backward_principled inside and outside its record limits
    (16 spp: one trace; 256 spp: render, loss, replay): Ec equals
    render_principled's bit for bit, and the loss and every gradient agree
    with the separate calls to atomic rounding, for L2 and L1."""
    torch = need_cuda()
    sc = scenes.with_principled(scenes.corner(res=24, tex=16, spp=16, bounces=3, seed=3), seed=5)
    g = GpuScene(sc)
    try:
        m = torch.from_numpy(sc.metallic).cuda()
        n = torch.from_numpy(sc.normal).cuda()
        tgt = torch.rand((sc.Hc, sc.Wc, 3), device="cuda", generator=torch.Generator("cuda").manual_seed(0)) * 0.1
        for spp in (16, 256):
            for kind in (0, 1):
                scale = 1.0 if kind == 0 else 1.0 / (sc.Hc * sc.Wc * 3)
                out = {}
                for fused in (True, False):
                    Ec = torch.empty((sc.Hc, sc.Wc, 3), device="cuda")
                    loss = torch.zeros(1, device="cuda")
                    gr = {"dIp": torch.zeros_like(g.Ip), "dA": torch.zeros_like(g.albedo),
                          "dR": torch.zeros_like(g.rough), "dM": torch.zeros_like(m), "dN": torch.zeros_like(n),
                          "dP": torch.zeros(11, device="cuda")}
                    if fused:
                        Ic = g.ctx.render_loss_backward_principled(
                            g.handle, g.albedo, g.rough, m, n, g.Ip, g.view, g.params, spp, sc.bounces, sc.seed,
                            tgt, loss, loss_kind=kind, scale=scale, Ec=Ec, dIp=gr["dIp"], dAlbedo=gr["dA"],
                            dRough=gr["dR"], dMetallic=gr["dM"], dNormal=gr["dN"], dParams=gr["dP"])
                    else:
                        Ic, _ = g.ctx.render_principled(g.handle, g.albedo, g.rough, m, n, g.Ip, g.view, g.params,
                                                        spp, sc.bounces, sc.seed, Ec=Ec)
                        dIc = torch.empty_like(Ic)
                        if kind == 0:
                            g.ctx.l2_loss(Ic, tgt, dIc, loss)
                        else:
                            g.ctx.l1_loss(Ic, tgt, dIc, loss, scale=scale)
                        g.ctx.render_backward_principled(g.handle, g.albedo, g.rough, m, n, g.Ip, g.view, g.params,
                                                         spp, sc.bounces, sc.seed, Ec, Ic, dIc, dIp=gr["dIp"],
                                                         dAlbedo=gr["dA"], dRough=gr["dR"], dMetallic=gr["dM"],
                                                         dNormal=gr["dN"], dParams=gr["dP"])
                    g.ctx.sync()
                    out[fused] = (Ec.cpu().numpy(), Ic.cpu().numpy(), loss.item(),
                                  {k: v.cpu().numpy().astype(np.float64) for k, v in gr.items()})
                (E1, I1, l1, g1), (E0, I0, l0, g0) = out[True], out[False]
                np.testing.assert_array_equal(E1, E0)
                np.testing.assert_allclose(I1, I0, rtol=1e-6, atol=1e-9)
                assert abs(l1 - l0) <= 1e-4 * abs(l0), (spp, kind, l1, l0)
                for k in g0:
                    np.testing.assert_allclose(g1[k], g0[k], rtol=1e-3, atol=1e-5 * np.abs(g0[k]).max(),
                                               err_msg=f"{spp} {kind} {k}")
    finally:
        g.close()
