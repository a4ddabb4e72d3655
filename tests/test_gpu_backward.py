"""Adjoint parity: GPU path-replay backward vs the oracle's FP64 adjoint on
the same paths, plus the loss and Adam kernels against plain NumPy."""
import numpy as np
import pytest

from paper_2503_12174_gb300 import scenes
from gpu_util import GpuScene, ctx, need_cuda

pytestmark = pytest.mark.gpu


def _grad_close(g, r, rtol, scale_tol):
    """|g - r| <= rtol |r| + scale_tol * max|r| element-wise."""
    g, r = np.asarray(g, np.float64).ravel(), np.asarray(r, np.float64).ravel()
    scale = np.abs(r).max()
    err = np.abs(g - r) - (rtol * np.abs(r) + scale_tol * scale)
    return bool(np.all(err <= 0)), float(np.max(np.abs(g - r) / (np.abs(r) + 1e-30))), scale


@pytest.mark.parametrize("accum", ["f32", "f64"])
@pytest.mark.parametrize("res,spp,bounces,clip", [(24, 4, 3, 0.0), (31, 5, 2, 0.05), (20, 16, 1, 0.0)])
def test_backward_matches_oracle(orc, res, spp, bounces, clip, accum):
    torch = need_cuda()
    from paper_2503_12174_gb300 import dpcs
    sc = scenes.corner(res=res, tex=32, spp=spp, bounces=bounces, seed=3)
    p = sc.params
    sc = sc.replace(params=scenes.Params(gamma_p=p.gamma_p, gain_p=1.2, gamma_c=p.gamma_c, gain_c=p.gain_c,
                                         wb=p.wb, k_proj=p.k_proj, ks=p.ks, f0=p.f0, clip=clip))
    g = GpuScene(sc)
    rng = np.random.default_rng(0)
    W = rng.normal(size=(sc.Hc, sc.Wc, 3)).astype(np.float32)
    try:
        Ec, Ic = g.render()
        g.ctx.set_grad_accum(dpcs.DPCS_ACCUM_F64 if accum == "f64" else dpcs.DPCS_ACCUM_F32)
        try:
            grads = g.backward(Ec, Ic, torch.from_numpy(W).cuda())
        finally:
            g.ctx.set_grad_accum(dpcs.DPCS_ACCUM_F32)
    finally:
        g.close()
    ref = orc.render_backward(sc, W.astype(np.float64))
    for k in ("dIp", "dalbedo", "drough"):
        ok, mx, scale = _grad_close(grads[k], ref[k], 1e-3, 1e-5)
        assert scale > 0 and ok, (k, mx, scale)
    ok, mx, _ = _grad_close(grads["dparams"], ref["dparams"], 1e-4, 1e-6)
    assert ok, ("dparams", grads["dparams"], ref["dparams"])


def test_backward_64_random_parameters_full_size(orc):
    """Compensation workload at 512x512 / 16 spp: the GPU gradient on 64
    random projector texels equals the oracle's gradient of the same pixels."""
    torch = need_cuda()
    sc = scenes.compensation(res=512, spp=16)
    g = GpuScene(sc)
    rng = np.random.default_rng(5)
    # loss on a random pixel subset so the oracle only replays those pixels
    px = rng.choice(sc.Hc * sc.Wc, 400, replace=False)
    Wfull = np.zeros((sc.Hc * sc.Wc, 3), np.float32)
    Wfull[px] = rng.normal(size=(len(px), 3))
    try:
        Ec, Ic = g.render()
        grads = g.backward(Ec, Ic, torch.from_numpy(Wfull.reshape(sc.Hc, sc.Wc, 3)).cuda())
    finally:
        g.close()
    ref = orc.render_backward(sc, Wfull[px].astype(np.float64), pixels=px)
    r = ref["dIp"].ravel()
    gg = grads["dIp"].ravel()
    nz = np.flatnonzero(np.abs(r) > 1e-3 * np.abs(r).max())
    pick = rng.choice(nz, min(64, len(nz)), replace=False)
    np.testing.assert_allclose(gg[pick], r[pick], rtol=1e-3, atol=1e-5 * np.abs(r).max())
    ok, mx, _ = _grad_close(grads["dparams"], ref["dparams"], 1e-3, 1e-6)
    assert ok, (grads["dparams"], ref["dparams"])


def _config3_first_step(orc, mode):
    """The compensation workload's first step at full size (512^2 camera,
    projector and textures, 16 spp, 3 bounces): Ip = 0.5, target = a render
    of the scene's random-blob projector image, L2 loss, every gradient.
    Returns the GPU gradients (accumulation ``mode``), the oracle's adjoint of
    the same paths for the same dLoss/dIc, and its unit-tap mass B."""
    torch = need_cuda()
    from paper_2503_12174_gb300 import dpcs

    sc = scenes.compensation(res=512, spp=16)
    g = GpuScene(sc)
    try:
        target, _ = g.render(Ip=g.Ip, seed=sc.seed + 7)
        P = torch.full_like(g.Ip, 0.5)
        Ec, Ic = g.render(Ip=P)
        dIc = torch.empty_like(Ic)
        loss = torch.empty(1, device=Ic.device)
        g.ctx.l2_loss(Ic, target, dIc, loss)
        g.Ip = P
        g.ctx.set_grad_accum(mode)
        try:
            grads = g.backward(Ec, Ic, dIc)
            again = g.backward(Ec, Ic, dIc)
        finally:
            g.ctx.set_grad_accum(dpcs.DPCS_ACCUM_F32)
        dIc_np = dIc.cpu().numpy().astype(np.float64)
    finally:
        g.close()
    scp = sc.replace(Ip=np.full_like(sc.Ip, 0.5))
    ref = orc.render_backward(scp, dIc_np, accel=True)
    mass = orc.render_backward(scp, np.abs(dIc_np), accel=True, unit_taps=True)
    return grads, again, ref, mass


# FP32 places a path vertex, and so its texel coordinates, to about 1e-4 of a
# texel at 512^2 (a few ulps of the hit point, magnified by the projection);
# a bilinear tap's weight can then move by up to ~1e-3, so a texel's gradient
# can move by 1e-3 of the total size B of the contributions that reach it
# through any tap (the oracle's unit-tap mass).
TAP_WEIGHT_TOL = 1e-3


@pytest.mark.parametrize("mode", ["f32", "f64"])
def test_backward_config3_64_random_parameters(orc, mode):
    """The full-size compensation step (config 3), 64 random parameters --
    40 projector texels, 13 albedo texels and all 11 response parameters
    (gamma_p, Gp, gamma_c, Gc, w):
    - each response parameter within 1e-4 relative of the oracle's FP64
      adjoint (sums over every pixel or texel, where tap-weight rounding
      cancels);
    - each texel within 1e-4 relative plus TAP_WEIGHT_TOL x its unit-tap mass;
    - the same texel bound on at least 99.9 % of all texels (the rest are
      paths whose discrete decisions -- frustum border, grazing shadow ray,
      horizon -- fall the other way in FP32 and FP64, as for images);
    - 64 directional derivatives, along smooth random fields over the
      projector image and the albedo map, within 1e-4 relative;
    - FP64 accumulation gives the same gradients bit for bit on a repeat."""
    from paper_2503_12174_gb300 import dpcs

    grads, again, ref, mass = _config3_first_step(
        orc, dpcs.DPCS_ACCUM_F64 if mode == "f64" else dpcs.DPCS_ACCUM_F32)
    rng = np.random.default_rng(64)
    picked = 0
    for kind, n in (("dIp", 40), ("dalbedo", 13)):
        r, gg, B = ref[kind].ravel(), grads[kind].ravel(), mass[kind].ravel()
        bound = 1e-4 * np.abs(r) + TAP_WEIGHT_TOL * B
        cand = np.flatnonzero(r != 0.0)
        pick = rng.choice(cand, n, replace=False)
        bad = np.abs(gg[pick] - r[pick]) > bound[pick]
        assert not bad.any(), (kind, pick[bad], gg[pick][bad], r[pick][bad], B[pick][bad])
        picked += n
        frac_ok = np.mean(np.abs(gg[cand] - r[cand]) <= bound[cand])
        assert frac_ok >= 0.999, (kind, frac_ok)
        # directional derivatives along smooth random fields
        H, W = ref[kind].shape[:2]
        yy, xx = np.mgrid[0:H, 0:W] / max(H, W)
        for _ in range(32):
            f = np.zeros((H, W))
            for _ in range(4):
                cx, cy, sg = rng.uniform(0, 1), rng.uniform(0, 1), rng.uniform(0.05, 0.3)
                f += rng.normal() * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * sg * sg))
            f = f[..., None] * rng.normal(size=(1, 1, 3))
            a, b = float((f * grads[kind]).sum()), float((f * ref[kind]).sum())
            assert abs(a - b) <= 1e-4 * abs(b), (kind, a, b)
    r, gg = ref["dparams"], grads["dparams"]
    bad = np.abs(gg - r) > 1e-4 * np.abs(r)
    assert not bad.any(), ("dparams", gg, r)
    picked += 11
    assert picked == 64
    if mode == "f64":
        for k in grads:
            assert np.array_equal(grads[k], again[k]), k


def test_backward_without_texture_outputs(orc):
    """dAlbedo = dRough = NULL (compensation's call) skips the texture
    scatters; dIp and dParams still equal the oracle's, and a later call that
    asks for the textures gets them."""
    torch = need_cuda()
    sc = scenes.corner(res=28, tex=32, spp=4, bounces=3, seed=9)
    g = GpuScene(sc)
    rng = np.random.default_rng(2)
    W = rng.normal(size=(sc.Hc, sc.Wc, 3)).astype(np.float32)
    try:
        Ec, Ic = g.render()
        dIp = torch.zeros_like(g.Ip)
        dP = torch.zeros(11, dtype=torch.float32, device=g.ctx.device)
        g.ctx.render_backward(g.handle, g.albedo, g.rough, g.Ip, g.view, g.params, sc.spp, sc.bounces, sc.seed, Ec,
                              Ic, torch.from_numpy(W).cuda(), dIp=dIp, dParams=dP)
        g.ctx.sync()
        full = g.backward(Ec, Ic, torch.from_numpy(W).cuda())
    finally:
        g.close()
    ref = orc.render_backward(sc, W.astype(np.float64))
    ok, mx, scale = _grad_close(dIp.cpu().numpy(), ref["dIp"], 1e-3, 1e-5)
    assert scale > 0 and ok, ("dIp", mx, scale)
    ok, mx, _ = _grad_close(dP.cpu().numpy(), ref["dparams"], 1e-4, 1e-6)
    assert ok, ("dparams", dP.cpu().numpy(), ref["dparams"])
    for k in ("dalbedo", "drough"):
        ok, mx, scale = _grad_close(full[k], ref[k], 1e-3, 1e-5)
        assert scale > 0 and ok, (k, mx, scale)


def test_l2_loss_and_adam():
    torch = need_cuda()
    c = ctx()
    rng = np.random.default_rng(1)
    a = rng.random((37, 41, 3)).astype(np.float32)
    b = rng.random((37, 41, 3)).astype(np.float32)
    A, B = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    d = torch.empty_like(A)
    loss = torch.empty(1, device="cuda")
    c.l2_loss(A, B, d, loss)
    c.sync()
    np.testing.assert_allclose(d.cpu().numpy(), a - b, rtol=0, atol=0)
    np.testing.assert_allclose(loss.item(), 0.5 * np.sum((a.astype(np.float64) - b) ** 2), rtol=1e-6)
    import oracle

    p = rng.random(1000).astype(np.float32)
    gr = rng.normal(size=1000).astype(np.float32)
    P, G = torch.from_numpy(p).cuda(), torch.from_numpy(gr).cuda()
    M, V = torch.zeros_like(P), torch.zeros_like(P)
    pr, mr, vr = p.astype(np.float64), np.zeros(1000), np.zeros(1000)
    for step in range(1, 4):
        c.adam(P, G, M, V, step, lr=0.05)
        oracle.adam_step(pr, gr.astype(np.float64), mr, vr, step, lr=0.05)
    c.sync()
    np.testing.assert_allclose(P.cpu().numpy(), pr, rtol=1e-5, atol=1e-6)
