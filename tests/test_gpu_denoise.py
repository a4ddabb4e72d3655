"""Eq. 11 on the GPU: guide features, the cross-bilateral filter and its
adjoint against the FP64 oracle, at small sizes with ragged tiles and on
crops of a full-size image; the denoised compensation gradient end to end."""
import numpy as np
import pytest

from paper_2503_12174_gb300 import dpcs, scenes
from gpu_util import GpuScene, ctx, need_cuda

pytestmark = pytest.mark.gpu

PRMS = [dict(radius=0, sigma_s=1.0, sigma_albedo=0.0, sigma_normal=0.0, sigma_depth=0.0),
        dict(radius=3, sigma_s=1.5, sigma_albedo=0.2, sigma_normal=0.0, sigma_depth=0.0),
        dict(radius=5, sigma_s=2.0, sigma_albedo=0.1, sigma_normal=0.3, sigma_depth=0.1),
        dict(radius=8, sigma_s=4.0, sigma_albedo=0.0, sigma_normal=0.5, sigma_depth=0.2)]


def _dp(p):
    return dpcs.make_denoise_params(**p)


def test_gbuffer_matches_oracle(orc):
    torch = need_cuda()
    sc = scenes.corner(res=48, tex=32, spp=1)
    g = GpuScene(sc)
    try:
        guide = g.ctx.gbuffer(g.handle, g.albedo, g.rough, g.view)
        g.ctx.sync()
        got = guide.cpu().numpy().astype(np.float64)
    finally:
        g.close()
    ref = orc.gbuffer(sc)
    same_hit = got[..., 7] == ref[..., 7]
    # The corner's seams project onto the image diagonals, through pixel
    # centres: those rays run exactly along an edge shared by two triangles.
    # A plain FP32 hit test can miss both triangles there (a crack); the
    # library's test is watertight near edges, so the GPU misses no pixel
    # that the FP64 oracle hits.
    assert not np.any((ref[..., 7] == 1.0) & (got[..., 7] == 0.0))
    assert same_hit.all()
    both = same_hit & (ref[..., 7] == 1.0)
    # a different triangle at a shared edge (FP32 vs FP64 hit tests) changes the normal
    agree = both & (np.abs(got[..., 3:6] - ref[..., 3:6]).max(axis=-1) < 1e-4)
    assert agree.sum() >= 0.995 * both.sum()
    np.testing.assert_allclose(got[agree][:, 0:3], ref[agree][:, 0:3], atol=2e-5)
    np.testing.assert_allclose(got[agree][:, 6], ref[agree][:, 6], rtol=2e-5)
    assert np.all(got[~(got[..., 7] == 1.0)] == 0.0)


@pytest.mark.parametrize("prm", PRMS)
@pytest.mark.parametrize("shape", [(37, 29), (16, 16), (5, 70)])
def test_denoise_forward_and_adjoint_match_oracle(orc, prm, shape):
    torch = need_cuda()
    c = ctx()
    H, W = shape
    rng = np.random.default_rng(H * 100 + W)
    sc = scenes.corner(res=max(H, W), tex=32, spp=1)
    gfull = orc.gbuffer(sc)[:H, :W].astype(np.float32)
    I = rng.uniform(0.0, 2.0, (H, W, 3)).astype(np.float32)
    dO = rng.normal(size=(H, W, 3)).astype(np.float32)
    guide = torch.from_numpy(np.ascontiguousarray(gfull)).cuda()
    out, wsum = c.denoise(torch.from_numpy(I).cuda(), guide, _dp(prm))
    seed = torch.from_numpy(rng.normal(size=(H, W, 3)).astype(np.float32)).cuda()
    dI = c.denoise_backward(torch.from_numpy(dO).cuda(), guide, wsum, _dp(prm), dIc=seed.clone())
    c.sync()
    ref, rden = orc.denoise(I.astype(np.float64), gfull.astype(np.float64), prm)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=2e-5, atol=1e-6)
    np.testing.assert_allclose(wsum.cpu().numpy(), rden, rtol=2e-5)
    rdI = orc.denoise_backward(dO.astype(np.float64), gfull.astype(np.float64), prm)
    # the adjoint accumulates into dIc
    np.testing.assert_allclose(dI.cpu().numpy() - seed.cpu().numpy(), rdI, rtol=1e-4, atol=2e-5)


def test_denoise_full_size_on_crops(orc):
    """1024 x 1024 at radius 5: crops of the GPU output against the oracle
    run on the same crop plus its halo."""
    torch = need_cuda()
    sc = scenes.heightfield(spp=1)
    g = GpuScene(sc)
    prm = PRMS[2]
    rng = np.random.default_rng(11)
    try:
        guide = g.ctx.gbuffer(g.handle, g.albedo, g.rough, g.view)
        I = torch.rand((sc.Hc, sc.Wc, 3), device="cuda")
        out, wsum = g.ctx.denoise(I, guide, _dp(prm))
        g.ctx.sync()
        gh, Ih, oh = guide.cpu().numpy(), I.cpu().numpy(), out.cpu().numpy()
    finally:
        g.close()
    r = prm["radius"]
    for (y0, x0) in [(0, 0), (sc.Hc - 40, sc.Wc - 40)] + [tuple(rng.integers(0, 980, 2)) for _ in range(3)]:
        y1, x1 = y0 + 40, x0 + 40
        cy0, cx0, cy1, cx1 = max(0, y0 - r), max(0, x0 - r), min(sc.Hc, y1 + r), min(sc.Wc, x1 + r)
        ref, _ = orc.denoise(Ih[cy0:cy1, cx0:cx1].astype(np.float64), gh[cy0:cy1, cx0:cx1].astype(np.float64), prm)
        np.testing.assert_allclose(oh[y0:y1, x0:x1], ref[y0 - cy0:y1 - cy0, x0 - cx0:x1 - cx0], rtol=2e-5, atol=1e-6)


def test_denoise_bad_arguments_refused():
    torch = need_cuda()
    c = ctx()
    I = torch.rand((8, 8, 3), device="cuda")
    guide = torch.zeros((8, 8, 8), device="cuda")
    for bad in (dict(radius=9, sigma_s=1.0), dict(radius=2, sigma_s=0.0), dict(radius=-1, sigma_s=1.0)):
        with pytest.raises(dpcs.DPCSError) as e:
            c.denoise(I, guide, dpcs.make_denoise_params(**bad))
        assert e.value.status == dpcs.DPCS_ERR_INVALID_ARG
    raw = torch.zeros(8 * 8 * 8 + 1, device="cuda")
    misaligned = raw[1:].view(8, 8, 8)  # 4-byte offset
    with pytest.raises(dpcs.DPCSError) as e:
        c.denoise(I, misaligned, dpcs.make_denoise_params())
    assert e.value.status == dpcs.DPCS_ERR_INVALID_ARG
    out, wsum = c.denoise(I, guide, dpcs.make_denoise_params(radius=1))  # the context still works
    c.sync()
    assert torch.isfinite(out).all()


def test_denoised_compensation_gradient_matches_oracle(orc):
    """Loss on D(Ic): dIp = replay(D^T(dL/dD)) on the GPU against the same
    chain in the oracle, on the same paths."""
    torch = need_cuda()
    sc = scenes.corner(res=24, tex=32, spp=4, bounces=2, seed=5)
    prm = PRMS[2]
    g = GpuScene(sc)
    rng = np.random.default_rng(6)
    W = rng.normal(size=(sc.Hc, sc.Wc, 3)).astype(np.float32)  # dL/dD(Ic)
    rg = orc.gbuffer(sc)  # one guide for both sides: the guide itself is tested above
    try:
        Ec, Ic = g.render()
        guide = torch.from_numpy(rg.astype(np.float32)).cuda()
        _, wsum = g.ctx.denoise(Ic, guide, _dp(prm))
        dIc = g.ctx.denoise_backward(torch.from_numpy(W).cuda(), guide, wsum, _dp(prm))
        dIp = torch.zeros_like(g.Ip)
        g.ctx.render_backward(g.handle, g.albedo, g.rough, g.Ip, g.view, g.params, sc.spp, sc.bounces, sc.seed, Ec,
                              Ic, dIc, dIp=dIp)
        g.ctx.sync()
        gdIp = dIp.cpu().numpy()
    finally:
        g.close()
    rdIc = orc.denoise_backward(W.astype(np.float64), rg.astype(np.float32).astype(np.float64), prm)
    ref = orc.render_backward(sc, rdIc)["dIp"]
    scale = np.abs(ref).max()
    assert scale > 0
    np.testing.assert_allclose(gdIp, ref, rtol=1e-3, atol=1e-4 * scale)
