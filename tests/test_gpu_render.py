"""Forward parity: GPU render (FP32) vs the FP64 oracle on the same Philox
stream.  Gate: |g - r| <= 1e-4 |r| + 1e-7 per channel on >= 99.9 % of the
pixels and the image mean within 1e-5 (relative)."""
import numpy as np
import pytest

from paper_2503_12174_gb300 import scenes
from gpu_util import GpuScene, crf_atol, need_cuda, pixel_parity

pytestmark = pytest.mark.gpu


def _ragged(sc, H, W):
    return sc.replace(Hc=H, Wc=W, Kc=scenes.intrinsics(W, H, 40.0))


def _check(orc, sc, pixels=None, spp=None):
    g = GpuScene(sc)
    try:
        Ec, Ic = g.render(spp=spp)
        Ec, Ic = Ec.cpu().numpy(), Ic.cpu().numpy()
        Ec2, Ic2 = g.render(spp=spp)
        np.testing.assert_array_equal(Ic, Ic2.cpu().numpy())  # deterministic
    finally:
        g.close()
    rE, rI = orc.render(sc, pixels=pixels, spp=spp)
    if pixels is not None:
        Ec, Ic = Ec.reshape(-1, 3)[pixels], Ic.reshape(-1, 3)[pixels]
    ok, info = pixel_parity(Ec, rE)
    assert ok, ("Ec", info)
    ok, info = pixel_parity(Ic, rI, atol=crf_atol(sc, rE))
    assert ok, ("Ic", info)
    assert np.abs(rE).max() > 0
    return info


def test_plane_direct_light_config(orc):
    _check(orc, scenes.plane())


def test_corner_ragged_multi_bounce(orc):
    _check(orc, _ragged(scenes.corner(res=64, spp=7, bounces=3), 29, 37))


def test_corner_clip_and_single_sample(orc):
    sc = scenes.corner(res=48, spp=1, bounces=4)
    p = sc.params
    sc = sc.replace(params=scenes.Params(gamma_p=p.gamma_p, gamma_c=p.gamma_c, gain_c=p.gain_c, wb=p.wb,
                                         k_proj=p.k_proj, ks=p.ks, f0=p.f0, clip=0.05))
    _check(orc, _ragged(sc, 33, 50))


def test_heightfield_russian_roulette(orc):
    sc = scenes.heightfield(spp=4, cam=40, proj=(48, 64), tex=64, n_vert=81)
    _check(orc, _ragged(sc, 33, 40))


def test_integrating_sphere(orc):
    sc = scenes.sphere(subdiv=3, res=24, spp=16, bounces=3)
    _check(orc, sc)


def test_corner_full_size_sampled_pixels(orc):
    """The benchmark's workload (256x256, 64 spp, 3 bounces) in the launch
    configuration the benchmark times, checked on 256 sampled pixels."""
    sc = scenes.corner(res=256, spp=64, bounces=3)
    px = np.random.default_rng(0).choice(sc.Hc * sc.Wc, 256, replace=False)
    _check(orc, sc, pixels=px)


def test_compensation_full_size_sampled_pixels(orc):
    sc = scenes.compensation(res=512, spp=16)
    px = np.random.default_rng(1).choice(sc.Hc * sc.Wc, 160, replace=False)
    _check(orc, sc, pixels=px)


def test_heightfield_full_size_sampled_pixels(orc):
    sc = scenes.heightfield(spp=8)
    px = np.random.default_rng(2).choice(sc.Hc * sc.Wc, 64, replace=False)
    _check(orc, sc, pixels=px)


def test_degenerate_inputs(orc):
    torch = need_cuda()
    sc = scenes.corner(res=16, spp=3)
    g = GpuScene(sc)
    try:
        Ec, Ic = g.render(bounces=0)
        assert not Ec.any() and not Ic.any()
        Ec, Ic = g.render(Ip=torch.zeros_like(g.Ip))
        assert not Ec.any()
    finally:
        g.close()
    empty = sc.replace(verts=np.zeros((0, 3), np.float32), tris=np.zeros((0, 3), np.int32),
                       uv=np.zeros((0, 2), np.float32))
    g = GpuScene(empty)
    try:
        Ec, Ic = g.render()
        assert not Ec.any()
    finally:
        g.close()


@pytest.mark.parametrize("case", ["plane", "corner_ragged", "heightfield", "corner_full_sampled"])
def test_ic_gate_as_stated(orc, case):
    """The image gate on Ic itself, with no propagated tolerance: |g - r| <=
    1e-4 |r| + 1e-7 per channel on >= 99.9 % of the pixels and the mean
    within 1e-5.  (The other tests hold Ec to this gate and Ic to the Ec gate
    carried through Eq. 5, which is looser where Ec is near 0 and gamma_c <
    1.)"""
    pixels = None
    if case == "plane":
        sc = scenes.plane()
    elif case == "corner_ragged":
        sc = _ragged(scenes.corner(res=64, spp=7, bounces=3), 29, 37)
    elif case == "heightfield":
        sc = _ragged(scenes.heightfield(spp=4, cam=40, proj=(48, 64), tex=64, n_vert=81), 33, 40)
    else:
        sc = scenes.corner(res=256, spp=64, bounces=3, seed=1000)
        pixels = np.random.default_rng(17).choice(sc.Hc * sc.Wc, 2000, replace=False)
    g = GpuScene(sc)
    try:
        _, Ic = g.render()
        Ic = Ic.cpu().numpy()
    finally:
        g.close()
    _, rI = orc.render(sc, pixels=pixels, accel=True)
    if pixels is not None:
        Ic = Ic.reshape(-1, 3)[pixels]
    ok, info = pixel_parity(Ic, rI)
    assert ok, info
