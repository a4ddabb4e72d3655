"""The wavefront render (DPCS_PATH_WAVEFRONT: trace and shade passes over
compacted path queues) traces the same paths as the megakernel with the same
per-vertex functions and the same summation order; only the compiler's
contraction of a few products can differ between the two kernels, by an ulp.
Each image is held to the oracle at the image gate and to the megakernel's
image at 1e-5 -- on ragged sizes, spp that the lanes per pixel do not divide,
Russian roulette, the longest paths, several chunk sizes and the degenerate
cases."""
import numpy as np
import pytest

from paper_2503_12174_gb300 import dpcs, scenes
from gpu_util import GpuScene, crf_atol, need_cuda, pixel_parity

pytestmark = pytest.mark.gpu


def _both(sc, chunk=0):
    g = GpuScene(sc)
    try:
        g.ctx.set_render_path(dpcs.DPCS_PATH_MEGAKERNEL)
        Em, Im = g.render()
        g.ctx.set_render_path(dpcs.DPCS_PATH_WAVEFRONT, chunk)
        try:
            Ew, Iw = g.render()
            Ew2, Iw2 = g.render()
        finally:
            g.ctx.set_render_path(dpcs.DPCS_PATH_MEGAKERNEL, 1 << 20)
        g.ctx.sync()
    finally:
        g.close()
    assert np.array_equal(Ew.cpu().numpy(), Ew2.cpu().numpy())  # deterministic
    return (Em.cpu().numpy(), Im.cpu().numpy()), (Ew.cpu().numpy(), Iw.cpu().numpy())


def _case(case):
    chunk = 0
    if case == "corner_ragged":
        sc = scenes.corner(res=29, tex=32, spp=7, bounces=3, seed=4).replace(Hc=29, Wc=37)
    elif case == "corner_7spp_chunks":
        sc = scenes.corner(res=64, tex=64, spp=7, bounces=3, seed=5)
        chunk = 4096  # many chunks, the last one partial
    elif case == "plane":
        sc = scenes.plane(res=64, spp=4)
    elif case == "heightfield_rr":
        sc = scenes.heightfield(spp=6, cam=48, proj=(40, 52), tex=64, n_vert=65)
    elif case == "sphere_8":
        sc = scenes.sphere(subdiv=3, res=24, spp=5, bounces=dpcs.DPCS_MAX_BOUNCES)
    elif case == "clip":
        p = scenes.corner(res=32).params
        sc = scenes.corner(res=32, tex=32, spp=3, bounces=4, seed=6).replace(
            params=scenes.Params(gamma_p=p.gamma_p, gain_p=p.gain_p, gamma_c=p.gamma_c, gain_c=p.gain_c, wb=p.wb,
                                 k_proj=p.k_proj, ks=p.ks, f0=p.f0, clip=0.02))
    elif case == "bounces0":
        sc = scenes.corner(res=16, tex=16, spp=4, bounces=0)
    else:
        sc = scenes.corner(res=40, tex=32, spp=1, bounces=3, seed=9)
    return sc, chunk


@pytest.mark.parametrize("case", ["corner_ragged", "corner_7spp_chunks", "plane", "heightfield_rr", "sphere_8",
                                  "clip", "bounces0", "spp1"])
def test_wavefront_matches_oracle_and_megakernel(orc, case):
    need_cuda()
    sc, chunk = _case(case)
    (Em, Im), (Ew, Iw) = _both(sc, chunk)
    if case == "bounces0":
        assert not Ew.any() and not Iw.any()
        return
    assert np.abs(Ew).max() > 0
    rE, rI = orc.render(sc, accel=True)
    ok, info = pixel_parity(Ew, rE)
    assert ok, info
    ok, info = pixel_parity(Iw, rI, atol=crf_atol(sc, rE))
    assert ok, info
    ok, info = pixel_parity(Ew, Em, rtol=1e-5, atol=1e-9, mean_rtol=1e-6)
    assert ok, info


def test_wavefront_matches_megakernel_on_the_benchmark_workload():
    """The forward workload the benchmark times (corner 256^2, 64 spp, 3
    bounces), with the default chunk and with one chunk per wave."""
    need_cuda()
    sc = scenes.corner(res=256, spp=64, bounces=3, seed=1000)
    for chunk in (0, 1 << 21):
        (Em, Im), (Ew, Iw) = _both(sc, chunk)
        ok, info = pixel_parity(Ew, Em, rtol=1e-5, atol=1e-9, mean_rtol=1e-6)
        assert ok, info


def test_wavefront_bad_options_refused():
    need_cuda()
    from gpu_util import ctx

    c = ctx()
    for path, chunk in ((2, 0), (1, 100), (1, 4097), (1, 1 << 29)):
        with pytest.raises(dpcs.DPCSError):
            c.set_render_path(path, chunk)
    c.set_render_path(dpcs.DPCS_PATH_MEGAKERNEL, 1 << 20)
