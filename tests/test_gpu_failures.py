"""Failure paths on the GPU, none of which faults or hangs it: the traversal
cap is reached on purpose and reported by dpcs_sync; bad arguments are
refused on the host before any launch; the context keeps working."""
import ctypes

import numpy as np
import pytest

from paper_2503_12174_gb300 import dpcs, scenes
from gpu_util import GpuScene, ctx, need_cuda

pytestmark = pytest.mark.gpu


def test_traversal_cap_reported_and_recovered():
    torch = need_cuda()
    sc = scenes.corner(res=24, spp=2, bounces=2)
    g = GpuScene(sc)
    try:
        g.ctx.set_visit_cap(3)  # far below what any ray through this tree needs
        Ic = torch.empty((sc.Hc, sc.Wc, 3), device="cuda")
        g.ctx.render(g.handle, g.albedo, g.rough, g.Ip, g.view, g.params, sc.spp, sc.bounces, sc.seed, Ic=Ic)
        with pytest.raises(dpcs.DPCSError) as e:
            g.ctx.sync()
        assert e.value.status == dpcs.DPCS_ERR_TRAVERSAL_LIMIT
        assert torch.isfinite(Ic).all()
        g.ctx.set_visit_cap(0)
        g.ctx.sync()  # the status word was cleared by the failing sync
        Ec, Ic2 = g.render()  # renders normally again
        assert Ic2.abs().sum().item() > 0
    finally:
        g.ctx.set_visit_cap(0)
        g.close()


def test_bad_arguments_refused_before_launch():
    torch = need_cuda()
    c = ctx()
    sc = scenes.corner(res=16, spp=2)
    g = GpuScene(sc)
    try:
        n0 = c.launch_count
        Ic = torch.empty((sc.Hc, sc.Wc, 3), device="cuda")
        for kw, status in [({"bounces": 9}, dpcs.DPCS_ERR_INVALID_ARG), ({"spp": 0}, dpcs.DPCS_ERR_INVALID_ARG),
                           ({"scene": 987654}, dpcs.DPCS_ERR_NOT_FOUND)]:
            with pytest.raises(dpcs.DPCSError) as e:
                c.render(kw.get("scene", g.handle), g.albedo, g.rough, g.Ip, g.view, g.params, kw.get("spp", 2),
                         kw.get("bounces", 2), 0, Ic=Ic)
            assert e.value.status == status
        bad = dpcs.view_of(sc)
        bad.Kc[0] = float("nan")
        with pytest.raises(dpcs.DPCSError) as e:
            c.render(g.handle, g.albedo, g.rough, g.Ip, bad, g.params, 2, 2, 0, Ic=Ic)
        assert e.value.status == dpcs.DPCS_ERR_INVALID_ARG
        with pytest.raises(dpcs.DPCSError) as e:  # triangle index out of range
            c.upload(sc.verts, np.array([[0, 1, len(sc.verts)]], np.int32), sc.uv)
        assert e.value.status == dpcs.DPCS_ERR_INVALID_ARG
        assert c.launch_count == n0  # nothing reached the GPU
        c.sync()
        Ec, Ic2 = g.render()
        assert torch.isfinite(Ic2).all()
    finally:
        g.close()


def test_hbm_budget_refuses_scratch():
    torch = need_cuda()
    small = dpcs.Context(0, hbm_budget_bytes=1 << 16)  # room for the status words, not a scene
    sc = scenes.corner(res=16, spp=2)
    with pytest.raises(dpcs.DPCSError) as e:
        small.upload(sc.verts, sc.tris, sc.uv)
    assert e.value.status == dpcs.DPCS_ERR_OOM
    small.close()


def test_bounds_checked_build_renders_the_same_image():
    """The DPCS_CHECK debug build checks every tree reference before reading
    it; on a correct tree it reports nothing and renders the image of the
    normal build bit for bit."""
    torch = need_cuda()
    from gpu_util import GpuScene

    sc = scenes.corner(res=32, tex=16, spp=8, bounces=3)
    g = GpuScene(sc)
    try:
        _, Ic = g.render()
        ref = Ic.cpu().numpy()
    finally:
        g.close()
    c = dpcs.Context(0, lib=dpcs.check_library())
    try:
        h = c.upload(sc.verts, sc.tris, sc.uv)
        dev = c.device
        alb, rough, Ip = (torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (sc.albedo, sc.rough, sc.Ip))
        Ic2, _ = c.render(h, alb, rough, Ip, dpcs.view_of(sc), dpcs.make_params(sc.params), sc.spp, sc.bounces, sc.seed)
        c.sync()  # raises if a check fired
        np.testing.assert_array_equal(Ic2.cpu().numpy(), ref)
        c.free(h)
    finally:
        c.close()
