"""dpcs_render_noalloc: the render entry point for callers that cannot
allocate device memory when they render (code recording a CUDA stream
capture, programs with a fixed up-front GPU memory budget, real-time loops).

It must produce what dpcs_render produces, call after call, without growing
the context's memory, and must refuse problem sizes beyond its fixed 8 MiB
scratch.  This file is collected last so that a run stopping at its first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_2503_12174_gb300 import dpcs, scenes

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    return torch


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_render_noalloc_matches_render_on_two_calls():
    torch = _torch()
    lib = dpcs.load_library()
    ctx = dpcs.Context(0)
    dev = ctx.device
    sc = scenes.corner(res=64, tex=64, spp=8, bounces=3, seed=11)
    h = ctx.upload(sc.verts, sc.tris, sc.uv)
    alb = torch.from_numpy(sc.albedo).to(dev)
    rough = torch.from_numpy(sc.rough).to(dev)
    view, prm = dpcs.view_of(sc), dpcs.make_params(sc.params)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(0)
    try:
        for call in range(2):  # two calls in a row, different projector images
            Ip = torch.from_numpy(rng.random(sc.Ip.shape, dtype=np.float32)).to(dev)
            Ic_ref, Ec_ref = torch.empty((sc.Hc, sc.Wc, 3), device=dev), torch.empty((sc.Hc, sc.Wc, 3), device=dev)
            ctx.render(h, alb, rough, Ip, view, prm, sc.spp, sc.bounces, sc.seed, Ic=Ic_ref, Ec=Ec_ref)
            ctx.sync()
            used = ctx.memory_used
            Ic = torch.full((sc.Hc, sc.Wc, 3), float("nan"), device=dev)
            Ec = torch.full((sc.Hc, sc.Wc, 3), float("nan"), device=dev)
            st = lib.dpcs_render_noalloc(ctx.handle, h, _p(alb), _p(rough), sc.Ht, sc.Wt, _p(Ip),
                                         ctypes.byref(view), ctypes.byref(prm), sc.spp, sc.bounces, sc.seed, _p(Ic),
                                         _p(Ec), stream)
            assert st == dpcs.DPCS_OK, dpcs.dpcs_last_error(ctx.handle)
            ctx.sync()
            assert ctx.memory_used == used  # nothing was allocated
            g, r = Ic.cpu().numpy().astype(np.float64), Ic_ref.cpu().numpy().astype(np.float64)
            assert np.isfinite(g).all() and np.abs(r).max() > 0
            np.testing.assert_allclose(g, r, rtol=1e-4, atol=1e-7)
            np.testing.assert_allclose(Ec.cpu().numpy(), Ec_ref.cpu().numpy(), rtol=1e-4, atol=1e-7)
    finally:
        ctx.free(h)
        ctx.close()


def test_render_noalloc_rejects_oversized_problems():
    torch = _torch()
    lib = dpcs.load_library()
    ctx = dpcs.Context(0)
    dev = ctx.device
    sc = scenes.corner(res=32, tex=32, spp=2, bounces=2)
    h = ctx.upload(sc.verts, sc.tris, sc.uv)
    try:
        big = sc.replace(Ip=np.zeros((768, 700, 3), np.float32))  # 537,600 + 1,024 texels > 524,288
        view, prm = dpcs.view_of(big), dpcs.make_params(big.params)
        alb = torch.from_numpy(big.albedo).to(dev)
        rough = torch.from_numpy(big.rough).to(dev)
        Ip = torch.from_numpy(big.Ip).to(dev)
        Ic = torch.zeros((big.Hc, big.Wc, 3), device=dev)
        st = lib.dpcs_render_noalloc(ctx.handle, h, _p(alb), _p(rough), big.Ht, big.Wt, _p(Ip), ctypes.byref(view),
                                     ctypes.byref(prm), big.spp, big.bounces, big.seed, _p(Ic), None,
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == dpcs.DPCS_ERR_INVALID_ARG
        assert "524288" in dpcs.dpcs_last_error(ctx.handle)
        ctx.sync()
        assert not Ic.any()
    finally:
        ctx.free(h)
        ctx.close()
