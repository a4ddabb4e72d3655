"""dpcs_render_noalloc: the render entry point for callers that cannot
allocate device memory when they render (host programs that give the GPU a
fixed memory budget up front and own every allocation in it, real-time loops
that cannot absorb an allocation's latency or failure mid-frame).

It must produce what dpcs_render produces, bit for bit, call after call,
without allocating anything, and must refuse problem sizes beyond its fixed
8 MiB scratch (524,288 texels of projector image plus textures).  This file
is collected last so that a run stopping at its first failure has already
run every other test; each test makes its own context, so it also passes
alone in a fresh process."""
import ctypes

import numpy as np
import pytest

from paper_2503_12174_gb300 import dpcs, scenes

pytestmark = pytest.mark.gpu

LIMIT = 524288  # texels of the library's fixed scratch (Hp*Wp + Ht*Wt)


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    return torch


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _noalloc(lib, ctx, h, sc, alb, rough, Ip, Ic, Ec):
    torch = _torch()
    view, prm = dpcs.view_of(sc), dpcs.make_params(sc.params)
    return lib.dpcs_render_noalloc(ctx.handle, h, _p(alb), _p(rough), sc.Ht, sc.Wt, _p(Ip), ctypes.byref(view),
                                   ctypes.byref(prm), sc.spp, sc.bounces, sc.seed, _p(Ic), _p(Ec),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_render_noalloc_matches_render_on_two_calls():
    """On a fresh context, before any dpcs_render: two calls in a row with
    different projector images leave the context's memory and the device's
    free memory unchanged, and each equals dpcs_render bit for bit."""
    torch = _torch()
    lib = dpcs.load_library()
    ctx = dpcs.Context(0)
    dev = ctx.device
    sc = scenes.corner(res=64, tex=64, spp=8, bounces=3, seed=11)
    h = ctx.upload(sc.verts, sc.tris, sc.uv)
    alb = torch.from_numpy(sc.albedo).to(dev)
    rough = torch.from_numpy(sc.rough).to(dev)
    rng = np.random.default_rng(0)
    Ips = [torch.from_numpy(rng.random(sc.Ip.shape, dtype=np.float32)).to(dev) for _ in range(2)]
    outs = [(torch.full((sc.Hc, sc.Wc, 3), float("nan"), device=dev),
             torch.full((sc.Hc, sc.Wc, 3), float("nan"), device=dev)) for _ in range(2)]
    try:
        ctx.sync()
        torch.cuda.synchronize()
        used0 = ctx.memory_used
        free = []
        for call in range(2):
            st = _noalloc(lib, ctx, h, sc, alb, rough, Ips[call], *outs[call])
            assert st == dpcs.DPCS_OK, dpcs.dpcs_last_error(ctx.handle)
            ctx.sync()
            assert ctx.memory_used == used0  # the context allocated nothing
            free.append(torch.cuda.mem_get_info(dev)[0])
        # the first call may load the library's module (and with it the
        # fixed array); the second call must not change free device memory
        assert free[1] == free[0]
        for call in range(2):
            Ec_ref = torch.empty_like(outs[call][1])
            Ic_ref, _ = ctx.render(h, alb, rough, Ips[call], dpcs.view_of(sc), dpcs.make_params(sc.params), sc.spp,
                                   sc.bounces, sc.seed, Ec=Ec_ref)
            ctx.sync()
            Ic, Ec = outs[call]
            assert torch.isfinite(Ic).all() and Ic_ref.abs().max() > 0
            assert torch.equal(Ic, Ic_ref)
            assert torch.equal(Ec, Ec_ref)
    finally:
        ctx.free(h)
        ctx.close()


def test_render_noalloc_at_exactly_the_limit():
    """Hp*Wp + Ht*Wt == 524,288 (a 512 x 1022 projector and 32 x 32 textures)
    is accepted and renders what dpcs_render renders; one texel more is
    refused before anything is launched."""
    torch = _torch()
    lib = dpcs.load_library()
    ctx = dpcs.Context(0)
    dev = ctx.device
    rng = np.random.default_rng(4)
    base = scenes.corner(res=48, tex=32, spp=4, bounces=3, seed=5)
    sc = base.replace(Ip=scenes.blob_image(rng, 512, 1022).astype(np.float32),
                      Kp=scenes.intrinsics(1022, 512, 45.0))
    assert sc.Hp * sc.Wp + sc.Ht * sc.Wt == LIMIT
    h = ctx.upload(sc.verts, sc.tris, sc.uv)
    try:
        alb = torch.from_numpy(sc.albedo).to(dev)
        rough = torch.from_numpy(sc.rough).to(dev)
        Ip = torch.from_numpy(sc.Ip).to(dev)
        Ic = torch.full((sc.Hc, sc.Wc, 3), float("nan"), device=dev)
        Ec = torch.full_like(Ic, float("nan"))
        for _ in range(2):
            st = _noalloc(lib, ctx, h, sc, alb, rough, Ip, Ic, Ec)
            assert st == dpcs.DPCS_OK, dpcs.dpcs_last_error(ctx.handle)
            ctx.sync()
            Ec_ref = torch.empty_like(Ec)
            Ic_ref, _ = ctx.render(h, alb, rough, Ip, dpcs.view_of(sc), dpcs.make_params(sc.params), sc.spp,
                                   sc.bounces, sc.seed, Ec=Ec_ref)
            ctx.sync()
            assert Ic_ref.abs().max() > 0
            assert torch.equal(Ic, Ic_ref) and torch.equal(Ec, Ec_ref)
        # one texel over: textures of 25 x 41 = 1025 texels
        over = sc.replace(albedo=np.full((25, 41, 3), 0.5, np.float32), rough=np.full((25, 41), 0.3, np.float32))
        assert over.Hp * over.Wp + over.Ht * over.Wt == LIMIT + 1
        Ic2 = torch.zeros_like(Ic)
        st = _noalloc(lib, ctx, h, over, torch.from_numpy(over.albedo).to(dev), torch.from_numpy(over.rough).to(dev),
                      Ip, Ic2, None)
        assert st == dpcs.DPCS_ERR_INVALID_ARG
        assert "524288" in dpcs.dpcs_last_error(ctx.handle)
        ctx.sync()
        assert not Ic2.any()
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
        alb = torch.from_numpy(big.albedo).to(dev)
        rough = torch.from_numpy(big.rough).to(dev)
        Ip = torch.from_numpy(big.Ip).to(dev)
        Ic = torch.zeros((big.Hc, big.Wc, 3), device=dev)
        st = _noalloc(lib, ctx, h, big, alb, rough, Ip, Ic, None)
        assert st == dpcs.DPCS_ERR_INVALID_ARG
        assert "524288" in dpcs.dpcs_last_error(ctx.handle)
        ctx.sync()
        assert not Ic.any()
    finally:
        ctx.free(h)
        ctx.close()
