"""The work counters of the DPCS_COUNTERS build (the algorithmic units the
rooflines count, and the two SIMT-efficiency counts): consistent with one
another and with the workload, and the counted render equals the normal
build's image bit for bit."""
import numpy as np
import pytest

from paper_2503_12174_gb300 import dpcs, scenes
from gpu_util import GpuScene, need_cuda

pytestmark = pytest.mark.gpu


def test_counters_are_consistent():
    torch = need_cuda()
    sc = scenes.corner(res=48, tex=32, spp=8, bounces=3, seed=2)
    c = dpcs.Context(0, lib=dpcs.counters_library())
    dev = c.device
    h = c.upload(sc.verts, sc.tris, sc.uv)
    try:
        alb, rough = torch.from_numpy(sc.albedo).to(dev), torch.from_numpy(sc.rough).to(dev)
        Ip = torch.from_numpy(sc.Ip).to(dev)
        view, prm = dpcs.view_of(sc), dpcs.make_params(sc.params)
        c.counters(reset=True)
        Ic, _ = c.render(h, alb, rough, Ip, view, prm, sc.spp, sc.bounces, sc.seed)
        n = c.counters(reset=True)
        c.sync()
        Ic = Ic.cpu().numpy()
    finally:
        c.free(h)
        c.close()
    assert n["paths"] == sc.Hc * sc.Wc * sc.spp
    assert n["rays"] >= n["paths"] and n["vertices"] <= n["rays"]
    assert n["lit"] <= n["shadow_rays"] <= n["vertices"]
    assert n["continuations"] <= n["vertices"]
    assert n["rays"] == n["paths"] + n["continuations"]  # every continuation traces one extension ray
    steps = n["node_visits"] + n["tri_tests"]
    # a warp iteration of the traversal loop does between 1 and 32 lanes' steps
    assert steps / 32 <= n["trav_warp_iters"] <= steps
    assert (n["rays"] + n["shadow_rays"]) / 32 <= n["path_warp_iters"]
    g = GpuScene(sc)
    try:
        _, Ic_ref = g.render()
    finally:
        g.close()
    np.testing.assert_array_equal(Ic, Ic_ref.cpu().numpy())
