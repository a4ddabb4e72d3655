"""Host side of the serving workload, on the CPU: the seeded request stream
has the stated mix (Poisson arrivals, 90 % relighting / 10 % compensation of
50 steps at 16 spp, camera sides 128..1024, spp log-uniform in [16, 256],
three resident scenes), and a request's view keeps the scene's field of view."""
import math

import numpy as np
import pytest

from paper_2503_12174_gb300 import dpcs, scenes, serving


def test_workload_mix_and_arrivals():
    stats = pytest.importorskip("scipy.stats")
    n, rate = 2000, 8.0
    wl = serving.make_workload(n, rate=rate, seed=100)
    assert len(wl) == n
    assert wl == serving.make_workload(n, rate=rate, seed=100)  # seeded
    t = np.array([r.t_arrival for r in wl])
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0.0)
    gaps = np.diff(t)
    # exponential gaps of mean 1 / rate
    assert abs(gaps.mean() * rate - 1.0) < 4.0 / math.sqrt(gaps.size)
    assert stats.kstest(gaps * rate, "expon").pvalue > 1e-3
    comp = np.array([r.kind == dpcs.DPCS_REQ_COMPENSATE for r in wl])
    assert abs(comp.mean() - 0.1) < 4.0 * math.sqrt(0.1 * 0.9 / n)
    for r in wl:
        assert r.side in serving.SIDES and 0 <= r.scene < 3
        if r.kind == dpcs.DPCS_REQ_COMPENSATE:
            assert (r.steps, r.spp) == (50, 16)
        else:
            assert r.kind == dpcs.DPCS_REQ_RELIGHT and r.steps == 0 and 16 <= r.spp <= 256
    relight_spp = np.array([r.spp for r in wl if r.kind == dpcs.DPCS_REQ_RELIGHT], np.float64)
    u = (np.log(relight_spp) - math.log(16)) / (math.log(256) - math.log(16))  # ~ U[0, 1] up to rounding of spp
    assert abs(u.mean() - 0.5) < 4.0 * math.sqrt(1 / 12 / u.size) + 0.01
    assert serving.SIDES[0] == 128 and serving.SIDES[-1] == 1024
    sides = np.array([r.side for r in wl])
    assert len(np.unique(sides)) == len(serving.SIDES)
    counts = np.bincount([r.scene for r in wl], minlength=3)
    assert np.all(np.abs(counts / n - 1 / 3) < 4.0 * math.sqrt(2 / 9 / n))


def test_workload_at_rate_zero_arrives_at_once():
    wl = serving.make_workload(50, rate=0.0, seed=3)
    assert all(r.t_arrival == 0.0 for r in wl)
    assert serving.make_workload(0, rate=5.0) == []


def test_request_view_keeps_the_field_of_view():
    sc = scenes.corner(res=256, spp=4, bounces=1)
    for side in (128, 384, 1024):
        v = serving.request_view(sc, side)
        Kc = np.array(v.Kc, np.float64).reshape(3, 3)
        K0 = np.asarray(sc.Kc, np.float64)
        assert (v.Hc, v.Wc) == (side, side) and (v.Hp, v.Wp) == (sc.Hp, sc.Wp)
        # the same rays through the same relative image positions
        np.testing.assert_allclose(Kc[:2] / side, K0[:2] / 256, rtol=1e-6)
        np.testing.assert_array_equal(Kc[2], K0[2])
        np.testing.assert_array_equal(np.array(v.Kp, np.float32), np.asarray(sc.Kp, np.float32).ravel())


class _FakeServeLib:
    """Stands in for libdpcs's serving entry points: records the requests it
    is given and refuses an unknown scene slot as the library does."""

    def __init__(self):
        self.requests = []

    def dpcs_serve_create(self, ctx, cfg, out):
        return dpcs.DPCS_OK

    def dpcs_serve_destroy(self, h):
        return dpcs.DPCS_OK

    def dpcs_serve_add_scene(self, h, scene, alb, rough, Ht, Wt, view, params, bounces, slot):
        slot._obj.value = 0
        return dpcs.DPCS_OK

    def dpcs_serve_submit(self, h, req, rid):
        r = req._obj
        self.requests.append((r.scene, r.Hc, r.Wc, r.Ip, r.Ic_out, r.target, r.Ip_out))
        if r.scene != 0:
            return dpcs.DPCS_ERR_NOT_FOUND
        rid._obj.value = len(self.requests)
        return dpcs.DPCS_OK


class _FakeCtx:
    def __init__(self):
        import torch

        self.lib = _FakeServeLib()
        self.handle = None
        self.device = torch.device("cpu")

    def check(self, status, what):
        if status != dpcs.DPCS_OK:
            raise dpcs.DPCSError(status, what)


def test_submit_checks_host_buffer_sizes():
    """The server copies whole images to and from the request's host
    buffers, which the library cannot check: the binding refuses a buffer of
    the wrong size, type or layout before the library sees the request."""
    torch = pytest.importorskip("torch")
    ctx = _FakeCtx()
    srv = dpcs.Server(ctx)
    view = dpcs.DpcsView()
    view.Hc, view.Wc, view.Hp, view.Wp = 32, 32, 20, 24
    slot = srv.add_scene(1, torch.zeros((4, 4, 3)), torch.zeros((4, 4)), view, dpcs.DpcsParams(), 2)
    Ip = torch.zeros((20, 24, 3))
    Ic = torch.zeros((16, 12, 3))
    rid = srv.submit(dpcs.DPCS_REQ_RELIGHT, slot, 16, 12, 8, 1, Ip, Ic)
    assert rid == 1 and ctx.lib.requests[-1][3] == Ip.data_ptr() and ctx.lib.requests[-1][4] == Ic.data_ptr()
    tgt, Ipo = np.zeros((16, 12, 3), np.float32), np.zeros((20, 24, 3), np.float32)
    srv.submit(dpcs.DPCS_REQ_COMPENSATE, slot, 16, 12, 8, 1, Ip, Ic, target=tgt, Ip_out=Ipo, steps=2)
    assert ctx.lib.requests[-1][5] == tgt.ctypes.data and ctx.lib.requests[-1][6] == Ipo.ctypes.data
    bad = [
        dict(Ip=torch.zeros((20, 23, 3))),                        # projector image of another size
        dict(Ic_out=torch.zeros((16, 11, 3))),                    # result buffer too small
        dict(Ic_out=torch.zeros((16, 12, 3), dtype=torch.float64)),
        dict(Ic_out=torch.zeros((12, 16, 3)).transpose(0, 1)),    # not contiguous
        dict(target=np.zeros((16, 12, 2), np.float32)),
        dict(Ip_out=np.zeros((20, 24, 3), np.float64)),
        dict(Ip=[0.0] * (20 * 24 * 3)),                           # not an array the request can point into
    ]
    n = len(ctx.lib.requests)
    for kw in bad:
        args = dict(Ip=Ip, Ic_out=Ic, target=tgt, Ip_out=Ipo)
        args.update(kw)
        with pytest.raises(ValueError):
            srv.submit(dpcs.DPCS_REQ_COMPENSATE, slot, 16, 12, 8, 1, args["Ip"], args["Ic_out"],
                       target=args["target"], Ip_out=args["Ip_out"], steps=2)
    assert len(ctx.lib.requests) == n  # none of them reached the library
    # sizes and scenes the library refuses itself are passed on to it
    with pytest.raises(dpcs.DPCSError) as e:
        srv.submit(dpcs.DPCS_REQ_RELIGHT, 5, 16, 12, 8, 1, Ip, Ic)
    assert e.value.status == dpcs.DPCS_ERR_NOT_FOUND
    srv.submit(dpcs.DPCS_REQ_RELIGHT, slot, 0, 12, 8, 1, Ip, Ic)
    assert ctx.lib.requests[-1][1] == 0
    srv.close()
