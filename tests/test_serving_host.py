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
