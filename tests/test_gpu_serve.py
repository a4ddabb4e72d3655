"""Continuous-batching server: each request's result is the same alone and
in the mix; admission never exceeds the HBM budget; bad requests are
rejected on the host."""
import ctypes

import numpy as np
import pytest

from paper_2503_12174_gb300 import dpcs, serving
from gpu_util import ctx, need_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    need_cuda()
    c = ctx()
    scs = serving.resident_scenes()
    gs = serving.GpuScenes(c, scs)
    host = serving.HostData(scs, pool=3)
    yield c, gs, host
    for h in gs.handles:
        c.free(h)


def _small_workload(n=14, steps=4):
    return serving.make_workload(n, rate=0.0, seed=3, comp_frac=0.25, comp_steps=steps, comp_spp=4,
                                 sides=(64, 96, 128), spp_range=(4, 40), pool=3)


def _check_against_alone(c, gs, host, wl, outs):
    for k, rq in enumerate(wl):
        sc = gs.scs[rq.scene]
        Ic_mix, Ip_mix = outs[k]
        if rq.kind == dpcs.DPCS_REQ_RELIGHT:
            Ip = host.ips[rq.scene][rq.ip_idx].cuda()
            Ic, _ = c.render(gs.handles[rq.scene], gs.alb[rq.scene], gs.rough[rq.scene], Ip,
                             serving.request_view(sc, rq.side), gs.params[rq.scene], rq.spp, sc.bounces, rq.seed)
            c.sync()
            np.testing.assert_array_equal(Ic_mix, Ic.cpu().numpy(), err_msg=f"relight request {k}")
        else:
            Ic, P = serving.compensate_alone(c, gs, rq.scene, rq.side, rq.spp, rq.seed, host.ips[rq.scene][rq.ip_idx],
                                             host.target(rq.scene, rq.side), rq.steps)
            c.sync()
            # gradients are summed with float atomics, so the Adam iterates agree to rounding only
            np.testing.assert_allclose(Ip_mix, P.cpu().numpy(), rtol=0, atol=2e-3, err_msg=f"compensation {k}")
            np.testing.assert_allclose(Ic_mix, Ic.cpu().numpy(), rtol=2e-3, atol=2e-4, err_msg=f"compensation {k}")


@pytest.mark.parametrize("policy", [dpcs.DPCS_SERVE_DEADLINE, dpcs.DPCS_SERVE_FIXED_SHARE,
                                    dpcs.DPCS_SERVE_QUANTA_DEADLINE])
def test_results_same_alone_and_in_mix(env, policy):
    need_cuda()
    c, gs, host = env
    wl = _small_workload()
    assert any(r.kind == dpcs.DPCS_REQ_COMPENSATE for r in wl) and any(r.kind == dpcs.DPCS_REQ_RELIGHT for r in wl)
    summary, outs = serving.run_server(c, gs, host, wl, keep_outputs=True, max_active=8, samples_per_iteration=1 << 18,
                                       quantum_samples=1 << 16, policy=policy)
    assert summary["requests"] == len(wl)
    assert summary["server"]["iterations"] > 2  # requests really were interleaved over several iterations
    _check_against_alone(c, gs, host, wl, outs)


def test_requests_admitted_while_others_run(env):
    """Continuous batching: a second wave of requests is submitted while the
    first wave's iterations are still on the GPU; the server admits them as
    slots free up, their work shares iterations with the first wave's, and
    every result equals the request run alone."""
    torch = need_cuda()
    c, gs, host = env
    wl = serving.make_workload(10, rate=0.0, seed=21, comp_frac=0.3, comp_steps=4, comp_spp=4, sides=(96, 128, 160),
                               spp_range=(8, 64), pool=3)
    assert any(r.kind == dpcs.DPCS_REQ_COMPENSATE for r in wl[5:])
    srv = dpcs.Server(c, max_active=4, max_inflight=2, samples_per_iteration=1 << 18, quantum_samples=1 << 16)
    slots = [srv.add_scene(gs.handles[i], gs.alb[i], gs.rough[i], dpcs.view_of(sc), gs.params[i], sc.bounces)
             for i, sc in enumerate(gs.scs)]
    outs = serving._result_buffers(gs, host, wl)
    ids = {}

    def submit(k):
        rq = wl[k]
        Ic, Ipo = outs[k]
        tgt = host.target(rq.scene, rq.side) if rq.kind == dpcs.DPCS_REQ_COMPENSATE else None
        ids[k] = srv.submit(rq.kind, slots[rq.scene], rq.side, rq.side, rq.spp, rq.seed, host.ips[rq.scene][rq.ip_idx],
                            Ic, target=tgt, Ip_out=Ipo, steps=rq.steps, lr=1e-2)

    try:
        for k in range(5):
            submit(k)
        srv.step()
        srv.step()
        st = srv.stats()
        assert st["active"] > 0 and st["completed"] < 5  # the first wave is still on the GPU
        for k in range(5, 10):  # the second wave arrives while the first runs
            submit(k)
        assert srv.stats()["waiting"] > 0  # more requests than slots: some wait for admission
        srv.drain(60.0)
        st = srv.stats()
        assert st["completed"] == 10 and st["failed"] == 0 and st["memory_used"] == 0
        for k in range(10):
            state, _ = srv.query(ids[k])
            assert state == dpcs.DPCS_REQ_DONE
        got = {k: (outs[k][0].numpy().copy(), None if outs[k][1] is None else outs[k][1].numpy().copy())
               for k in range(10)}
    finally:
        srv.close()
    _check_against_alone(c, gs, host, wl, got)


def test_admission_respects_hbm_budget(env):
    c, gs, host = env
    wl = serving.make_workload(24, rate=0.0, seed=9, comp_frac=0.0, sides=(128, 192, 256), spp_range=(4, 16), pool=3)
    budget = 3 * (256 * 256 * 12 + 512 * 512 * 28 + 4096)  # room for about three requests
    summary = serving.run_server(c, gs, host, wl, hbm_budget_bytes=budget, max_active=64,
                                 samples_per_iteration=1 << 20, quantum_samples=1 << 18)
    st = summary["server"]
    assert summary["requests"] == len(wl) and st["failed"] == 0
    assert 0 < st["memory_high_water"] <= budget
    assert st["memory_used"] == 0


def test_bad_requests_rejected_on_host(env):
    torch = need_cuda()
    c, gs, host = env
    srv = dpcs.Server(c, hbm_budget_bytes=1 << 20)
    sc = gs.scs[1]
    slot = srv.add_scene(gs.handles[1], gs.alb[1], gs.rough[1], dpcs.view_of(sc), gs.params[1], sc.bounces)
    Ic = torch.empty((64, 64, 3)).pin_memory()
    with pytest.raises(dpcs.DPCSError) as e:  # needs more device memory than the whole budget
        srv.submit(dpcs.DPCS_REQ_RELIGHT, slot, 1024, 1024, 16, 1, host.ips[1][0], torch.empty((1024, 1024, 3)))
    assert e.value.status == dpcs.DPCS_ERR_OOM
    with pytest.raises(dpcs.DPCSError) as e:
        srv.submit(dpcs.DPCS_REQ_RELIGHT, 7, 64, 64, 16, 1, host.ips[1][0], Ic)
    assert e.value.status == dpcs.DPCS_ERR_NOT_FOUND
    with pytest.raises(dpcs.DPCSError) as e:
        srv.submit(dpcs.DPCS_REQ_COMPENSATE, slot, 64, 64, 16, 1, host.ips[1][0], Ic)  # no target
    assert e.value.status == dpcs.DPCS_ERR_INVALID_ARG
    with pytest.raises(dpcs.DPCSError) as e:
        srv.submit(dpcs.DPCS_REQ_RELIGHT, slot, 0, 64, 16, 1, host.ips[1][0], Ic)
    assert e.value.status == dpcs.DPCS_ERR_INVALID_ARG
    assert srv.stats()["submitted"] == 0
    srv.close()
