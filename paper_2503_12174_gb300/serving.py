"""Serving workload and drivers around the native continuous-batching server.

The workload stands in for the paper's two downstream tasks under load:
ProCams relighting (Eq. 7) and projector compensation (Eq. 13).
- Requests arrive as a seeded Poisson process over three resident scenes: the
  one-quad plane, the 256x256 corner and the 512x512 corner.
- Camera sides are drawn from {128, 192, ..., 1024}; samples per pixel are
  log-uniform in [16, 256].
- 90 % of requests relight a random projector image.
- 10 % compensate a projector image towards a target: 50 forward+backward Adam
  steps at 16 spp.

``run_server`` drives ``dpcs.Server``: requests are submitted at their arrival
times and the server steps in between.  ``run_per_call`` is the plain
baseline: one synchronous library call (or compensation loop) per request,
in arrival order, on the same GPU.
"""
from __future__ import annotations

import dataclasses
import math
import time

import numpy as np

from . import dpcs, scenes

SIDES = tuple(range(128, 1025, 64))


@dataclasses.dataclass
class Request:
    t_arrival: float
    kind: int
    scene: int
    side: int
    spp: int
    seed: int
    steps: int
    ip_idx: int


def resident_scenes():
    """The three scenes kept on the device (the plane, corner and
    compensation workloads)."""
    plane = scenes.plane(res=64)
    p = plane.params
    plane = plane.replace(params=scenes.Params(gamma_p=p.gamma_p, k_proj=4.0, gain_c=2.0, ks=0.0),
                          albedo=np.full((64, 64, 3), 0.5, np.float32), bounces=1)
    return [plane, scenes.corner(res=256, spp=64, bounces=3), scenes.compensation(512, 16)]


def make_workload(n: int, rate: float, seed: int = 0, comp_frac: float = 0.1, comp_steps: int = 50,
                  comp_spp: int = 16, sides=SIDES, spp_range=(16, 256), n_scenes: int = 3, pool: int = 8):
    """n requests with Poisson arrivals at `rate` per second (rate <= 0: all at t = 0)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, n) if rate > 0 else np.zeros(n)
    t = np.cumsum(gaps) - (gaps[0] if n else 0.0)
    out = []
    lo, hi = math.log(spp_range[0]), math.log(spp_range[1])
    for i in range(n):
        comp = rng.random() < comp_frac
        spp = int(round(math.exp(rng.uniform(lo, hi))))
        out.append(Request(t_arrival=float(t[i]), kind=dpcs.DPCS_REQ_COMPENSATE if comp else dpcs.DPCS_REQ_RELIGHT,
                           scene=int(rng.integers(0, n_scenes)), side=int(rng.choice(sides)),
                           spp=comp_spp if comp else spp, seed=int(rng.integers(0, 2**62)),
                           steps=comp_steps if comp else 0, ip_idx=int(rng.integers(0, pool))))
    return out


class HostData:
    """Pinned host inputs: a pool of projector images per scene and a smooth
    target per (scene, side) for compensation."""

    def __init__(self, scs, pool: int = 8, seed: int = 7):
        import torch

        rng = np.random.default_rng(seed)
        self.ips = []
        for sc in scs:
            imgs = []
            for _ in range(pool):
                im = scenes.blob_image(rng, sc.Hp, sc.Wp)
                imgs.append(torch.from_numpy(im).pin_memory())
            self.ips.append(imgs)
        self.targets = {}

    def target(self, scene: int, side: int):
        import torch

        key = (scene, side)
        if key not in self.targets:
            y, x = np.meshgrid(np.linspace(0, 1, side), np.linspace(0, 1, side), indexing="ij")
            t = np.stack([0.4 + 0.2 * np.sin(6 * x + k) * np.cos(5 * y - k) for k in range(3)], -1)
            self.targets[key] = torch.from_numpy(t.astype(np.float32)).pin_memory()
        return self.targets[key]


def request_view(sc, side: int):
    """The scene's view at camera size side x side with the same field of view
    (the same float32 scaling the server applies)."""
    Kc = np.asarray(sc.Kc, np.float32).copy()
    sx = np.float32(side) / np.float32(sc.Wc)
    sy = np.float32(side) / np.float32(sc.Hc)
    Kc[0, :] = Kc[0, :] * sx
    Kc[1, :] = Kc[1, :] * sy
    return dpcs.make_view(Kc, side, side, sc.Kp, sc.Rp, sc.tp, sc.Hp, sc.Wp)


class GpuScenes:
    def __init__(self, ctx, scs):
        import torch

        self.scs = scs
        self.handles, self.alb, self.rough, self.params = [], [], [], []
        for sc in scs:
            self.handles.append(ctx.upload(sc.verts, sc.tris, sc.uv))
            self.alb.append(torch.from_numpy(sc.albedo).to(ctx.device))
            self.rough.append(torch.from_numpy(sc.rough).to(ctx.device))
            self.params.append(dpcs.make_params(sc.params))


def _percentiles(lat):
    if not lat:
        return None, None, None
    a = np.asarray(lat)
    return float(np.percentile(a, 50)), float(np.percentile(a, 99)), float(a.mean())


def summarize(records, wall_s):
    rel = [r["latency_ms"] for r in records if r["kind"] == dpcs.DPCS_REQ_RELIGHT]
    com = [r["latency_ms"] for r in records if r["kind"] == dpcs.DPCS_REQ_COMPENSATE]
    p50, p99, mean = _percentiles(rel)
    c50, c99, cmean = _percentiles(com)
    return {"requests": len(records), "requests_per_s": len(records) / wall_s if wall_s > 0 else None,
            "wall_s": wall_s, "relight_p50_ms": p50, "relight_p99_ms": p99, "relight_mean_ms": mean,
            "compensation_p50_ms": c50, "compensation_p99_ms": c99,
            "samples_per_s_M": sum(r["samples"] for r in records) / wall_s / 1e6 if wall_s > 0 else None}


def _samples(req):
    return req.side * req.side * req.spp * (max(req.steps, 1))


def _result_buffers(gs: GpuScenes, host: HostData, workload):
    """Pinned host buffers for every request's results (Ic, and Ip for
    compensation) and its compensation target, made before the clock starts
    so that neither way of serving pays for pinning host memory."""
    import torch

    outs = []
    for rq in workload:
        sc = gs.scs[rq.scene]
        Ic = torch.empty((rq.side, rq.side, 3), dtype=torch.float32).pin_memory()
        Ipo = None
        if rq.kind == dpcs.DPCS_REQ_COMPENSATE:
            Ipo = torch.empty((sc.Hp, sc.Wp, 3), dtype=torch.float32).pin_memory()
            host.target(rq.scene, rq.side)
        outs.append((Ic, Ipo))
    return outs


def run_server(ctx, gs: GpuScenes, host: HostData, workload, keep_outputs=False, **server_kw):
    """Drive the native server with the workload.  Latency of a request = its
    queueing delay before submission + the server's submit-to-result time."""
    import torch

    srv = dpcs.Server(ctx, **server_kw)
    slots = [srv.add_scene(gs.handles[i], gs.alb[i], gs.rough[i], dpcs.view_of(sc), gs.params[i], sc.bounces)
             for i, sc in enumerate(gs.scs)]
    torch.cuda.synchronize()
    n = len(workload)
    pending = {}
    records = []
    outputs = {}
    outs = _result_buffers(gs, host, workload)
    i = 0
    t0 = time.perf_counter()
    while i < n or pending:
        now = time.perf_counter() - t0
        while i < n and workload[i].t_arrival <= now:
            rq = workload[i]
            Ic, Ipo = outs[i]
            tgt = host.target(rq.scene, rq.side) if rq.kind == dpcs.DPCS_REQ_COMPENSATE else None
            rid = srv.submit(rq.kind, slots[rq.scene], rq.side, rq.side, rq.spp, rq.seed, host.ips[rq.scene][rq.ip_idx],
                             Ic, target=tgt, Ip_out=Ipo, steps=rq.steps, lr=1e-2)
            pending[rid] = (i, time.perf_counter() - t0 - rq.t_arrival, Ic, Ipo)
            i += 1
        done = srv.step()
        for rid in list(pending):
            st, lat = srv.query(rid)
            if st == dpcs.DPCS_REQ_DONE:
                k, late, Ic, Ipo = pending.pop(rid)
                rq = workload[k]
                records.append({"idx": k, "kind": rq.kind, "latency_ms": lat + late * 1e3, "samples": _samples(rq)})
                if keep_outputs:
                    outputs[k] = (Ic.numpy().copy(), None if Ipo is None else Ipo.numpy().copy())
            elif st == dpcs.DPCS_REQ_FAILED:
                raise RuntimeError(f"request {rid} failed")
        if not done and not pending and i < n:
            time.sleep(max(0.0, min(0.002, workload[i].t_arrival - (time.perf_counter() - t0))))
    wall = time.perf_counter() - t0
    stats = srv.stats()
    srv.close()
    out = summarize(records, wall)
    out["server"] = stats
    return (out, outputs) if keep_outputs else out


def compensate_alone(ctx, gs: GpuScenes, scene: int, side: int, spp: int, seed: int, Ip_host, target_host, steps: int,
                     lr: float = 1e-2):
    """The compensation loop of one request through the plain per-call API:
    step k renders with seed + k, takes the L2 loss and the path adjoint in
    one call (render_loss_backward), then an Adam step on Ip clamped to
    [0, 1]."""
    import torch

    sc = gs.scs[scene]
    dev = ctx.device
    view = request_view(sc, side)
    P = Ip_host.to(dev, non_blocking=True)
    tgt = target_host.to(dev, non_blocking=True)
    M, V, G = torch.zeros_like(P), torch.zeros_like(P), torch.zeros_like(P)
    Ic = torch.empty((side, side, 3), device=dev)
    Ec = torch.empty_like(Ic)
    loss = torch.empty(1, device=dev)
    for k in range(steps):
        s = seed + k
        G.zero_()
        ctx.render_loss_backward(gs.handles[scene], gs.alb[scene], gs.rough[scene], P, view, gs.params[scene], spp,
                                 sc.bounces, s, tgt, loss, loss_kind=0, Ic=Ic, Ec=Ec, dIp=G)
        ctx.adam(P, G, M, V, k + 1, lr=lr)
    return Ic, P


def run_per_call(ctx, gs: GpuScenes, host: HostData, workload, keep_outputs=False):
    """Plain baseline: requests in arrival order, one synchronous call (or
    compensation loop) each, results read back before the next starts."""
    import torch

    dev = ctx.device
    records, outputs = [], {}
    outs = _result_buffers(gs, host, workload)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k, rq in enumerate(workload):
        now = time.perf_counter() - t0
        if rq.t_arrival > now:
            time.sleep(rq.t_arrival - now)
        sc = gs.scs[rq.scene]
        Ic_host, Ip_out = outs[k]
        if rq.kind == dpcs.DPCS_REQ_RELIGHT:
            Ip = host.ips[rq.scene][rq.ip_idx].to(dev, non_blocking=True)
            Ic, _ = ctx.render(gs.handles[rq.scene], gs.alb[rq.scene], gs.rough[rq.scene], Ip,
                               request_view(sc, rq.side), gs.params[rq.scene], rq.spp, sc.bounces, rq.seed)
        else:
            Ic, P = compensate_alone(ctx, gs, rq.scene, rq.side, rq.spp, rq.seed, host.ips[rq.scene][rq.ip_idx],
                                     host.target(rq.scene, rq.side), rq.steps)
            Ip_out.copy_(P, non_blocking=True)
        Ic_host.copy_(Ic, non_blocking=True)
        torch.cuda.synchronize()
        t_done = time.perf_counter() - t0
        records.append({"idx": k, "kind": rq.kind, "latency_ms": (t_done - rq.t_arrival) * 1e3,
                        "samples": _samples(rq)})
        if keep_outputs:
            outputs[k] = (Ic_host.numpy().copy(), None if Ip_out is None else Ip_out.numpy().copy())
    wall = time.perf_counter() - t0
    out = summarize(records, wall)
    return (out, outputs) if keep_outputs else out
