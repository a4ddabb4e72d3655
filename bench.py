"""Throughput of the DPCS path tracer on one or more GPUs.

Default workload (one step = one forward render, Eq. 7): the interreflection
corner scene -- three orthogonal planes and an occluding box, T = 1026,
Lambert+GGX textures 256x256, projector 256x256, camera 256x256, 64 samples
per pixel, 3 bounces.  Metric: camera samples per second (Msamples/s).

The same JSON line also carries
  fwd_bwd   : one projector-compensation step (render, L2 loss, path-replay
              adjoint, Adam on Ip; Eq. 13) on the corner scene at 512x512,
              16 spp -- the forward+backward throughput;
  e2e       : the forward metric through the public API with the projector
              image uploaded from pinned host memory and Ic read back every step;
  roofline  : the render kernel's FP32 arithmetic rate against the GPU's FP32
              peak (algorithmic FLOPs counted by the DPCS_COUNTERS build);
  roofline_load / roofline_atomic / roofline_issue : the render kernel's
              node, triangle and texel loads against the measured L2 load
              rate, the replay's float4 atomics against the measured atomic
              rate, and the render kernel's warp instructions against the
              SMs' issue rate;
  compensation, denoise, fit (with a camera-pose step), heightfield (with
              the morphing and rigidly moved surface), principled (metallic
              and normal maps) and serving : the other workloads of the path;
  cpu_baseline : the FP64 oracle on the host cores over a bounded pixel sample.

``--impl reference`` times the oracle alone (the reference arm).  Under
torchrun every rank renders its own independent image (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Msamples/s fwd and fwd+bwd; relight p50/p99 ms under load vs per-call render"
UNIT = "Msamples/s"
WORKLOAD = "corner scene T=1026, camera/projector/textures 256x256, 64 spp, 3 bounces, forward render"
FWD_BWD_WORKLOAD = "corner scene T=1026 at 512x512 (camera, projector, textures), 16 spp, 3 bounces: " \
                   "render + L2 loss + path adjoint (one fused trace) with the gradients of Ip, albedo, roughness " \
                   "and the 11 PRF/CRF/white-balance parameters + Adam on Ip"
L2_FLUSH_BYTES = 256 << 20

# DRAM bytes (read + write) of one k_render launch of this workload, from an
# ncu capture of the same command.  It holds only for the kernel sources it
# was measured on; once they change, the roofline's traffic is reported as
# null until a new capture is taken.
RENDER_TRAFFIC = {"bytes": 20629504, "sources_sha256": "508f75db6f855332a222fba620eb55bc1b90fe365e09b9af620bbc64d8698124"}
# Warp instructions one k_render launch of the forward workload issues, and
# the active lanes per instruction, from the same ncu capture
# (smsp__inst_executed.sum, smsp__thread_inst_executed_per_inst_executed);
# reported while the kernel sources keep this hash.
RENDER_ISSUE = {"warp_instructions": 1192796769, "lanes_per_instruction": 13.54,
                "sources_sha256": "508f75db6f855332a222fba620eb55bc1b90fe365e09b9af620bbc64d8698124"}
# The same two figures for one k_render_grad launch of the compensation step
# with every gradient requested.
FWD_BWD_TRAFFIC = {"bytes": 1898995712,
                   "sources_sha256": "508f75db6f855332a222fba620eb55bc1b90fe365e09b9af620bbc64d8698124"}
FWD_BWD_ISSUE = {"warp_instructions": 1407314884, "lanes_per_instruction": 15.14,
                 "sources_sha256": "508f75db6f855332a222fba620eb55bc1b90fe365e09b9af620bbc64d8698124"}
# the kernels' sources and the tree builder (its topology sets the node visits)
KERNEL_SOURCES = ("paper_2503_12174_gb300/csrc/render.cu", "paper_2503_12174_gb300/csrc/device.cuh",
                  "paper_2503_12174_gb300/csrc/internal.h", "paper_2503_12174_gb300/csrc/lbvh.cu")


def kernel_sources_sha256() -> str:
    import hashlib

    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()

# FP32 arithmetic operations (add, sub, mul, div, sqrt; an FMA counts 2) per
# unit of work, counted from the formulas the kernels evaluate:
FLOP = {
    "node_visits": 26,     # two slab tests: 6 sub + 6 mul each, plus the far-bound widening
    "tri_tests": 46,       # Moller-Trumbore: 2 cross, 4 dot, reciprocal, 3 scalings, origin shift, u+v
    "paths": 27,           # film point, Kc^-1 product, normalisation
    "vertices": 140,       # hit point, normal, UVs, bilinear albedo/roughness, projector projection, shadow setup
    "lit": 160,            # bilinear Ep, geometry term, GGX evaluation with roughness derivative, contribution
    "continuations": 230,  # frame, lobe sample (cosine or visible-normal GGX), pdf, BRDF, throughput
}
# the adjoint's reverse sweep per recorded vertex: per channel the path
# throughput, the BRDF values, dEp, dalbedo, the roughness term and the
# suffix A (about 20), two sets of bilinear weights (16) and the scattered
# products (16 for albedo + roughness, 12 for Ep)
SWEEP_FLOP_PER_VERTEX = 104
# bytes each unit of work loads through L1 (128-bit loads of the layouts in
# csrc/internal.h): a 64-byte node, a 48-byte triangle, three 8-byte UVs,
# four 16-byte texels for albedo+roughness and four for Ep
LOAD_BYTES = {"node_visits": 64, "tri_tests": 48, "vertices": 24 + 4 * 16, "lit": 4 * 16}
# the Eq. 11 filter's settings in the benchmark, and its FP32 operations per
# window tap: albedo, normal and depth distances (8 + 8 + 2), the exponent
# (7), the exponential (2) and the weighted sums (7)
DENOISE_PARAMS = {"radius": 5, "sigma_s": 2.0, "sigma_albedo": 0.1, "sigma_normal": 0.3, "sigma_depth": 0.1}
DENOISE_FLOP_PER_TAP = 34
FIT_PAIRS = 15  # the paper's training set size K
POSE_PAIRS = 3  # pairs per pose step (13 evaluations each with central differences)
POSE_EDGE_SPP = 16  # pose adjoint: samples per pixel edge
POSE_SIL_SPP = 16   # pose adjoint: samples per silhouette edge


def denoise_taps(H: int, W: int, r: int) -> int:
    """Window taps inside an H x W image over all pixels (the window is
    separable in its clipping: taps = sum_y n_y * sum_x n_x)."""
    def n(L):
        return sum(min(L - 1, i + r) - max(0, i - r) + 1 for i in range(L))
    return n(H) * n(W)


# the probes' sizes: a buffer that stays in L2 like the scene and textures, and
# the 512 x 512 gradient texture the compensation replay scatters into
PROBE_L2_BYTES = 32 << 20
PROBE_ATOMIC_TEXELS = 512 * 512


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="dpcs", choices=["dpcs", "reference"])
    ap.add_argument("--fwd-bwd-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target oracle time for cpu_baseline")
    ap.add_argument("--serve-requests", type=int, default=120, help="requests per serving run (0 = skip)")
    ap.add_argument("--serve-rates", default="3,8,14", help="Poisson arrival rates (requests/s) of the load sweep")
    ap.add_argument("--heightfield-steps", type=int, default=2, help="timed steps of the 200k-triangle workload (0 = skip)")
    ap.add_argument("--comp-steps", type=int, default=100, help="Adam steps of the full compensation run (0 = skip)")
    ap.add_argument("--fit-steps", type=int, default=10, help="timed steps of the Eq. 9 scene fit (0 = skip)")
    ap.add_argument("--principled-steps", type=int, default=5,
                    help="timed steps of the principled-material renders (0 = skip)")
    ap.add_argument("--denoise-steps", type=int, default=20,
                    help="timed calls of the Eq. 11 filter and denoised compensation steps (0 = skip)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        cmd = ["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS), "--format=csv,noheader,nounits", "-lms", "100"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.15)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
def aggregate(local_total_ms: float, samples_per_rank: int, steps: int, dist=None, device=None):
    """Whole-job throughput: every rank processed samples_per_rank x steps
    samples; the job took the slowest rank's time.  Returns (Msamples/s,
    max total ms over ranks)."""
    import torch

    ws = dist.get_world_size() if dist else 1
    t = local_total_ms
    if dist:
        x = torch.tensor([local_total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return samples_per_rank * ws * steps / (t / 1e3) / 1e6, t


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    import platform

    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def _cpu_baseline(sc, seconds: float, steps: int | None = None, brute_seconds: float = 0.0):
    """The FP64 oracle in its timing mode (median-split BVH; the same hits,
    images and estimator as its brute-force parity mode) on a bounded random
    pixel sample of ``sc``, all host cores.  Returns (Msamples/s, cores,
    sample description, per-step values, brute-force Msamples/s or None)."""
    import oracle

    oracle.build()
    cores = oracle.num_threads(os.cpu_count() or 1)
    rng = np.random.default_rng(123)
    npix = sc.Hc * sc.Wc
    probe = rng.choice(npix, min(256, npix), replace=False)
    t0 = time.perf_counter()
    oracle.render(sc, pixels=probe, accel=True)
    dt = max(time.perf_counter() - t0, 1e-3)
    per_pixel = dt / len(probe)
    brute = None
    if brute_seconds > 0:
        t0 = time.perf_counter()
        oracle.render(sc, pixels=probe[:32])
        bdt = max(time.perf_counter() - t0, 1e-3)
        nb = int(min(npix, max(32, brute_seconds / (bdt / 32))))
        pxb = rng.choice(npix, nb, replace=False)
        t0 = time.perf_counter()
        oracle.render(sc, pixels=pxb)
        brute = nb * sc.spp / (time.perf_counter() - t0) / 1e6
    if steps is None:
        n = int(min(npix, max(64, seconds / per_pixel)))
        px = rng.choice(npix, n, replace=False)
        t0 = time.perf_counter()
        oracle.render(sc, pixels=px, accel=True)
        dt = time.perf_counter() - t0
        val = n * sc.spp / dt / 1e6
        return (val, cores, f"{n} random pixels x {sc.spp} spp of the workload ({dt:.1f} s, FP64, BVH timing mode)",
                [val], brute)
    n = int(min(npix, max(32, seconds / per_pixel)))
    vals = []
    for k in range(steps):
        px = rng.choice(npix, n, replace=False)
        t0 = time.perf_counter()
        oracle.render(sc, pixels=px, accel=True)
        vals.append(n * sc.spp / (time.perf_counter() - t0) / 1e6)
    return (statistics.mean(vals), cores, f"{n} random pixels x {sc.spp} spp per step (FP64, BVH timing mode)",
            vals, brute)


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from paper_2503_12174_gb300 import scenes

    import oracle

    sc = scenes.corner(res=256, spp=64, bounces=3)
    oracle.build()
    cores = oracle.num_threads(os.cpu_count() or 1)
    # every step renders the whole workload image (all pixels, all samples)
    # with the oracle in its timing mode
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.render(sc, accel=True)
        times.append(time.perf_counter() - t0)
    timed = times[args.warmup:]
    ms = 1e3 * sum(timed) / len(timed)
    v = sc.n_samples / (ms / 1e3) / 1e6
    sample = f"the whole {sc.Hc}x{sc.Wc} image x {sc.spp} spp per step (FP64, BVH timing mode)"
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "reference": "FP64 CPU oracle, BVH timing mode (same hits as its "
                                                          "brute-force parity mode)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2503_12174_gb300 import build as _build

    if rank == 0:  # one rank compiles; the others load what it built
        _build.build()
        _build.build(variant="_counters", defines=("DPCS_COUNTERS",))
        _build.build_probe()
    if dist:
        dist.barrier()
    from paper_2503_12174_gb300 import dpcs, scenes

    dev = torch.device("cuda", local)
    ctx = dpcs.Context(local)
    flush_buf = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def flush(k):
        flush_buf.fill_(float(k))

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x: float) -> float:
        if not dist:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    # ------------------------------------------------------------ forward
    sc = scenes.corner(res=256, spp=64, bounces=3, seed=1000 + rank)
    h = ctx.upload(sc.verts, sc.tris, sc.uv)
    alb = torch.from_numpy(sc.albedo).to(dev)
    rough = torch.from_numpy(sc.rough).to(dev)
    Ip = torch.from_numpy(sc.Ip).to(dev)
    view, prm = dpcs.view_of(sc), dpcs.make_params(sc.params)
    Ic = torch.empty((sc.Hc, sc.Wc, 3), device=dev)
    Ec = torch.empty_like(Ic)
    stream = torch.cuda.current_stream()

    def fwd():
        ctx.render(h, alb, rough, Ip, view, prm, sc.spp, sc.bounces, sc.seed, Ic=Ic, Ec=Ec)

    for k in range(args.warmup):
        flush(k)
        fwd()
    ctx.sync()
    gpu_uuid = None
    try:
        gpu_uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches0 = ctx.launch_count
    barrier()
    ctx.timing(True)
    with ClockSampler(gpu_uuid) as clocks:
        for k in range(args.steps):
            flush(k)
            starts[k].record(stream)
            fwd()
            ends[k].record(stream)
        barrier()
    ctx.sync()
    launches = ctx.launch_count - launches0
    render_ms, render_n = ctx.kernel_time(0)
    ctx.timing(False)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    value, total_ms = aggregate(sum(step_ms), sc.n_samples, args.steps, dist, dev)
    ms_per_step = total_ms / args.steps
    kernel_ms = render_ms / max(render_n, 1)

    # ------------------------------------------------------------ e2e (host buffers)
    Ip_host = torch.from_numpy(sc.Ip.copy()).pin_memory()
    Ic_host = torch.empty((sc.Hc, sc.Wc, 3), dtype=torch.float32).pin_memory()
    Ip_dev = torch.empty_like(Ip)

    def e2e_step():
        Ip_dev.copy_(Ip_host, non_blocking=True)
        ctx.render(h, alb, rough, Ip_dev, view, prm, sc.spp, sc.bounces, sc.seed, Ic=Ic)
        Ic_host.copy_(Ic, non_blocking=True)

    for k in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    e_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    for k in range(args.steps):
        flush(k)
        e_s[k].record(stream)
        e2e_step()
        e_e[k].record(stream)
    barrier()
    e2e_ms = max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(e_s, e_e)))
    e2e_val = sc.n_samples * ws * args.steps / (e2e_ms / 1e3) / 1e6
    np.testing.assert_array_equal(Ic_host.numpy(), Ic.cpu().numpy())

    # ------------------------------------------------------------ fwd + bwd (compensation step)
    # The compensation workload as stated: render, L2 loss against a target
    # rendered from another projector image, the path-replay adjoint with the
    # gradients of Ip, the albedo and roughness textures and the 11 PRF / CRF /
    # white-balance parameters, then Adam on Ip.
    cs = scenes.compensation(res=512, spp=16, seed=2000 + rank)
    hc = ctx.upload(cs.verts, cs.tris, cs.uv)
    calb = torch.from_numpy(cs.albedo).to(dev)
    crough = torch.from_numpy(cs.rough).to(dev)
    cview, cprm = dpcs.view_of(cs), dpcs.make_params(cs.params)
    target = torch.empty((cs.Hc, cs.Wc, 3), device=dev)
    ctx.render(hc, calb, crough, torch.from_numpy(cs.Ip).to(dev), cview, cprm, cs.spp, cs.bounces, cs.seed + 7,
               Ic=target)
    P = torch.full((cs.Hp, cs.Wp, 3), 0.5, device=dev)
    M, V, G = torch.zeros_like(P), torch.zeros_like(P), torch.zeros_like(P)
    gA, gR = torch.zeros_like(calb), torch.zeros_like(crough)
    gP = torch.zeros(11, device=dev)
    cIc = torch.empty((cs.Hc, cs.Wc, 3), device=dev)
    cEc = torch.empty_like(cIc)
    dIc = torch.empty_like(cIc)
    loss = torch.empty(1, device=dev)
    step_no = [0]

    def zero_grads(all_grads):
        G.zero_()
        if all_grads:
            gA.zero_()
            gR.zero_()
            gP.zero_()

    def comp_step_unfused(all_grads=True):
        step_no[0] += 1
        ctx.render(hc, calb, crough, P, cview, cprm, cs.spp, cs.bounces, cs.seed + step_no[0], Ic=cIc, Ec=cEc)
        ctx.l2_loss(cIc, target, dIc, loss)
        zero_grads(all_grads)
        ctx.render_backward(hc, calb, crough, P, cview, cprm, cs.spp, cs.bounces, cs.seed + step_no[0], cEc, cIc,
                            dIc, dIp=G, dAlbedo=gA if all_grads else None, dRough=gR if all_grads else None,
                            dParams=gP if all_grads else None)
        ctx.adam(P, G, M, V, step_no[0], lr=1e-2)

    # the same step as the library's fused call: render, loss and adjoint in
    # one trace of the paths (dpcs_render_loss_backward), then Adam
    def comp_step_fused(all_grads=True):
        step_no[0] += 1
        zero_grads(all_grads)
        ctx.render_loss_backward(hc, calb, crough, P, cview, cprm, cs.spp, cs.bounces, cs.seed + step_no[0], target,
                                 loss, loss_kind=0, Ic=cIc, Ec=cEc, dIp=G, dAlbedo=gA if all_grads else None,
                                 dRough=gR if all_grads else None, dParams=gP if all_grads else None)
        ctx.adam(P, G, M, V, step_no[0], lr=1e-2)

    def timed_steps(fn, n):
        """ms per step of n timed steps (L2 flushed before each), and the
        library's kernel times (render-side, replay-side) per step."""
        for k in range(args.warmup):
            flush(k)
            fn()
        ctx.sync()
        s_ev = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        e_ev = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        barrier()
        ctx.timing(True)
        for k in range(n):
            flush(k)
            s_ev[k].record(stream)
            fn()
            e_ev[k].record(stream)
        barrier()
        ctx.sync()
        k0, n0 = ctx.kernel_time(0)
        k1, n1 = ctx.kernel_time(1)
        ctx.timing(False)
        ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(s_ev, e_ev))) / n
        return ms, (k0 / n if n0 else None), (k1 / n if n1 else None)

    nfb = args.fwd_bwd_steps
    fb_ms, fused_ms, _ = timed_steps(lambda: comp_step_fused(True), nfb)
    fbu_ms, crender_ms, replay_ms = timed_steps(lambda: comp_step_unfused(True), nfb)
    ip_ms, ip_kernel_ms, _ = timed_steps(lambda: comp_step_fused(False), nfb)
    ipu_ms, _, ip_replay_ms = timed_steps(lambda: comp_step_unfused(False), nfb)
    ctx.set_grad_accum(dpcs.DPCS_ACCUM_F64)
    f64_ms, f64_kernel_ms, _ = timed_steps(lambda: comp_step_fused(True), nfb)
    ctx.set_grad_accum(dpcs.DPCS_ACCUM_F32)

    def msps(ms):
        return cs.n_samples * ws / (ms / 1e3) / 1e6

    fb_val = msps(fb_ms)

    # ------------------------------------------------------------ roofline (counters build, untimed)
    counts = None
    flops = None
    try:
        cctx = dpcs.Context(local, lib=dpcs.counters_library())
        ch = cctx.upload(sc.verts, sc.tris, sc.uv)
        cctx.counters(reset=True)
        cctx.render(ch, alb, rough, Ip, view, prm, sc.spp, sc.bounces, sc.seed, Ic=torch.empty_like(Ic))
        counts = cctx.counters(reset=True)
        # the replay of one compensation step: its float4 atomic scatters
        cch = cctx.upload(cs.verts, cs.tris, cs.uv)
        cctx.render(cch, calb, crough, P, cview, cprm, cs.spp, cs.bounces, cs.seed + 1, Ic=cIc, Ec=cEc)
        cctx.counters(reset=True)
        cctx.render_backward(cch, calb, crough, P, cview, cprm, cs.spp, cs.bounces, cs.seed + 1, cEc, cIc, dIc,
                             dIp=torch.zeros_like(P), dAlbedo=torch.zeros_like(calb), dRough=torch.zeros_like(crough),
                             dParams=torch.zeros(11, device=dev))
        replay_counts = cctx.counters(reset=True)
        # the fused step: its forward work and the vertices it sweeps
        cctx.render_loss_backward(cch, calb, crough, P, cview, cprm, cs.spp, cs.bounces, cs.seed + 1, target, loss,
                                  loss_kind=0, Ic=cIc, Ec=cEc, dIp=torch.zeros_like(P),
                                  dAlbedo=torch.zeros_like(calb), dRough=torch.zeros_like(crough),
                                  dParams=torch.zeros(11, device=dev))
        grad_counts = cctx.counters(reset=True)
        cctx.close()
        flops = sum(FLOP[k] * counts[k] for k in FLOP)
    except Exception as e:  # the roofline stays unreported rather than guessed
        counts = {"error": str(e)[:200]}
        replay_counts = None
        grad_counts = None
    # measured roofs the driver's peaks file lacks: L2 load bandwidth and scattered float4 atomics
    from paper_2503_12174_gb300 import probe as _probe

    l2_gbs = _probe.dpcs_probe_l2_load(local, PROBE_L2_BYTES, 256)
    atomic_g = _probe.dpcs_probe_atomic4(local, PROBE_ATOMIC_TEXELS, 1 << 28)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tflops = sms * 128 * 2 * sm_max_mhz * 1e6 / 1e12
    roof = None
    roof_load = None
    roof_atomic = None
    if flops:
        lbytes = sum(LOAD_BYTES[k] * counts[k] for k in LOAD_BYTES)
        l_tbs = lbytes / (kernel_ms / 1e3) / 1e12
        roof_load = {"bound": "l2", "kernel": "k_render", "achieved": l_tbs, "peak": l2_gbs / 1e3, "unit": "TB/s",
                     "frac": l_tbs / (l2_gbs / 1e3), "bytes_per_launch": lbytes,
                     "peak_basis": f"measured: dpcs_probe_l2_load (measurement library), {PROBE_L2_BYTES >> 20} MiB read with 16 B "
                                   "L2-only loads, best of 3",
                     "l1_nominal_peak": sms * 128 * sm_max_mhz * 1e6 / 1e12}
    if replay_counts and replay_ms:
        n_atom = 4 * (replay_counts["vertices"] + replay_counts["lit"])
        r_ms = replay_ms
        roof_atomic = {"bound": "atomic", "kernel": "k_replay", "achieved": n_atom / (r_ms / 1e3) / 1e9,
                       "peak": atomic_g, "unit": "Gatomics/s", "frac": n_atom / (r_ms / 1e3) / 1e9 / atomic_g,
                       "atomics_per_launch": n_atom, "kernel_ms": r_ms,
                       "peak_basis": f"measured: dpcs_probe_atomic4, float4 adds at random texels of a "
                                     f"{PROBE_ATOMIC_TEXELS}-texel buffer, best of 3",
                       "counts_per_launch": replay_counts}
        achieved = flops / (kernel_ms / 1e3) / 1e12
        traffic = RENDER_TRAFFIC["bytes"] if RENDER_TRAFFIC["sources_sha256"] == kernel_sources_sha256() else None
        simt = {}
        if counts.get("trav_warp_iters"):
            simt["traversal"] = (counts["node_visits"] + counts["tri_tests"]) / (32.0 * counts["trav_warp_iters"])
        if counts.get("path_warp_iters"):
            simt["path_loop"] = (counts["rays"] + counts["shadow_rays"]) / (32.0 * counts["path_warp_iters"])
        roof = {"bound": "alu", "kernel": "k_render", "achieved": achieved, "peak": peak_tflops,
                "unit": "TFLOP/s", "frac": achieved / peak_tflops, "traffic": traffic,
                "flops_per_launch": flops, "kernel_ms": kernel_ms,
                "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 FLOP/FMA x {sm_max_mhz:.0f} MHz (max SM clock)",
                "simt_efficiency": simt, "counts_per_launch": counts}
    roof_fb = None
    if grad_counts and "vertices" in grad_counts and fused_ms:
        fb_flops = sum(FLOP[k] * grad_counts[k] for k in FLOP) + SWEEP_FLOP_PER_VERTEX * grad_counts["vertices"]
        ach = fb_flops / (fused_ms / 1e3) / 1e12
        n_atom = 4 * (grad_counts["vertices"] + grad_counts["lit"])
        roof_fb = {"bound": "alu", "kernel": "k_render_grad", "achieved": ach, "peak": peak_tflops, "unit": "TFLOP/s",
                   "frac": ach / peak_tflops, "flops_per_launch": fb_flops, "kernel_ms": fused_ms,
                   "float4_atomics_per_launch": n_atom,
                   "atomic_rate_g_per_s": n_atom / (fused_ms / 1e3) / 1e9, "atomic_peak_g_per_s": atomic_g,
                   "traffic": FWD_BWD_TRAFFIC["bytes"] if FWD_BWD_TRAFFIC["sources_sha256"] == kernel_sources_sha256()
                   else None,
                   "counts_per_launch": grad_counts}
        if FWD_BWD_ISSUE["sources_sha256"] == kernel_sources_sha256():
            inst = FWD_BWD_ISSUE["warp_instructions"]
            issue_peak = 4 * sms * sm_max_mhz * 1e6 / 1e9
            roof_fb["issue"] = {"achieved": inst / (fused_ms / 1e3) / 1e9, "peak": issue_peak,
                                "unit": "G warp-instructions/s", "frac": inst / (fused_ms / 1e3) / 1e9 / issue_peak,
                                "warp_instructions_per_launch": inst,
                                "lanes_per_instruction": FWD_BWD_ISSUE["lanes_per_instruction"]}
    roof_issue = None
    if RENDER_ISSUE["sources_sha256"] == kernel_sources_sha256():
        # instruction issue: each SM sub-partition issues at most one warp
        # instruction per cycle, four per SM
        inst = RENDER_ISSUE["warp_instructions"]
        issue_peak = 4 * sms * sm_max_mhz * 1e6 / 1e9
        issue = inst / (kernel_ms / 1e3) / 1e9
        roof_issue = {"bound": "issue", "kernel": "k_render", "achieved": issue, "peak": issue_peak,
                      "unit": "G warp-instructions/s", "frac": issue / issue_peak, "kernel_ms": kernel_ms,
                      "warp_instructions_per_launch": inst,
                      "lanes_per_instruction": RENDER_ISSUE["lanes_per_instruction"],
                      "peak_basis": f"{sms} SMs x 4 schedulers x 1 warp-instruction/cycle x {sm_max_mhz:.0f} MHz",
                      "source": "instruction count of one launch of this workload, from an ncu capture of the same "
                                "kernel sources"}

    # ------------------------------------------------------------ full compensation (Eq. 13): eager vs CUDA graph
    comp_out = None
    if args.comp_steps > 0:
        from paper_2503_12174_gb300 import compensate

        cmp_res = {}
        for mode in ("eager", "graph"):
            cm = compensate.Compensation(ctx, hc, calb, crough, cview, cprm, cs.spp, cs.bounces, args.comp_steps,
                                         lr=1e-2, seed=4000 + rank, graph=(mode == "graph"))
            init = torch.full((cs.Hp, cs.Wp, 3), 0.5, device=dev)
            cm.run(init, target)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(2)]
            barrier()
            for k in range(2):
                ev[k][0].record(stream)
                _, hist = cm.run(init, target)
                ev[k][1].record(stream)
            barrier()
            ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev)) / 2
            losses = hist.cpu().numpy()
            cmp_res[mode] = {"ms": ms, "Msamples_per_s": cs.n_samples * args.comp_steps * ws / (ms / 1e3) / 1e6,
                             "loss_first": float(losses[0]), "loss_last": float(losses[-1])}
            del cm
        comp_out = {"workload": f"{FWD_BWD_WORKLOAD}; {args.comp_steps} steps from Ip = 0.5", **cmp_res}

    # ------------------------------------------------------------ Eq. 11 denoiser (cross-bilateral filter)
    den_out = None
    if args.denoise_steps > 0:
        from paper_2503_12174_gb300 import compensate

        dprm = dpcs.make_denoise_params(**DENOISE_PARAMS)
        guide = ctx.gbuffer(hc, calb, crough, cview)
        X = torch.rand((cs.Hc, cs.Wc, 3), device=dev)
        Dout, Wsum, dX = torch.empty_like(X), torch.empty((cs.Hc, cs.Wc), device=dev), torch.zeros_like(X)

        def timed(fn, n):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(n):
                fn()
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1) / n

        n = args.denoise_steps
        f_ms = timed(lambda: ctx.denoise(X, guide, dprm, out=Dout, wsum=Wsum), n)
        b_ms = timed(lambda: ctx.denoise_backward(X, guide, Wsum, dprm, dIc=dX), n)
        g_ms = timed(lambda: ctx.gbuffer(hc, calb, crough, cview, guide=guide), n)
        flops = denoise_taps(cs.Hc, cs.Wc, DENOISE_PARAMS["radius"]) * DENOISE_FLOP_PER_TAP
        d_tflops = flops / (f_ms / 1e3) / 1e12
        cm = compensate.Compensation(ctx, hc, calb, crough, cview, cprm, cs.spp, cs.bounces, n, lr=1e-2,
                                     seed=5000 + rank, graph=True, denoise=dprm)
        init = torch.full((cs.Hp, cs.Wp, 3), 0.5, device=dev)
        cm.run(init, target)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        _, dhist = cm.run(init, target)
        e1.record(stream)
        barrier()
        dc_ms = max_over_ranks(e0.elapsed_time(e1))
        dl = dhist.cpu().numpy()
        del cm
        den_out = {
            "workload": f"cross-bilateral filter of Eq. 11 on the {cs.Hc}x{cs.Wc} compensation image, "
                        f"radius {DENOISE_PARAMS['radius']}, guide = first hit through each pixel centre",
            "params": DENOISE_PARAMS, "filter_ms": f_ms, "adjoint_ms": b_ms, "gbuffer_ms": g_ms,
            "roofline": {"bound": "alu", "kernel": "k_bilateral", "achieved": d_tflops, "peak": peak_tflops,
                         "unit": "TFLOP/s", "frac": d_tflops / peak_tflops, "flops_per_launch": flops,
                         "flop_per_tap": DENOISE_FLOP_PER_TAP},
            "denoised_compensation": {"steps": n, "ms": dc_ms,
                                      "Msamples_per_s": cs.n_samples * n * ws / (dc_ms / 1e3) / 1e6,
                                      "loss_first": float(dl[0]), "loss_last": float(dl[-1]),
                                      "workload": f"corner scene T=1026 at {cs.Hc}x{cs.Wc} (camera, projector, textures), "
                                                  f"{cs.spp} spp, {cs.bounces} bounces: render keeping the path records + "
                                                  "Eq. 11 filter + L2 loss on D(Ic) + filter adjoint + sweep over the "
                                                  "kept records + Adam on Ip, one CUDA graph"},
        }

    # ------------------------------------------------------------ scene-parameter fitting (Eq. 9)
    fit_out = None
    if args.fit_steps > 0:
        from paper_2503_12174_gb300 import fit

        fs = scenes.corner(res=256, tex=256, spp=16, bounces=3, seed=6000 + rank)
        fh = ctx.upload(fs.verts, fs.tris, fs.uv)
        f_alb, f_rough = torch.from_numpy(fs.albedo).to(dev), torch.from_numpy(fs.rough).to(dev)
        fview, fprm = dpcs.view_of(fs), dpcs.make_params(fs.params)
        frng = np.random.default_rng(6100 + rank)
        pairs = []
        for i in range(FIT_PAIRS):  # captures: the true scene at 64 spp
            Ip_i = torch.from_numpy(scenes.blob_image(frng, fs.Hp, fs.Wp).astype(np.float32)).to(dev)
            cap, _ = ctx.render(fh, f_alb, f_rough, Ip_i, fview, fprm, 64, fs.bounces, 6200 + i)
            pairs.append((Ip_i, cap))
        p0 = scenes.Params(gamma_p=(2.5, 2.5, 2.5), gain_p=fs.params.gain_p, gamma_c=(0.7, 0.7, 0.7),
                           gain_c=fs.params.gain_c, wb=(1.0, 1.0, 1.0), k_proj=fs.params.k_proj, ks=fs.params.ks,
                           f0=fs.params.f0)
        half = torch.full_like(f_alb, 0.5)
        fobj = fit.SceneFit(ctx, fh, fview, dpcs.make_params(p0), half, torch.full_like(f_rough, 0.5), pairs, fs.spp,
                            fs.bounces, tv_weight=1e-5, denoise=dpcs.make_denoise_params(**DENOISE_PARAMS),
                            seed=6300 + rank)
        fobj.step()  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        fhist = fobj.run(args.fit_steps)
        e1.record(stream)
        barrier()
        fit_ms = max_over_ranks(e0.elapsed_time(e1))
        true_alb = f_alb.double()
        fit_out = {
            "workload": f"Eq. 9 fit on the corner scene at {fs.Hc}x{fs.Wc} (camera, projector, textures): "
                        f"{FIT_PAIRS} projector/capture pairs per step at {fs.spp} spp, {fs.bounces} bounces, "
                        "Eq. 11 denoiser before the L1 loss, TV 1e-5, Adam on albedo, roughness, gamma_p, gamma_c, w",
            "steps": args.fit_steps, "ms_per_step": fit_ms / args.fit_steps,
            "Msamples_per_s": FIT_PAIRS * fs.n_samples * args.fit_steps * ws / (fit_ms / 1e3) / 1e6,
            "loss_first": float(fhist[0]), "loss_last": float(fhist[-1]),
            "albedo_mae_start": float((half.double() - true_alb).abs().mean()),
            "albedo_mae_end": float((fobj.albedo.double() - true_alb).abs().mean()),
        }
        # camera-pose refinement on the same scene, from a pose off by ~1
        # degree: Adam steps on the pose with its gradient from the pose
        # adjoint (per pair one render, L1 term and dpcs_pose_backward) and
        # from central differences (13 evaluations of the data term, each a
        # rigid transform + refit and POSE_PAIRS renders)
        from paper_2503_12174_gb300 import pose as pose_mod

        xi0 = np.array([0.01, -0.008, 0.006, 0.01, -0.01, 0.015])
        fit_out["pose"] = {}
        for grad_kind in ("adjoint", "differences"):
            pr = pose_mod.PoseRefine(ctx, fh, fview, fprm, f_alb, f_rough, pairs[:POSE_PAIRS], fs.spp, fs.bounces,
                                     seed=6400 + rank, xi0=xi0, lr=2e-3, gradient=grad_kind,
                                     edge_spp=POSE_EDGE_SPP, sil_spp=POSE_SIL_SPP)
            pr.step()  # warm-up
            torch.cuda.synchronize()
            barrier()
            t0 = time.perf_counter()
            e0.record(stream)
            phist = [pr.step() for _ in range(args.fit_steps)]
            e1.record(stream)
            e1.synchronize()
            pose_wall_ms = (time.perf_counter() - t0) * 1e3
            barrier()
            pose_ms = max_over_ranks(e0.elapsed_time(e1))
            xi_end = pr.xi.cpu().numpy().astype(np.float64)
            ctx.transform(fh, np.eye(3), np.zeros(3))
            if grad_kind == "adjoint":
                work = (f"{POSE_PAIRS} pairs: per pair one render, the mean L1 term and the pose adjoint (interior "
                        f"samples as the render, {POSE_EDGE_SPP} samples per pixel edge, {POSE_SIL_SPP} per "
                        "silhouette edge), then Adam on the pose")
                paths = POSE_PAIRS * fs.n_samples * (2 + 4 * POSE_EDGE_SPP / fs.spp)  # render + adjoint paths
            else:
                work = (f"{POSE_PAIRS} pairs: 13 evaluations of the mean L1 data term per step (transform + refit, "
                        "renders, L1 terms), then Adam on the pose")
                paths = 13 * POSE_PAIRS * fs.n_samples
            fit_out["pose"][grad_kind] = {
                "workload": "camera-pose refinement, same scene and renders, " + work,
                "steps": args.fit_steps, "ms_per_step": pose_ms / args.fit_steps,
                "wall_ms_per_step": pose_wall_ms / args.fit_steps,
                "Mpaths_per_s": paths * args.fit_steps * ws / (pose_ms / 1e3) / 1e6,
                "loss_first": float(phist[0]), "loss_last": float(phist[-1]),
                "pose_error_start": [float(np.linalg.norm(xi0[:3])), float(np.linalg.norm(xi0[3:]))],
                "pose_error_end": [float(np.linalg.norm(xi_end[:3])), float(np.linalg.norm(xi_end[3:]))],
            }
        del fobj, pairs, pr
        ctx.free(fh)

    # ------------------------------------------------------------ large displaced surface (T = 199,712)
    hf_out = None
    if args.heightfield_steps > 0:
        hs = scenes.heightfield(spp=256, seed=3000 + rank)
        hh = ctx.upload(hs.verts, hs.tris, hs.uv)
        halb = torch.from_numpy(hs.albedo).to(dev)
        hrough = torch.from_numpy(hs.rough).to(dev)
        hIp = torch.from_numpy(hs.Ip).to(dev)
        hview, hprm = dpcs.view_of(hs), dpcs.make_params(hs.params)
        hIc = torch.empty((hs.Hc, hs.Wc, 3), device=dev)
        hEc = torch.empty_like(hIc)
        hG = torch.zeros_like(hIp)

        def hf_fwd(spp):
            ctx.render(hh, halb, hrough, hIp, hview, hprm, spp, hs.bounces, hs.seed, Ic=hIc, Ec=hEc)

        # a compensation step against a target image: render, L2 loss and the
        # adjoint to Ip in one trace of the paths (4 bounces, 1 sample per lane)
        htarget = (torch.rand_like(hIc) * 0.5).contiguous()
        hloss = torch.zeros(1, device=dev)

        hgA, hgR, hgP = torch.zeros_like(halb), torch.zeros_like(hrough), torch.zeros(11, device=dev)

        def hf_fb(spp):
            hG.zero_()
            hgA.zero_()
            hgR.zero_()
            hgP.zero_()
            ctx.render_loss_backward(hh, halb, hrough, hIp, hview, hprm, spp, hs.bounces, hs.seed, htarget, hloss,
                                     loss_kind=0, Ic=hIc, Ec=hEc, dIp=hG, dAlbedo=hgA, dRough=hgR, dParams=hgP)

        res = {}
        for name, fn, spp in (("fwd", hf_fwd, 256), ("fwd_bwd", hf_fb, 32)):
            fn(spp)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.heightfield_steps)]
            barrier()
            for k in range(args.heightfield_steps):
                flush(k)
                ev[k][0].record(stream)
                fn(spp)
                ev[k][1].record(stream)
            barrier()
            ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev)) / args.heightfield_steps
            res[name] = {"value": hs.Hc * hs.Wc * spp * ws / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": ms,
                         "spp": spp}
        # a morphing surface re-lit frame by frame (Sec. 4.4): per frame the
        # new vertex positions go up from host memory, the tree is refitted
        # and the frame is rendered at 16 spp; against a full re-upload
        nfr = args.heightfield_steps + 2
        frames = [(hs.verts + np.float32(0.01 * np.sin(0.7 * f + 3.0 * hs.verts[:, :1]))
                   * np.asarray([0.0, 0.0, 1.0], np.float32)).astype(np.float32) for f in range(nfr)]
        ctx.update(hh, frames[0])
        hf_fwd(16)
        torch.cuda.synchronize()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(nfr - 1)]
        barrier()
        for f in range(1, nfr):
            ev[f - 1][0].record(stream)
            ctx.update(hh, frames[f])
            ev[f - 1][1].record(stream)
            hf_fwd(16)
            ev[f - 1][2].record(stream)
        barrier()
        torch.cuda.synchronize()
        upd_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b, _ in ev)) / (nfr - 1)
        frame_ms = max_over_ranks(sum(a.elapsed_time(c) for a, _, c in ev)) / (nfr - 1)
        t0 = time.perf_counter()
        hh2 = ctx.upload(frames[-1], hs.tris, hs.uv)
        rebuild_ms = (time.perf_counter() - t0) * 1e3
        ctx.free(hh2)
        # a rigid move of the whole surface (camera-pose refinement): transform + refit on the device
        evt = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
        from paper_2503_12174_gb300 import pose as pose_mod
        for k, (a, b) in enumerate(evt):
            a.record(stream)
            ctx.transform(hh, pose_mod.rotation([0.001 * k, 0.0, 0.002]), np.array([0.0, 0.001 * k, 0.0]))
            b.record(stream)
        torch.cuda.synchronize()
        transform_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evt[1:]) / (len(evt) - 1))
        res["morph"] = {"workload": "heightfield vertices moved every frame, then rendered at 16 spp",
                        "update_ms": upd_ms, "frame_ms": frame_ms, "full_upload_ms": rebuild_ms,
                        "rigid_transform_ms": transform_ms, "frames": nfr - 1}
        ctx.sync()
        ctx.free(hh)
        hf_out = {"workload": f"heightfield T={hs.T}, camera {hs.Hc}x{hs.Wc}, projector {hs.Wp}x{hs.Hp}, "
                              f"textures 512x512, {hs.bounces} bounces, Russian roulette from vertex 2 (q=0.75); "
                              "fwd_bwd = render + L2 loss + adjoint to Ip, textures and response parameters in one fused call",
                  **res}

    # ------------------------------------------------------------ principled material (metallic + normal maps)
    pbr_out = None
    if args.principled_steps > 0:
        # the forward workload and the compensation workload with seeded
        # metallic and normal maps of their texture sizes
        ps = scenes.with_principled(sc, seed=4000 + rank)
        pm = torch.from_numpy(ps.metallic).to(dev)
        pn = torch.from_numpy(ps.normal).to(dev)
        pcs = scenes.with_principled(cs, seed=4100 + rank)
        cpm = torch.from_numpy(pcs.metallic).to(dev)
        cpn = torch.from_numpy(pcs.normal).to(dev)
        gA, gR = torch.zeros_like(calb), torch.zeros_like(crough)
        gM, gN = torch.zeros_like(cpm), torch.zeros_like(cpn)

        def pbr_fwd():
            ctx.render_principled(h, alb, rough, pm, pn, Ip, view, prm, sc.spp, sc.bounces, sc.seed, Ic=Ic, Ec=Ec)

        def pbr_step():  # compensation step: render, L2 loss, adjoint to Ip, Adam
            step_no[0] += 1
            ctx.render_principled(hc, calb, crough, cpm, cpn, P, cview, cprm, cs.spp, cs.bounces,
                                  cs.seed + step_no[0], Ic=cIc, Ec=cEc)
            ctx.l2_loss(cIc, target, dIc, loss)
            G.zero_()
            ctx.render_backward_principled(hc, calb, crough, cpm, cpn, P, cview, cprm, cs.spp, cs.bounces,
                                           cs.seed + step_no[0], cEc, cIc, dIc, dIp=G)
            ctx.adam(P, G, M, V, step_no[0], lr=1e-2)

        def pbr_step_fused():  # the same step in one trace: render, L2 loss and adjoint, then Adam
            step_no[0] += 1
            G.zero_()
            ctx.render_loss_backward_principled(hc, calb, crough, cpm, cpn, P, cview, cprm, cs.spp, cs.bounces,
                                                cs.seed + step_no[0], target, loss, loss_kind=0, Ic=cIc, Ec=cEc,
                                                dIp=G)
            ctx.adam(P, G, M, V, step_no[0], lr=1e-2)

        def pbr_all():  # one fitting pass: every material gradient (albedo, roughness, metallic, normal map)
            ctx.render_principled(hc, calb, crough, cpm, cpn, P, cview, cprm, cs.spp, cs.bounces, cs.seed,
                                  Ic=cIc, Ec=cEc)
            ctx.render_backward_principled(hc, calb, crough, cpm, cpn, P, cview, cprm, cs.spp, cs.bounces, cs.seed,
                                           cEc, cIc, dIc, dAlbedo=gA, dRough=gR, dMetallic=gM, dNormal=gN)

        res = {}
        for name, fn, n_samp in (("fwd", pbr_fwd, sc.n_samples), ("fwd_bwd", pbr_step, cs.n_samples),
                                 ("fwd_bwd_fused", pbr_step_fused, cs.n_samples),
                                 ("fwd_bwd_material", pbr_all, cs.n_samples)):
            for k in range(args.warmup):
                flush(k)
                fn()
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.principled_steps)]
            barrier()
            for k in range(args.principled_steps):
                flush(k)
                ev[k][0].record(stream)
                fn()
                ev[k][1].record(stream)
            barrier()
            ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev)) / args.principled_steps
            res[name] = {"value": n_samp * ws / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": ms}
        pbr_out = {"workload": f"principled material (metallic map + normal map): fwd = corner {sc.Hc}x{sc.Wc}, "
                               f"{sc.spp} spp, {sc.bounces} bounces; fwd_bwd = compensation step at {cs.Hc}x{cs.Wc}, "
                               f"{cs.spp} spp (render, L2 loss, replay adjoint to Ip, Adam); fwd_bwd_fused = the same step "
                               "in one trace (dpcs_render_loss_backward_principled); fwd_bwd_material = "
                               "render + replay with albedo, roughness, metallic and normal-map gradients",
                   **res}

    # ------------------------------------------------------------ serving vs one call per request
    serving_out = None
    if args.serve_requests > 0:
        from paper_2503_12174_gb300 import serving

        scs = serving.resident_scenes()
        gs = serving.GpuScenes(ctx, scs)
        host = serving.HostData(scs)
        warm = serving.make_workload(6, rate=0.0, seed=99, sides=(128, 256), spp_range=(16, 32), comp_steps=2)
        serving.run_server(ctx, gs, host, warm)
        serving.run_per_call(ctx, gs, host, warm)
        keep = ("requests_per_s", "relight_p50_ms", "relight_p99_ms", "compensation_p50_ms", "compensation_p99_ms",
                "samples_per_s_M", "wall_s")
        sweep = []
        deadline = dict(policy=dpcs.DPCS_SERVE_DEADLINE, relight_slack=4.0, compensation_slack=0.5)
        for rate in [float(x) for x in args.serve_rates.split(",") if x]:
            wl = serving.make_workload(args.serve_requests, rate=rate, seed=100 + rank)
            srv = serving.run_server(ctx, gs, host, wl)
            per = serving.run_per_call(ctx, gs, host, wl)
            entry = {"offered_rate_per_s": rate, "server": {k: srv[k] for k in keep},
                     "per_call": {k: per[k] for k in keep}, "server_iterations": srv["server"]["iterations"],
                     "server_memory_high_water_bytes": srv["server"]["memory_high_water"]}
            if rate >= 8.0:  # the deadline policies beside the default fixed share
                dl = serving.run_server(ctx, gs, host, wl, **deadline)
                entry["server_deadline_policy"] = {k: dl[k] for k in keep}
                qd = serving.run_server(ctx, gs, host, wl, **dict(deadline, policy=dpcs.DPCS_SERVE_QUANTA_DEADLINE,
                                                                  compensation_slack=0.1))
                entry["server_quanta_deadline_policy"] = {k: qd[k] for k in keep}
            sweep.append(entry)
        sat = serving.make_workload(args.serve_requests, rate=0.0, seed=200 + rank)
        srv_sat = serving.run_server(ctx, gs, host, sat)
        per_sat = serving.run_per_call(ctx, gs, host, sat)
        for hh in gs.handles:
            ctx.free(hh)
        serving_out = {
            "workload": f"{args.serve_requests} requests per run over 3 resident scenes (plane, corner256, corner512); "
                        "camera side in {128..1024 step 64}, spp log-uniform 16-256; 90% relight, "
                        "10% compensation (50 Adam steps, 16 spp); Poisson arrivals",
            "policy": "server = fixed share (relighting quanta, compensation within half of each iteration); "
                      "server_deadline_policy = earliest deadline first, slack 4 (relight) and 0.5 (compensation); "
                      "server_quanta_deadline_policy = the relighting quanta, then the deadline order, slack 4 "
                      "(relight) and 0.1 (compensation)",
            "load_sweep": sweep,
            "saturated": {"server_requests_per_s": srv_sat["requests_per_s"],
                          "per_call_requests_per_s": per_sat["requests_per_s"],
                          "server_relight_p99_ms": srv_sat["relight_p99_ms"],
                          "per_call_relight_p99_ms": per_sat["relight_p99_ms"]},
        }

    # ------------------------------------------------------------ CPU baseline
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, cores, sample, _, brute = _cpu_baseline(sc, seconds=args.cpu_seconds, brute_seconds=4.0)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample, "cpu_model": cpu_model(),
               "brute_force_value": brute}

    clk = clocks.summary()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "samples_per_step_per_gpu": sc.n_samples, "spp": sc.spp,
                       "bounces": sc.bounces, "triangles": sc.T, "resolution": [sc.Hc, sc.Wc],
                       "l2": f"flushed: {L2_FLUSH_BYTES >> 20} MiB write between timed steps (inputs < L2)",
                       "parallelism": f"replicas x{ws} (independent images, no collective)"},
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(Ip_host.numel() * 4),
                    "d2h_bytes_per_step": int(Ic_host.numel() * 4)},
            "fwd_bwd": {"value": fb_val, "unit": UNIT, "workload": FWD_BWD_WORKLOAD,
                        "ms_per_step": fb_ms, "steps": nfb, "samples_per_step_per_gpu": cs.n_samples,
                        "fused_kernel_ms": fused_ms,
                        "unfused": {"value": msps(fbu_ms), "ms_per_step": fbu_ms, "render_kernel_ms": crender_ms,
                                    "replay_kernel_ms": replay_ms,
                                    "workload": "the same step as separate render, L2 loss, replay adjoint calls"},
                        "fp64_accumulation": {"value": msps(f64_ms), "ms_per_step": f64_ms,
                                              "fused_kernel_ms": f64_kernel_ms,
                                              "workload": "the same fused step with FP64 gradient accumulators "
                                                          "(dpcs_set_grad_accum DPCS_ACCUM_F64)"},
                        "ip_only": {"value": msps(ip_ms), "ms_per_step": ip_ms, "fused_kernel_ms": ip_kernel_ms,
                                    "unfused_value": msps(ipu_ms), "unfused_replay_kernel_ms": ip_replay_ms,
                                    "workload": "the same step asking only for dIp (no texture or response "
                                                "gradients)"}},
            "roofline_fwd_bwd": roof_fb,
            "roofline": roof,
            "roofline_load": roof_load,
            "roofline_atomic": roof_atomic,
            "roofline_issue": roof_issue,
            "compensation": comp_out,
            "denoise": den_out,
            "fit": fit_out,
            "heightfield": hf_out,
            "principled": pbr_out,
            "serving": serving_out,
            "cpu_baseline": cpu,
            "clocks": clk,
            "gpu_launches": int(launches),
            "kernel_ms_per_step": kernel_ms,
        }
        # the headline figures again, last on the line, so that a reader of
        # its tail alone sees them
        summ = {"fwd": value, "fwd_kernel_ms": kernel_ms, "fwd_alu_frac": roof["frac"] if roof else None,
                "fwd_issue_frac": roof_issue["frac"] if roof_issue else None,
                "fwd_traffic_bytes": roof["traffic"] if roof else None,
                "fwd_bwd_all_grads": fb_val, "fwd_bwd_all_grads_unfused": msps(fbu_ms),
                "fwd_bwd_fp64_accum": msps(f64_ms), "fwd_bwd_ip_only": msps(ip_ms),
                "fwd_bwd_alu_frac": roof_fb["frac"] if roof_fb else None,
                "e2e": e2e_val, "cpu_baseline": cpu["value"] if cpu else None}
        if hf_out:
            summ["heightfield_fwd"] = hf_out["fwd"]["value"]
            summ["heightfield_fwd_bwd"] = hf_out["fwd_bwd"]["value"]
        if comp_out:
            summ["compensation_100_steps_ms"] = comp_out["graph"]["ms"]
        if fit_out and "pose" in fit_out:
            summ["pose_step_ms"] = {k: v["ms_per_step"] for k, v in fit_out["pose"].items()}
        if serving_out:
            summ["serving"] = [{"rate": x["offered_rate_per_s"], "srv_relight_p99": x["server"]["relight_p99_ms"],
                                "call_relight_p99": x["per_call"]["relight_p99_ms"],
                                "srv_comp_p99": x["server"]["compensation_p99_ms"],
                                "call_comp_p99": x["per_call"]["compensation_p99_ms"],
                                "deadline_relight_p99": x.get("server_deadline_policy", {}).get("relight_p99_ms"),
                                "deadline_comp_p99": x.get("server_deadline_policy", {}).get("compensation_p99_ms"),
                                "qdeadline_relight_p99": x.get("server_quanta_deadline_policy", {}).get("relight_p99_ms"),
                                "qdeadline_comp_p99": x.get("server_quanta_deadline_policy", {}).get("compensation_p99_ms")}
                               for x in serving_out["load_sweep"]]
        line["summary"] = short_figures(summ)
        print(json.dumps(line), flush=True)
    ctx.free(h)
    ctx.free(hc)
    ctx.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def short_figures(x):
    """x with floats rounded to 4 significant digits and None entries of
    dicts dropped (the summary is repeated at the end of the line to be read
    from its tail, so it is kept short)."""
    if isinstance(x, float):
        return float(f"{x:.4g}")
    if isinstance(x, dict):
        return {k: short_figures(v) for k, v in x.items() if v is not None}
    if isinstance(x, list):
        return [short_figures(v) for v in x]
    return x


if __name__ == "__main__":
    main()
