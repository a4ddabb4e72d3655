"""Projector compensation (Eq. 13): Ip* = argmin_Ip |R(Ip, theta) - Ic|.

The loop runs entirely on the device through the C ABI.  Each step renders
Ic = R(Ip) with a fresh Philox key (seed + k), takes the L2 loss against the
target, carries dL/dIc back to Ip with the path adjoint, and applies an Adam
step followed by the clamp of Ip to [0, 1].  By default the render, loss and
adjoint are one call that traces each path once
(``Context.render_loss_backward``); with the denoiser the render keeps its
path records and the adjoint sweeps them (``keep`` / ``kept``) instead of
tracing again.  ``fused=False`` makes the separate render, loss and replay
calls instead.

With ``denoise`` set (a ``dpcs.DpcsDenoiseParams``), the loss is taken on
the denoised image D(Ic) of Eq. 11 instead, and dL/dD is carried back to
dL/dIc by the filter's adjoint before the replay.  The filter's guide is the
scene's first hit through each pixel centre, computed once.

With ``metallic`` / ``normal`` maps the scene uses the principled material
of Sec. 3.2: the one-trace step is ``render_loss_backward_principled``, and
with the denoiser the principled render keeps its path records as well.

With ``graph=True`` the whole loop is captured once as a CUDA graph and then
replayed.  The steps are unrolled in the graph, so every step keeps its own
seed and Adam step number, and one replay runs the full compensation.  The
library's scratch memory is sized by one eager step before the capture.
"""
from __future__ import annotations

from . import dpcs


class Compensation:
    """Device state and (optionally) a captured CUDA graph for one scene,
    view and target size."""

    def __init__(self, ctx: dpcs.Context, scene: int, albedo, rough, view: dpcs.DpcsView, params: dpcs.DpcsParams,
                 spp: int, bounces: int, steps: int, lr: float = 1e-2, seed: int = 0, graph: bool = True,
                 denoise: dpcs.DpcsDenoiseParams | None = None, guide=None, fused: bool = True, metallic=None,
                 normal=None):
        import torch

        self.ctx, self.scene, self.albedo, self.rough = ctx, scene, albedo, rough
        self.metallic, self.normal = metallic, normal
        self.principled = metallic is not None or normal is not None
        self.view, self.params, self.spp, self.bounces = view, params, int(spp), int(bounces)
        self.steps, self.lr, self.seed = int(steps), float(lr), int(seed)
        dev = ctx.device
        f32 = torch.float32
        self.P = torch.zeros((view.Hp, view.Wp, 3), dtype=f32, device=dev)
        self.P0 = torch.zeros_like(self.P)
        self.M, self.V, self.G = torch.zeros_like(self.P), torch.zeros_like(self.P), torch.zeros_like(self.P)
        self.target = torch.zeros((view.Hc, view.Wc, 3), dtype=f32, device=dev)
        self.Ic = torch.empty_like(self.target)
        self.Ec = torch.empty_like(self.target)
        self.dIc = torch.empty_like(self.target)
        self.loss = torch.zeros(1, dtype=f32, device=dev)
        self.history = torch.zeros(self.steps, dtype=f32, device=dev)
        self.denoise = denoise
        self.fused = bool(fused)
        if denoise is not None:
            self.guide = guide if guide is not None else ctx.gbuffer(scene, albedo, rough, view)
            self.D = torch.empty_like(self.target)
            self.wsum = torch.empty((view.Hc, view.Wc), dtype=f32, device=dev)
            self.dD = torch.empty_like(self.target)
        self.graph = None
        if graph:
            self._step(0)  # sizes the library's scratch outside the capture
            torch.cuda.synchronize()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph):
                self._loop()

    def _step(self, k: int):
        c = self.ctx
        s = self.seed + k
        if self.principled:
            self._step_principled(k, s)
            return
        if self.denoise is None and self.fused:  # render, loss and adjoint in one trace of the paths
            self.G.zero_()
            c.render_loss_backward(self.scene, self.albedo, self.rough, self.P, self.view, self.params, self.spp,
                                   self.bounces, s, self.target, self.loss, loss_kind=0, Ic=self.Ic, Ec=self.Ec,
                                   dIp=self.G)
            self.history[k].copy_(self.loss[0])
            c.adam(self.P, self.G, self.M, self.V, k + 1, lr=self.lr, lo=0.0, hi=1.0)
            return
        keep = self.denoise is not None and self.fused  # the filter couples pixels: keep the paths for the adjoint
        c.render(self.scene, self.albedo, self.rough, self.P, self.view, self.params, self.spp, self.bounces, s,
                 Ic=self.Ic, Ec=self.Ec, keep=keep)
        if self.denoise is None:
            c.l2_loss(self.Ic, self.target, self.dIc, self.loss)
        else:
            c.denoise(self.Ic, self.guide, self.denoise, out=self.D, wsum=self.wsum)
            c.l2_loss(self.D, self.target, self.dD, self.loss)
            self.dIc.zero_()
            c.denoise_backward(self.dD, self.guide, self.wsum, self.denoise, dIc=self.dIc)
        self.history[k].copy_(self.loss[0])
        self.G.zero_()
        c.render_backward(self.scene, self.albedo, self.rough, self.P, self.view, self.params, self.spp, self.bounces, s,
                          self.Ec, self.Ic, self.dIc, dIp=self.G, kept=keep)
        c.adam(self.P, self.G, self.M, self.V, k + 1, lr=self.lr, lo=0.0, hi=1.0)

    def _step_principled(self, k: int, s: int):
        c = self.ctx
        self.G.zero_()
        if self.denoise is None and self.fused:  # one trace of the paths
            c.render_loss_backward_principled(self.scene, self.albedo, self.rough, self.metallic, self.normal, self.P,
                                              self.view, self.params, self.spp, self.bounces, s, self.target,
                                              self.loss, loss_kind=0, Ic=self.Ic, Ec=self.Ec, dIp=self.G)
        else:
            keep = self.denoise is not None and self.fused  # the filter couples pixels: keep the paths
            c.render_principled(self.scene, self.albedo, self.rough, self.metallic, self.normal, self.P, self.view,
                                self.params, self.spp, self.bounces, s, Ic=self.Ic, Ec=self.Ec, keep=keep)
            if self.denoise is None:
                c.l2_loss(self.Ic, self.target, self.dIc, self.loss)
            else:
                c.denoise(self.Ic, self.guide, self.denoise, out=self.D, wsum=self.wsum)
                c.l2_loss(self.D, self.target, self.dD, self.loss)
                self.dIc.zero_()
                c.denoise_backward(self.dD, self.guide, self.wsum, self.denoise, dIc=self.dIc)
            c.render_backward_principled(self.scene, self.albedo, self.rough, self.metallic, self.normal, self.P,
                                         self.view, self.params, self.spp, self.bounces, s, self.Ec, self.Ic,
                                         self.dIc, dIp=self.G, kept=keep)
        self.history[k].copy_(self.loss[0])
        c.adam(self.P, self.G, self.M, self.V, k + 1, lr=self.lr, lo=0.0, hi=1.0)

    def _loop(self):
        self.P.copy_(self.P0)
        self.M.zero_()
        self.V.zero_()
        for k in range(self.steps):
            self._step(k)

    # -- step by step, with checkpoints -----------------------------------------
    def start(self, Ip_init, target):
        """Eager use: set the start image and target, clear the Adam state."""
        self.P0.copy_(Ip_init)
        self.target.copy_(target)
        self.P.copy_(self.P0)
        self.M.zero_()
        self.V.zero_()
        self.done = 0

    def advance(self, n: int):
        """Run the next n steps eagerly (steps done + 1 .. done + n)."""
        first = getattr(self, "done", 0)
        if first + n > self.steps:
            raise ValueError(f"{first} + {n} steps exceed the {self.steps} this object was built for")
        for k in range(first, first + n):
            self._step(k)
        self.done = first + n
        return self.P, self.history[:self.done]

    def save(self, path: str):
        """Checkpoint: Ip, the Adam moments, the target, the steps done, the seed and lr (.npz)."""
        import numpy as np

        np.savez(path, P=self.P.cpu().numpy(), M=self.M.cpu().numpy(), V=self.V.cpu().numpy(),
                 target=self.target.cpu().numpy(), history=self.history.cpu().numpy(),
                 done=getattr(self, "done", 0), seed=self.seed, lr=self.lr)

    def resume(self, path: str):
        """Restore a checkpoint written by save(); advance() then continues
        with the next step's Philox key and Adam step number."""
        import numpy as np
        import torch

        z = np.load(path)
        if int(z["seed"]) != self.seed or float(z["lr"]) != self.lr:
            raise ValueError("checkpoint seed or learning rate differs from this compensation")
        for name in ("P", "M", "V", "target"):
            getattr(self, name).copy_(torch.from_numpy(z[name]))
        self.history.copy_(torch.from_numpy(z["history"]))
        self.done = int(z["done"])

    def run(self, Ip_init, target):
        """Compensate towards `target` (Hc x Wc x 3) from `Ip_init` (Hp x Wp x
        3); returns (Ip*, per-step losses) as device tensors."""
        self.P0.copy_(Ip_init)
        self.target.copy_(target)
        if self.graph is not None:
            self.graph.replay()
        else:
            self._loop()
        return self.P, self.history
