"""Scene-parameter fitting (Eq. 9): estimate the BRDF maps and the projector
/ camera responses from K projected images and their captures,

    theta* = argmin (1/K) sum_i |D(R(Ip_i, theta)) - Ic_i| + lambda L(m),

with |.| the L1 norm (a mean over the pixels and channels of the K pairs),
L(m) the total variation of the BRDF maps (albedo, roughness and, with the
principled material, metallic), and D the optional cross-bilateral
denoiser of Eq. 11.  theta = albedo, roughness, gamma_p, gamma_c and the
white balance w, plus the metallic map and the normal map Vn when they are
given (the principled material of Sec. 3.2), and the camera pose Rc, tc
when a starting pose is given (``pose.PoseRefine``: one Adam step on the
pose after each step on the other parameters, its gradient from the pose
adjoint, or from central differences with the principled material); the gains
Gp and Gc stay at their given constants (Sec. 3.2).  Each step renders
every pair with a fresh Philox key, accumulates the path-replay gradients
of all pairs, adds the total-variation gradient and takes one Adam step per
parameter group, each followed by the clamp to the group's range: albedo [0, 1], roughness
[0.01, 1], metallic [0, 1], normal map [0, 1]^3 (Sec. 4.3), gamma_p [2, 3],
gamma_c [1/3, 1], w [0.2, 2.5] (Sec. 3.2).

Without the denoiser each pair's render, L1 term and adjoint are one call
that traces its paths once (``Context.render_loss_backward``); with it, the
render keeps its path records and the adjoint sweeps them.  ``fused=False``
makes separate calls that trace twice.  The principled material takes the
same routes (``render_loss_backward_principled``; with the denoiser, the
principled render keeps its records).  Every step
runs in the library's kernels; the only host traffic per step is reading
back the 11 response parameters the next renders take by value (and, with
the pose, its data terms and its 18-number gradient, or the 13 K data terms
of its differences).
"""
from __future__ import annotations

from . import dpcs
from .autograd import params_vector, with_vector  # noqa: F401  (re-exported for callers of the fit)

PARAM_RANGES = {"gamma_p": (slice(0, 3), 2.0, 3.0), "gamma_c": (slice(4, 7), 1.0 / 3.0, 1.0),
                "wb": (slice(8, 11), 0.2, 2.5)}
ROUGH_MIN = 0.01


class SceneFit:
    """Device state of one fit: the parameters, their Adam moments and the
    per-pair buffers.  ``pairs`` is a list of (Ip, Ic) device tensors."""

    def __init__(self, ctx: dpcs.Context, scene: int, view: dpcs.DpcsView, params0: dpcs.DpcsParams, albedo0, rough0,
                 pairs, spp: int, bounces: int, lr_tex: float = 2e-2, lr_params: float = 1e-2, tv_weight: float = 0.0,
                 denoise: dpcs.DpcsDenoiseParams | None = None, fit_params: bool = True, seed: int = 0,
                 fused: bool = True, metallic0=None, normal0=None, pose_xi0=None, pose_lr: float = 1e-3,
                 pose_gradient: str | None = None, pose_edge_spp: int = 16):
        import torch

        self.ctx, self.scene, self.view = ctx, scene, view
        self.pairs = list(pairs)
        self.K = len(self.pairs)
        self.spp, self.bounces, self.seed = int(spp), int(bounces), int(seed)
        self.lr_tex, self.lr_params, self.tv_weight = float(lr_tex), float(lr_params), float(tv_weight)
        self.denoise, self.fit_params, self.fused = denoise, bool(fit_params), bool(fused)
        dev = ctx.device
        f32 = torch.float32
        self.albedo = albedo0.clone().contiguous()
        self.rough = rough0.clone().contiguous()
        # principled material: metallic (Ht, Wt) and normal map (Ht, Wt, 3), each optional
        self.principled = metallic0 is not None or normal0 is not None
        self.metallic = None if metallic0 is None else metallic0.clone().contiguous()
        self.normal = None if normal0 is None else normal0.clone().contiguous()
        self.gM = None if self.metallic is None else torch.zeros_like(self.metallic)
        self.gN = None if self.normal is None else torch.zeros_like(self.normal)
        if self.metallic is not None:
            self.mM, self.vM = torch.zeros_like(self.metallic), torch.zeros_like(self.metallic)
        if self.normal is not None:
            self.mN, self.vN = torch.zeros_like(self.normal), torch.zeros_like(self.normal)
        self.params = params0
        self.pvec = torch.tensor(params_vector(params0), dtype=f32, device=dev)
        self.gA, self.gR = torch.zeros_like(self.albedo), torch.zeros_like(self.rough)
        self.gP = torch.zeros(11, dtype=f32, device=dev)
        self.mA, self.vA = torch.zeros_like(self.albedo), torch.zeros_like(self.albedo)
        self.mR, self.vR = torch.zeros_like(self.rough), torch.zeros_like(self.rough)
        self.mP, self.vP = torch.zeros(11, dtype=f32, device=dev), torch.zeros(11, dtype=f32, device=dev)
        img = (view.Hc, view.Wc, 3)
        self.Ic, self.Ec = torch.empty(img, dtype=f32, device=dev), torch.empty(img, dtype=f32, device=dev)
        self.dIc = torch.empty(img, dtype=f32, device=dev)
        if denoise is not None:
            self.guide = torch.empty((view.Hc, view.Wc, 8), dtype=f32, device=dev)
            self.D, self.dD = torch.empty(img, dtype=f32, device=dev), torch.empty(img, dtype=f32, device=dev)
            self.wsum = torch.empty((view.Hc, view.Wc), dtype=f32, device=dev)
        # camera pose (Rc, tc): when pose_xi0 is given, every step ends with one
        # pose step (pose.PoseRefine) on the updated maps, and the renders use
        # the scene moved to the current pose with the matching view
        self.pose = None
        if pose_xi0 is not None:
            from .pose import PoseRefine

            self.pose = PoseRefine(ctx, scene, view, params0, self.albedo, self.rough, self.pairs, spp, bounces,
                                   seed=seed + 7919, xi0=pose_xi0, lr=pose_lr, metallic=self.metallic,
                                   normal=self.normal, gradient=pose_gradient, edge_spp=pose_edge_spp)
            self.view = self.pose.apply(pose_xi0)
        # K data terms, TV(albedo), TV(rough) [, TV(metallic)]
        self.losses = torch.zeros(self.K + 2 + (self.metallic is not None), dtype=f32, device=dev)
        self.scale = 1.0 / (self.K * view.Hc * view.Wc * 3)
        self.k = 0

    def step(self):
        """One Adam step over all K pairs; returns the device loss terms."""
        c = self.ctx
        self.k += 1
        self.gA.zero_()
        self.gR.zero_()
        self.gP.zero_()
        for g in (self.gM, self.gN):
            if g is not None:
                g.zero_()
        if self.denoise is not None:  # the guide follows the current albedo; its weights are not differentiated
            c.gbuffer(self.scene, self.albedo, self.rough, self.view, guide=self.guide)
        for i, (Ip, target) in enumerate(self.pairs):
            s = self.seed + (self.k - 1) * self.K + i
            if self.principled:
                self._pair_principled(Ip, target, s, i)
                continue
            if self.denoise is None and self.fused:  # render, L1 term and adjoint in one trace of the paths
                c.render_loss_backward(self.scene, self.albedo, self.rough, Ip, self.view, self.params, self.spp,
                                       self.bounces, s, target, self.losses[i:i + 1], loss_kind=1, scale=self.scale,
                                       Ic=self.Ic, Ec=self.Ec, dAlbedo=self.gA, dRough=self.gR,
                                       dParams=self.gP if self.fit_params else None)
                continue
            keep = self.fused  # the denoiser couples pixels: keep the paths for the adjoint
            c.render(self.scene, self.albedo, self.rough, Ip, self.view, self.params, self.spp, self.bounces, s,
                     Ic=self.Ic, Ec=self.Ec, keep=keep)
            if self.denoise is None:
                c.l1_loss(self.Ic, target, self.dIc, self.losses[i:i + 1], scale=self.scale)
            else:
                c.denoise(self.Ic, self.guide, self.denoise, out=self.D, wsum=self.wsum)
                c.l1_loss(self.D, target, self.dD, self.losses[i:i + 1], scale=self.scale)
                self.dIc.zero_()
                c.denoise_backward(self.dD, self.guide, self.wsum, self.denoise, dIc=self.dIc)
            c.render_backward(self.scene, self.albedo, self.rough, Ip, self.view, self.params, self.spp, self.bounces,
                              s, self.Ec, self.Ic, self.dIc, dAlbedo=self.gA, dRough=self.gR,
                              dParams=self.gP if self.fit_params else None, kept=keep)
        K = self.K
        c.tv_loss(self.albedo, self.gA, self.losses[K:K + 1], self.tv_weight)
        c.tv_loss(self.rough, self.gR, self.losses[K + 1:K + 2], self.tv_weight)
        if self.metallic is not None:
            c.tv_loss(self.metallic, self.gM, self.losses[K + 2:K + 3], self.tv_weight)
        c.adam(self.albedo, self.gA, self.mA, self.vA, self.k, lr=self.lr_tex, lo=0.0, hi=1.0)
        c.adam(self.rough, self.gR, self.mR, self.vR, self.k, lr=self.lr_tex, lo=ROUGH_MIN, hi=1.0)
        if self.metallic is not None:
            c.adam(self.metallic, self.gM, self.mM, self.vM, self.k, lr=self.lr_tex, lo=0.0, hi=1.0)
        if self.normal is not None:
            c.adam(self.normal, self.gN, self.mN, self.vN, self.k, lr=self.lr_tex, lo=0.0, hi=1.0)
        if self.fit_params:
            for sl, lo, hi in PARAM_RANGES.values():
                c.adam(self.pvec[sl], self.gP[sl], self.mP[sl], self.vP[sl], self.k, lr=self.lr_params, lo=lo, hi=hi)
            self.params = with_vector(self.params, self.pvec.cpu().tolist())
        if self.pose is not None:
            from .pose import posed_view

            self.pose.params = self.params
            self.pose.step()
            self.view = posed_view(self.pose.view, *self.pose.pose())
        return self.losses

    def _pair_principled(self, Ip, target, s, i):
        """One pair with the principled material: render, (D,) L1, adjoint with every map's gradient."""
        c = self.ctx
        if self.denoise is None and self.fused:  # one trace of the paths
            c.render_loss_backward_principled(self.scene, self.albedo, self.rough, self.metallic, self.normal, Ip,
                                              self.view, self.params, self.spp, self.bounces, s, target,
                                              self.losses[i:i + 1], loss_kind=1, scale=self.scale, Ic=self.Ic,
                                              Ec=self.Ec, dAlbedo=self.gA, dRough=self.gR, dMetallic=self.gM,
                                              dNormal=self.gN, dParams=self.gP if self.fit_params else None)
            return
        keep = self.fused  # with the denoiser: keep the paths for the adjoint
        c.render_principled(self.scene, self.albedo, self.rough, self.metallic, self.normal, Ip, self.view,
                            self.params, self.spp, self.bounces, s, Ic=self.Ic, Ec=self.Ec, keep=keep)
        if self.denoise is None:
            c.l1_loss(self.Ic, target, self.dIc, self.losses[i:i + 1], scale=self.scale)
        else:
            c.denoise(self.Ic, self.guide, self.denoise, out=self.D, wsum=self.wsum)
            c.l1_loss(self.D, target, self.dD, self.losses[i:i + 1], scale=self.scale)
            self.dIc.zero_()
            c.denoise_backward(self.dD, self.guide, self.wsum, self.denoise, dIc=self.dIc)
        c.render_backward_principled(self.scene, self.albedo, self.rough, self.metallic, self.normal, Ip, self.view,
                                     self.params, self.spp, self.bounces, s, self.Ec, self.Ic, self.dIc,
                                     dAlbedo=self.gA, dRough=self.gR, dMetallic=self.gM, dNormal=self.gN,
                                     dParams=self.gP if self.fit_params else None, kept=keep)

    def run(self, steps: int):
        """`steps` Adam steps; returns the per-step total loss (host list)."""
        import torch

        hist = torch.zeros(steps, dtype=torch.float32, device=self.ctx.device)
        for k in range(steps):
            hist[k] = self.step().sum()
        return hist.cpu().tolist()
