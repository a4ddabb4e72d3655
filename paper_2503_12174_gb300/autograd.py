"""The renderer as a torch.autograd.Function: Ic = R(Ip, theta) (Eq. 7) with
its path-replay adjoint as the backward, so that projector compensation
(Eq. 13) and scene fitting (Eq. 9) can be written with torch optimisers.

    Ic = render(ctx, scene, albedo, rough, Ip, view, params, spp, bounces, seed, pvec=None,
                metallic=None, normal=None, pose=None, pose_R0=None, pose_t0=None,
                edge_spp=16, sil_spp=16)

``albedo`` (Ht x Wt x 3), ``rough`` (Ht x Wt) and ``Ip`` (Hp x Wp x 3) are
device tensors; ``pvec`` (11 floats: gamma_p(3), Gp, gamma_c(3), Gc, w(3)),
when given, replaces the response parameters of ``params`` and receives their
gradient.  ``metallic`` (Ht x Wt) and ``normal`` (Ht x Wt x 3), when either
is given, select the principled material of Sec. 3.2
(dpcs_render_principled) and receive their gradients too.  The backward
asks the library only for the gradients autograd needs: without albedo or
roughness gradients the replay skips the texture scatters.  Both passes run in the library's kernels; each call renders with
Philox key ``seed``, and the backward re-traces the same paths.

``pose`` (6 values xi = (omega, delta) around the pose (``pose_R0``,
``pose_t0``), as in ``pose.pose_of``), when given, is the camera pose (Rc,
tc) of Sec. 3.2: the forward moves the scene to it (``dpcs_scene_transform``;
the scene stays there after the call) and renders with the posed view, and
the backward gives its gradient by the pose adjoint (``dpcs_pose_backward``,
``edge_spp`` / ``sil_spp`` samples per pixel edge / silhouette edge, its paths
under ``pose.adjoint_key(seed)``) projected on the parameters' twists.

The backward re-traces the scene as it is when the backward runs, so moving
the scene between a render and its backward (``Context.update``,
``Context.transform``, or another render with a pose) makes that backward
raise instead of returning the gradient of another geometry.
"""
from __future__ import annotations

from . import dpcs


def params_vector(p: dpcs.DpcsParams):
    """[gamma_p(3), Gp, gamma_c(3), Gc, wb(3)] -- the layout of dParams."""
    return list(p.gamma_p) + [p.gain_p] + list(p.gamma_c) + [p.gain_c] + list(p.wb)


def with_vector(p: dpcs.DpcsParams, v) -> dpcs.DpcsParams:
    """A copy of p with its response parameters taken from v (params_vector layout)."""
    q = dpcs.DpcsParams.from_buffer_copy(bytes(p))
    q.gamma_p[:] = [float(x) for x in v[0:3]]
    q.gain_p = float(v[3])
    q.gamma_c[:] = [float(x) for x in v[4:7]]
    q.gain_c = float(v[7])
    q.wb[:] = [float(x) for x in v[8:11]]
    return q


def _function():
    import torch

    class DPCSRender(torch.autograd.Function):
        @staticmethod
        def forward(fctx, albedo, rough, Ip, pvec, metallic, normal, pose_xi, ctx, scene, view, params, spp, bounces,
                    seed, frame, edge_spp, sil_spp):
            p = params if pvec is None else with_vector(params, pvec.detach().cpu().tolist())
            xi = None
            if pose_xi is not None:
                from . import pose as pose_mod

                xi = pose_xi.detach().cpu().double().numpy()
                R, t = pose_mod.pose_of(xi, *frame)
                ctx.transform(scene, R, t)
                view = pose_mod.posed_view(view, R, t)
            Ec = torch.empty((view.Hc, view.Wc, 3), dtype=torch.float32, device=ctx.device)
            principled = metallic is not None or normal is not None
            if principled:
                Ic, _ = ctx.render_principled(scene, albedo, rough, metallic, normal, Ip, view, p, spp, bounces, seed,
                                              Ec=Ec)
            else:
                Ic, _ = ctx.render(scene, albedo, rough, Ip, view, p, spp, bounces, seed, Ec=Ec)
            fctx.save_for_backward(albedo, rough, Ip, Ec, Ic, metallic, normal)
            fctx.moves = ctx.scene_moves(scene)
            fctx.meta = (ctx, scene, view, p, spp, bounces, seed, pvec is not None, principled)
            fctx.pose = (xi, frame, edge_spp, sil_spp, pose_xi)
            return Ic

        @staticmethod
        def backward(fctx, dIc):
            albedo, rough, Ip, Ec, Ic, metallic, normal = fctx.saved_tensors
            ctx, scene, view, p, spp, bounces, seed, has_pvec, principled = fctx.meta
            if ctx.scene_moves(scene) != fctx.moves:
                raise RuntimeError("dpcs autograd: the scene was moved (update or transform, another posed render "
                                   "included) after this render; its backward would re-trace the moved scene")
            need = fctx.needs_input_grad
            dA = torch.zeros_like(albedo) if need[0] else None
            dR = torch.zeros_like(rough) if need[1] else None
            dIp = torch.zeros_like(Ip) if need[2] else None
            dP = torch.zeros(11, dtype=torch.float32, device=ctx.device) if has_pvec and need[3] else None
            dM = torch.zeros_like(metallic) if metallic is not None and need[4] else None
            dN = torch.zeros_like(normal) if normal is not None and need[5] else None
            g = dIc.to(torch.float32).contiguous()
            if principled and any(x is not None for x in (dA, dR, dIp, dP, dM, dN)):
                ctx.render_backward_principled(scene, albedo, rough, metallic, normal, Ip, view, p, spp, bounces, seed,
                                               Ec, Ic, g, dIp=dIp, dAlbedo=dA, dRough=dR, dMetallic=dM, dNormal=dN,
                                               dParams=dP)
            elif any(x is not None for x in (dA, dR, dIp, dP)):
                ctx.render_backward(scene, albedo, rough, Ip, view, p, spp, bounces, seed, Ec, Ic, g, dIp=dIp,
                                    dAlbedo=dA, dRough=dR, dParams=dP)
            dX = None
            xi, frame, edge_spp, sil_spp, pose_xi = fctx.pose
            if xi is not None and need[6]:
                from . import pose as pose_mod

                key = pose_mod.adjoint_key(seed)
                if principled:
                    W = ctx.pose_backward_principled(scene, albedo, rough, metallic, normal, Ip, view, p, spp,
                                                     bounces, key, Ec, Ic, g, edge_spp, sil_spp)
                else:
                    W = ctx.pose_backward(scene, albedo, rough, Ip, view, p, spp, bounces, key, Ec, Ic, g, edge_spp,
                                          sil_spp)
                gx = pose_mod.project(W.cpu().numpy(), pose_mod.twists(xi, *frame))
                dX = torch.as_tensor(gx, dtype=pose_xi.dtype, device=pose_xi.device)
            return dA, dR, dIp, dP, dM, dN, dX, None, None, None, None, None, None, None, None, None, None

    return DPCSRender


_DPCSRender = None


def render(ctx: dpcs.Context, scene: int, albedo, rough, Ip, view: dpcs.DpcsView, params: dpcs.DpcsParams,
           spp: int, bounces: int, seed: int, pvec=None, metallic=None, normal=None, pose=None, pose_R0=None,
           pose_t0=None, edge_spp: int = 16, sil_spp: int = 16):
    """Differentiable Ic = R(Ip, theta); see the module docstring."""
    global _DPCSRender
    if _DPCSRender is None:
        _DPCSRender = _function()
    return _DPCSRender.apply(albedo, rough, Ip, pvec, metallic, normal, pose, ctx, scene, view, params, int(spp),
                             int(bounces), int(seed), (pose_R0, pose_t0), int(edge_spp), int(sil_spp))
