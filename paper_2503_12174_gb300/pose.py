"""Camera-pose refinement: the rotation Rc and translation tc that Sec. 3.2
lists among the scene parameters theta of Eq. 9 and refines slightly.

Renders put the camera at the origin (Eq. 6).  A camera at pose (Rc, tc)
sees a world point x at Rc x + tc, so the pose is applied to the scene: the
mesh moves by ``dpcs_scene_transform`` and the projector extrinsics become
Rp' = Rp Rc^T, tp' = tp - Rp' tc (``posed_view``).

The pose is xi = (omega, delta) around a starting pose (R0, t0):
Rc = exp([omega]x) R0 (Rodrigues), tc = t0 + delta.  Each pose parameter
moves the posed scene with a twist (a, b) (``twists``).  Its gradient comes
either from the adjoint (``dpcs_pose_backward``: dLoss/d(a, b) with the
interior, pixel-edge and silhouette terms of the box-filtered pixel means,
one call per pair, projected on the six twists) or from central differences
with common random numbers (every evaluation renders with the same Philox
keys; six parameters cost twelve renders per pair).  Both include what the
image does where silhouettes cross pixels -- the visibility terms that path
replay with detached sampling (the adjoint of every other parameter) leaves
out.
"""
from __future__ import annotations

import math

import numpy as np

from . import dpcs


def rotation(omega) -> np.ndarray:
    """exp([omega]x): rotation by |omega| about omega / |omega| (Rodrigues)."""
    w = np.asarray(omega, np.float64).reshape(3)
    th = float(np.linalg.norm(w))
    K = np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])
    if th < 1e-8:  # series to second order
        return np.eye(3) + K + 0.5 * (K @ K)
    return np.eye(3) + (math.sin(th) / th) * K + ((1.0 - math.cos(th)) / (th * th)) * (K @ K)


def pose_of(xi, R0=None, t0=None):
    """(Rc, tc) of pose parameters xi = (omega, delta) around (R0, t0)."""
    xi = np.asarray(xi, np.float64).reshape(6)
    R0 = np.eye(3) if R0 is None else np.asarray(R0, np.float64)
    t0 = np.zeros(3) if t0 is None else np.asarray(t0, np.float64)
    return rotation(xi[:3]) @ R0, t0 + xi[3:]


def left_jacobian(omega) -> np.ndarray:
    """J with d/ds exp([omega + s e]x) = [J e]x exp([omega]x) at s = 0 (the
    left Jacobian of the rotation-vector map)."""
    w = np.asarray(omega, np.float64).reshape(3)
    th = float(np.linalg.norm(w))
    K = np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])
    if th < 1e-5:  # series: 1/2 - th^2/24 and 1/6 - th^2/120
        return np.eye(3) + (0.5 - th * th / 24.0) * K + (1.0 / 6.0 - th * th / 120.0) * (K @ K)
    return np.eye(3) + ((1.0 - math.cos(th)) / (th * th)) * K + ((th - math.sin(th)) / (th ** 3)) * (K @ K)


def twists(xi, R0=None, t0=None) -> np.ndarray:
    """(6, 6): for each pose parameter, the motion (a, b) of the posed scene
    in the camera frame at pose xi, a point y moving with a x y + b.  The
    scene sits at y = exp([omega]x) R0 x + t0 + delta: rotation parameter k
    turns it about t = t0 + delta with a = J(omega) e_k (b = -a x t);
    translation parameter k moves it with a = 0, b = e_k."""
    xi = np.asarray(xi, np.float64).reshape(6)
    t = (np.zeros(3) if t0 is None else np.asarray(t0, np.float64)) + xi[3:]
    J = left_jacobian(xi[:3])
    out = np.zeros((6, 6))
    for k in range(3):
        a = J[:, k]
        out[k, :3] = a
        out[k, 3:] = -np.cross(a, t)
        out[3 + k, 3 + k] = 1.0
    return out


def posed_extrinsics(Rp, tp, R, t):
    """Projector extrinsics seen from a camera at pose (R, t): (Rp R^T, tp - Rp R^T t)."""
    Rp2 = np.asarray(Rp, np.float64).reshape(3, 3) @ np.asarray(R, np.float64).T
    return Rp2, np.asarray(tp, np.float64).reshape(3) - Rp2 @ np.asarray(t, np.float64).reshape(3)


def posed_view(view: dpcs.DpcsView, R, t) -> dpcs.DpcsView:
    """``view`` with its projector extrinsics moved for a camera at pose (R, t)."""
    Rp2, tp2 = posed_extrinsics(np.array(view.Rp[:]), np.array(view.tp[:]), R, t)
    return dpcs.make_view(np.array(view.Kc[:]).reshape(3, 3), view.Hc, view.Wc,
                          np.array(view.Kp[:]).reshape(3, 3), Rp2, tp2, view.Hp, view.Wp)


def central_differences(loss, xi, h):
    """Gradient of ``loss`` (a callable on 6-vectors returning a float) at xi
    by central differences with steps h (6 values): 12 evaluations."""
    xi = np.asarray(xi, np.float64).reshape(6)
    h = np.broadcast_to(np.asarray(h, np.float64), (6,))
    g = np.zeros(6)
    for k in range(6):
        e = np.zeros(6)
        e[k] = h[k]
        g[k] = (loss(xi + e) - loss(xi - e)) / (2.0 * h[k])
    return g


def adjoint_key(seed: int) -> int:
    """Philox key of the pose adjoint's paths for a render with key ``seed``:
    the same low word, the high word moved by one, so that the two sets of
    samples are independent."""
    return (int(seed) + (1 << 32)) & (2**64 - 1)


def project(wrench, tw) -> np.ndarray:
    """Gradient of each pose parameter from dLoss/d(a, b): ``wrench`` is the
    (3, 6) or (6,) output of ``dpcs_pose_backward`` (its terms are summed),
    ``tw`` the (K, 6) twists of the parameters."""
    w = np.asarray(wrench, np.float64)
    w = w.reshape(-1, 6).sum(axis=0)
    return np.asarray(tw, np.float64).reshape(-1, 6) @ w


class PoseRefine:
    """Refines the camera pose against K projector/capture pairs by Adam on
    the gradient of the Eq. 9 data term (the mean L1 error; the other scene
    parameters stay fixed).  ``pairs`` is a list of (Ip, Ic) device tensors;
    ``metallic`` / ``normal`` select the principled material.

    ``gradient="adjoint"`` (the default, either material): each step moves
    the scene to the pose, and per pair renders, takes the L1 term and calls
    ``dpcs_pose_backward`` (``edge_spp`` and ``sil_spp`` samples per pixel
    edge and per silhouette edge), then one Adam step on xi.  Its noise
    falls with the pixel count: small images want more edge samples (64 at
    48 x 48 pixels recovers the pose about as central differences do at
    higher cost; 16 suffices at 256 x 256).
    ``gradient="differences"``: thirteen pose evaluations per step, each a scene transform, K renders and
    K L1 terms, at xi and at xi +- h e_k."""

    def __init__(self, ctx: dpcs.Context, scene: int, view: dpcs.DpcsView, params: dpcs.DpcsParams, albedo, rough,
                 pairs, spp: int, bounces: int, seed: int = 0, xi0=None, R0=None, t0=None, h_rot: float = 1e-3,
                 h_trans: float = 1e-3, lr: float = 1e-3, metallic=None, normal=None, gradient: str | None = None,
                 edge_spp: int = 16, sil_spp: int = 16):
        import torch

        self.ctx, self.scene, self.view, self.params = ctx, scene, view, params
        self.albedo, self.rough, self.metallic, self.normal = albedo, rough, metallic, normal
        self.principled = metallic is not None or normal is not None
        if gradient is None:
            gradient = "adjoint"
        if gradient not in ("adjoint", "differences"):
            raise ValueError("gradient must be 'adjoint' or 'differences'")
        self.gradient = gradient
        self.edge_spp, self.sil_spp = int(edge_spp), int(sil_spp)
        self.pairs = list(pairs)
        self.K = len(self.pairs)
        self.spp, self.bounces, self.seed = int(spp), int(bounces), int(seed)
        self.R0 = np.eye(3) if R0 is None else np.asarray(R0, np.float64)
        self.t0 = np.zeros(3) if t0 is None else np.asarray(t0, np.float64)
        self.h = np.array([h_rot] * 3 + [h_trans] * 3)
        self.lr = float(lr)
        dev = ctx.device
        f32 = torch.float32
        self.xi = torch.tensor(np.zeros(6) if xi0 is None else np.asarray(xi0, np.float64), dtype=f32, device=dev)
        self.g = torch.zeros(6, dtype=f32, device=dev)
        self.m, self.v = torch.zeros(6, dtype=f32, device=dev), torch.zeros(6, dtype=f32, device=dev)
        img = (view.Hc, view.Wc, 3)
        self.Ic = torch.empty(img, dtype=f32, device=dev)
        self.Ec = torch.empty(img, dtype=f32, device=dev)
        self.dIc = torch.empty(img, dtype=f32, device=dev)
        self.wrench = torch.zeros((3, 6), dtype=torch.float64, device=dev)
        self.terms = torch.zeros((13, self.K), dtype=f32, device=dev)  # per evaluation and pair
        self.scale = 1.0 / (self.K * view.Hc * view.Wc * 3)
        self.k = 0

    def apply(self, xi):
        """Move the scene to pose xi; returns the matching view."""
        R, t = pose_of(xi, self.R0, self.t0)
        self.ctx.transform(self.scene, R, t)
        return posed_view(self.view, R, t)

    def _key(self, i: int) -> int:
        return self.seed + (self.k - 1) * self.K + i  # the same keys for every evaluation of a step

    def _evaluate(self, xi, row: int):
        c = self.ctx
        v = self.apply(xi)
        for i, (Ip, target) in enumerate(self.pairs):
            s = self._key(i)
            if self.metallic is not None or self.normal is not None:
                c.render_principled(self.scene, self.albedo, self.rough, self.metallic, self.normal, Ip, v,
                                    self.params, self.spp, self.bounces, s, Ic=self.Ic)
            else:
                c.render(self.scene, self.albedo, self.rough, Ip, v, self.params, self.spp, self.bounces, s,
                         Ic=self.Ic)
            c.l1_loss(self.Ic, target, self.dIc, self.terms[row, i:i + 1], scale=self.scale)

    def _adjoint(self, xi):
        """Data term and its pose gradient at xi by dpcs_pose_backward.  The
        adjoint traces its paths under another Philox key than the render
        whose L1 residual it weights: with the render's own samples the
        interior term (each sample's value times the change of its pixel
        footprint) would correlate with sign(Ic - target) and carry a bias of
        about the loss itself times the mean footprint change, which does
        not vanish at the true pose."""
        c = self.ctx
        v = self.apply(xi)
        self.wrench.zero_()
        for i, (Ip, target) in enumerate(self.pairs):
            s = self._key(i)
            if self.principled:
                c.render_principled(self.scene, self.albedo, self.rough, self.metallic, self.normal, Ip, v,
                                    self.params, self.spp, self.bounces, s, Ic=self.Ic, Ec=self.Ec)
            else:
                c.render(self.scene, self.albedo, self.rough, Ip, v, self.params, self.spp, self.bounces, s,
                         Ic=self.Ic, Ec=self.Ec)
            c.l1_loss(self.Ic, target, self.dIc, self.terms[12, i:i + 1], scale=self.scale)
            if self.principled:
                c.pose_backward_principled(self.scene, self.albedo, self.rough, self.metallic, self.normal, Ip, v,
                                           self.params, self.spp, self.bounces, adjoint_key(s), self.Ec, self.Ic,
                                           self.dIc, self.edge_spp, self.sil_spp, wrench=self.wrench)
            else:
                c.pose_backward(self.scene, self.albedo, self.rough, Ip, v, self.params, self.spp, self.bounces,
                                adjoint_key(s), self.Ec, self.Ic, self.dIc, self.edge_spp, self.sil_spp,
                                wrench=self.wrench)
        g = project(self.wrench.cpu().numpy(), twists(xi, self.R0, self.t0))
        return float(self.terms[12].sum().cpu()), g

    def step(self) -> float:
        """One Adam step on the pose; returns the data term at the pose the step started from."""
        import torch

        self.k += 1
        xi = self.xi.cpu().numpy().astype(np.float64)
        if self.gradient == "adjoint":
            L0, g = self._adjoint(xi)
        else:
            self._evaluate(xi, 12)
            for k in range(6):
                e = np.zeros(6)
                e[k] = self.h[k]
                self._evaluate(xi + e, 2 * k)
                self._evaluate(xi - e, 2 * k + 1)
            L = self.terms.sum(dim=1).cpu().numpy().astype(np.float64)
            g = (L[0:12:2] - L[1:12:2]) / (2.0 * self.h)
            L0 = float(L[12])
        self.g.copy_(torch.from_numpy(g.astype(np.float32)))
        self.ctx.adam(self.xi, self.g, self.m, self.v, self.k, lr=self.lr, lo=-1.0, hi=1.0)
        self.apply(self.xi.cpu().numpy().astype(np.float64))
        return L0

    def pose(self):
        """Current (Rc, tc)."""
        return pose_of(self.xi.cpu().numpy().astype(np.float64), self.R0, self.t0)
