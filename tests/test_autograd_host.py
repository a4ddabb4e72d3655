"""Host logic of the autograd wrapper, run on the CPU against a stand-in for
the library context (no GPU, no kernels): which gradients the backward asks
the library for, how the pose gradient is projected, and the refusal of a
backward whose scene was moved after its render."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2503_12174_gb300 import autograd, dpcs, pose  # noqa: E402


class FakeContext:
    """Records the calls the wrapper makes; Ic = 2 Ip, and the backward adds
    2 dIc to dIp (the image sizes of the view below are all 4 x 4)."""

    def __init__(self):
        self.device = torch.device("cpu")
        self.moves = {}
        self.calls = []

    def scene_moves(self, scene):
        return self.moves.get(scene, 0)

    def transform(self, scene, R, t):
        self.calls.append(("transform", np.asarray(R).copy(), np.asarray(t).copy()))
        self.moves[scene] = self.moves.get(scene, 0) + 1

    def update(self, scene, verts):
        self.moves[scene] = self.moves.get(scene, 0) + 1

    def render(self, scene, albedo, rough, Ip, view, p, spp, bounces, seed, Ec=None):
        self.calls.append(("render", view.Hc, seed))
        Ec.copy_(Ip)
        return 2.0 * Ip, Ec

    def render_backward(self, scene, albedo, rough, Ip, view, p, spp, bounces, seed, Ec, Ic, dIc, dIp=None,
                        dAlbedo=None, dRough=None, dParams=None):
        self.calls.append(("render_backward", dIp is not None, dAlbedo is not None, dRough is not None,
                           dParams is not None))
        if dIp is not None:
            dIp += 2.0 * dIc

    def pose_backward(self, scene, albedo, rough, Ip, view, p, spp, bounces, key, Ec, Ic, dIc, edge_spp, sil_spp):
        self.calls.append(("pose_backward", key, edge_spp, sil_spp))
        return torch.arange(1.0, 7.0)


def _inputs():
    view = dpcs.DpcsView()
    view.Hc = view.Wc = view.Hp = view.Wp = 4
    for i in range(3):
        view.Kc[4 * i] = view.Kp[4 * i] = view.Rp[4 * i] = 1.0
    albedo = torch.full((2, 2, 3), 0.5)
    rough = torch.full((2, 2), 0.5)
    Ip = torch.rand((4, 4, 3), generator=torch.Generator().manual_seed(0)).requires_grad_(True)
    return view, dpcs.DpcsParams(), albedo, rough, Ip


def test_backward_asks_only_for_the_gradients_autograd_needs():
    ctx = FakeContext()
    view, params, albedo, rough, Ip = _inputs()
    Ic = autograd.render(ctx, 7, albedo, rough, Ip, view, params, 4, 2, 11)
    W = torch.rand((4, 4, 3), generator=torch.Generator().manual_seed(1))
    (Ic * W).sum().backward()
    assert ctx.calls == [("render", 4, 11), ("render_backward", True, False, False, False)]
    np.testing.assert_allclose(Ip.grad.numpy(), 2.0 * W.numpy(), rtol=0, atol=0)


def test_backward_refuses_a_scene_moved_after_the_render():
    ctx = FakeContext()
    view, params, albedo, rough, Ip = _inputs()
    Ic = autograd.render(ctx, 7, albedo, rough, Ip, view, params, 4, 2, 11)
    ctx.update(7, None)
    with pytest.raises(RuntimeError, match="moved"):
        Ic.sum().backward()
    # another scene's moves do not matter
    Ic = autograd.render(ctx, 7, albedo, rough, Ip, view, params, 4, 2, 11)
    ctx.update(8, None)
    Ic.sum().backward()


def test_pose_gradient_and_a_second_posed_render_before_the_backward():
    ctx = FakeContext()
    view, params, albedo, rough, _ = _inputs()
    Ip = torch.rand((4, 4, 3), generator=torch.Generator().manual_seed(2))
    R0, t0 = pose.rotation([0.01, 0.0, -0.02]), np.array([0.0, 0.01, 0.0])
    x0 = np.array([0.003, -0.002, 0.001, 0.004, 0.0, -0.001])
    xi = torch.tensor(x0, dtype=torch.float64, requires_grad=True)
    Ic = autograd.render(ctx, 7, albedo, rough, Ip, view, params, 4, 2, 11, pose=xi, pose_R0=R0, pose_t0=t0,
                         edge_spp=3, sil_spp=5)
    R, t = pose.pose_of(x0, R0, t0)
    assert ctx.calls[0][0] == "transform"
    np.testing.assert_allclose(ctx.calls[0][1], R, rtol=0, atol=1e-15)
    np.testing.assert_allclose(ctx.calls[0][2], t, rtol=0, atol=1e-15)
    Ic.sum().backward()
    assert ctx.calls[-1] == ("pose_backward", pose.adjoint_key(11), 3, 5)
    expect = pose.project(np.arange(1.0, 7.0), pose.twists(x0, R0, t0))
    np.testing.assert_allclose(xi.grad.numpy(), expect, rtol=1e-12, atol=0)
    # two posed renders, then the first one's backward: the scene sits at the second pose
    a = autograd.render(ctx, 7, albedo, rough, Ip, view, params, 4, 2, 11, pose=xi, pose_R0=R0, pose_t0=t0)
    autograd.render(ctx, 7, albedo, rough, Ip, view, params, 4, 2, 12, pose=xi, pose_R0=R0, pose_t0=t0)
    with pytest.raises(RuntimeError, match="moved"):
        a.sum().backward()
