"""Host logic of camera-pose refinement, on the CPU against a stand-in for
the library context whose data term is a known smooth function of the pose:
the central-difference gradient pairs its thirteen evaluations correctly
and renders all of them with the step's keys; the adjoint route passes the
adjoint's own key and projects the summed wrench on the twists; the step
moves the scene to the updated pose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2503_12174_gb300 import dpcs, pose  # noqa: E402

T_STAR = np.array([0.02, -0.01, 0.03])
R_STAR = pose.rotation([0.02, 0.01, -0.015])
WRENCH = np.arange(18, dtype=np.float64).reshape(3, 6) / 10.0 - 0.8


def phi(R, t):
    """The stand-in's data term of a pose (the same for every pair)."""
    return 1.0 + 0.5 * float(np.sum((np.asarray(t) - T_STAR) ** 2)) + 0.5 * float(np.sum((np.asarray(R) - R_STAR) ** 2))


class FakeContext:
    def __init__(self):
        self.device = torch.device("cpu")
        self.R, self.t = np.eye(3), np.zeros(3)
        self.keys, self.adjoint_keys, self.transforms = [], [], []

    def transform(self, scene, R, t):
        self.R, self.t = np.asarray(R, np.float64), np.asarray(t, np.float64)
        self.transforms.append((self.R.copy(), self.t.copy()))

    def render(self, scene, albedo, rough, Ip, view, params, spp, bounces, seed, Ic=None, Ec=None):
        self.keys.append(seed)
        Ic.fill_(phi(self.R, self.t))
        if Ec is not None:
            Ec.copy_(Ic)

    def l1_loss(self, Ic, target, dIc, loss, scale=1.0):
        r = Ic.double() - target.double()
        loss.fill_(float(scale * r.abs().sum()))
        dIc.copy_(scale * torch.sign(r))

    def pose_backward(self, scene, albedo, rough, Ip, view, params, spp, bounces, key, Ec, Ic, dIc, edge_spp,
                      sil_spp, wrench=None):
        self.adjoint_keys.append((key, edge_spp, sil_spp))
        wrench += torch.from_numpy(WRENCH)

    def adam(self, p, g, m, v, step, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8, lo=0.0, hi=1.0):
        p.sub_(lr * torch.sign(g)).clamp_(lo, hi)


def _refine(ctx, gradient, xi0):
    view = dpcs.DpcsView()
    view.Hc, view.Wc, view.Hp, view.Wp = 3, 4, 4, 4
    for i in range(3):
        view.Kc[4 * i] = view.Kp[4 * i] = view.Rp[4 * i] = 1.0
    pairs = [(torch.zeros((4, 4, 3)), torch.zeros((3, 4, 3))) for _ in range(2)]
    return pose.PoseRefine(ctx, 0, view, dpcs.DpcsParams(), None, None, pairs, 4, 2, seed=30, xi0=xi0,
                           gradient=gradient, lr=1e-3, edge_spp=5, sil_spp=7)


def test_central_differences_pair_their_evaluations():
    xi0 = np.array([0.01, -0.02, 0.005, 0.01, 0.0, -0.02])
    ctx = FakeContext()
    pr = _refine(ctx, "differences", xi0)
    L0 = pr.step()
    assert L0 == pytest.approx(phi(*pose.pose_of(xi0)), rel=1e-6)
    # 13 evaluations of 2 pairs, every one with the step's keys
    assert ctx.keys == [30, 31] * 13
    h = pr.h
    expect = np.array([(phi(*pose.pose_of(xi0 + h[k] * e)) - phi(*pose.pose_of(xi0 - h[k] * e))) / (2 * h[k])
                       for k, e in enumerate(np.eye(6))])
    np.testing.assert_allclose(pr.g.numpy(), expect, rtol=0, atol=2e-4)
    assert np.abs(expect).min() > 1e-3
    # the step moves the scene to the updated pose: xi - lr sign(g)
    xi1 = xi0 - 1e-3 * np.sign(expect)
    np.testing.assert_allclose(pr.xi.numpy(), xi1, rtol=0, atol=1e-7)
    R1, t1 = pose.pose_of(pr.xi.numpy().astype(np.float64))
    np.testing.assert_allclose(ctx.transforms[-1][0], R1, atol=1e-12)
    np.testing.assert_allclose(ctx.transforms[-1][1], t1, atol=1e-12)
    pr.step()
    assert ctx.keys[26:] == [32, 33] * 13  # the next step's keys


def test_adjoint_route_projects_the_summed_wrench():
    xi0 = np.array([0.004, 0.002, -0.003, 0.0, 0.01, 0.005])
    ctx = FakeContext()
    pr = _refine(ctx, "adjoint", xi0)
    L0 = pr.step()
    assert L0 == pytest.approx(phi(*pose.pose_of(xi0)), rel=1e-6)
    assert ctx.keys == [30, 31]
    assert ctx.adjoint_keys == [(pose.adjoint_key(30), 5, 7), (pose.adjoint_key(31), 5, 7)]
    expect = pose.project(2.0 * WRENCH, pose.twists(xi0))
    np.testing.assert_allclose(pr.g.numpy(), expect, rtol=1e-6)


def test_unknown_gradient_is_refused():
    with pytest.raises(ValueError):
        _refine(FakeContext(), "finite", np.zeros(6))
