"""Host logic of the Eq. 9 fit, on the CPU against a stand-in for the library
context: Philox keys per step and pair, the L1 mean's scale, one Adam step
number per step for every group, the Sec. 3.2 ranges of the response
parameters, the gains Gp and Gc held at their constants, and the next step
rendering with the updated responses."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2503_12174_gb300 import autograd, dpcs, fit  # noqa: E402


class FakeContext:
    """render_loss_backward records its key, scale and response parameters
    and writes a fixed gradient: +1 for every response parameter (so that
    Adam pushes each one down to its lower bound) and 0.5 for the maps;
    adam is Adam with bias correction, then the clamp."""

    def __init__(self):
        self.device = torch.device("cpu")
        self.renders, self.adams, self.tv = [], [], []

    def render_loss_backward(self, scene, albedo, rough, Ip, view, params, spp, bounces, seed, target, loss,
                             loss_kind=0, scale=1.0, Ic=None, Ec=None, dAlbedo=None, dRough=None, dParams=None):
        assert loss_kind == 1
        self.renders.append((seed, scale, autograd.params_vector(params)))
        loss.fill_(1.0)
        dAlbedo += 0.5
        dRough += 0.5
        if dParams is not None:
            dParams += 1.0

    def tv_loss(self, tex, grad, loss, weight):
        self.tv.append((tuple(tex.shape), weight))

    def adam(self, p, g, m, v, step, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8, lo=0.0, hi=1.0):
        self.adams.append((tuple(p.shape), step, lo, hi))
        m.mul_(beta1).add_((1 - beta1) * g)
        v.mul_(beta2).add_((1 - beta2) * g * g)
        p.sub_(lr * (m / (1 - beta1 ** step)) / ((v / (1 - beta2 ** step)).sqrt() + eps)).clamp_(lo, hi)


def _fit(ctx, fit_params=True):
    view = dpcs.DpcsView()
    view.Hc, view.Wc, view.Hp, view.Wp = 6, 5, 4, 4
    p0 = dpcs.DpcsParams()
    p0.gamma_p[:] = [2.2, 2.4, 2.0]
    p0.gain_p = 1.3
    p0.gamma_c[:] = [0.45, 0.5, 0.55]
    p0.gain_c = 4.0
    p0.wb[:] = [1.1, 1.0, 0.9]
    pairs = [(torch.zeros((4, 4, 3)), torch.zeros((6, 5, 3))) for _ in range(2)]
    return fit.SceneFit(ctx, 3, view, p0, torch.full((8, 8, 3), 0.5), torch.full((8, 8), 0.5), pairs, 4, 2,
                        lr_params=0.5, tv_weight=1e-5, seed=5, fit_params=fit_params)


def test_keys_scale_and_adam_steps():
    ctx = FakeContext()
    f = _fit(ctx)
    for _ in range(3):
        f.step()
    assert [r[0] for r in ctx.renders] == [5, 6, 7, 8, 9, 10]  # seed + (step - 1) K + pair
    assert all(r[1] == pytest.approx(1.0 / (2 * 6 * 5 * 3)) for r in ctx.renders)
    # per step: albedo, roughness, then gamma_p, gamma_c, w, each with that step's number
    steps = [a[1] for a in ctx.adams]
    assert steps == [1] * 5 + [2] * 5 + [3] * 5
    bounds = [(a[0], a[2], a[3]) for a in ctx.adams[:5]]
    assert bounds == [((8, 8, 3), 0.0, 1.0), ((8, 8), fit.ROUGH_MIN, 1.0), ((3,), 2.0, 3.0),
                      ((3,), pytest.approx(1.0 / 3.0), 1.0), ((3,), 0.2, 2.5)]
    assert ctx.tv == [((8, 8, 3), 1e-5), ((8, 8), 1e-5)] * 3


def test_response_ranges_gains_held_and_next_render_uses_the_update():
    ctx = FakeContext()
    f = _fit(ctx)
    for _ in range(12):
        f.step()
    first = ctx.renders[0][2]
    v = np.array(autograd.params_vector(f.params))
    # a positive gradient drives each fitted response to its lower bound
    np.testing.assert_allclose(v[0:3], 2.0, rtol=0, atol=1e-6)
    np.testing.assert_allclose(v[4:7], 1.0 / 3.0, rtol=0, atol=1e-6)
    np.testing.assert_allclose(v[8:11], 0.2, rtol=0, atol=1e-6)
    # Sec. 3.2 keeps the gains at their constants
    assert v[3] == pytest.approx(first[3]) and v[7] == pytest.approx(first[7])
    assert first[3] == pytest.approx(1.3) and first[7] == pytest.approx(4.0)
    # each step renders with the responses of the step before
    after_one = ctx.renders[2][2]
    assert after_one != first and after_one[3] == first[3]
    assert all(2.0 - 1e-6 <= x <= 2.2 for x in after_one[0:3])


def test_without_response_fitting_the_responses_stay():
    ctx = FakeContext()
    f = _fit(ctx, fit_params=False)
    for _ in range(3):
        f.step()
    assert all(r[2] == ctx.renders[0][2] for r in ctx.renders)
    assert len(ctx.adams) == 2 * 3  # albedo and roughness only
