"""Host logic of projector compensation (Eq. 13), on the CPU against a
stand-in for the library context: every step renders under Philox key
seed + k and takes Adam step k + 1, and a checkpoint written after some steps
and resumed by a fresh object continues that numbering, so the result equals
an uninterrupted run bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2503_12174_gb300 import compensate, dpcs  # noqa: E402


class FakeContext:
    """render_loss_backward: Ic = 0.5 Ip + 1e-3 key (a key-dependent stand-in
    for the Monte Carlo noise), L = 1/2 |Ic - target|^2, dIp += 0.5 (Ic - target);
    adam: the update of Adam with bias correction, then the clamp."""

    def __init__(self):
        self.device = torch.device("cpu")
        self.keys, self.adam_steps = [], []

    def render_loss_backward(self, scene, albedo, rough, P, view, params, spp, bounces, seed, target, loss,
                             loss_kind=0, Ic=None, Ec=None, dIp=None):
        assert loss_kind == 0
        self.keys.append(seed)
        Ic.copy_(0.5 * P + 1e-3 * seed)
        Ec.copy_(Ic)
        r = Ic - target
        loss.fill_(float(0.5 * (r.double() ** 2).sum()))
        dIp += 0.5 * r

    def adam(self, p, g, m, v, step, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8, lo=0.0, hi=1.0):
        self.adam_steps.append(step)
        m.mul_(beta1).add_((1 - beta1) * g)
        v.mul_(beta2).add_((1 - beta2) * g * g)
        mh = m / (1 - beta1 ** step)
        vh = v / (1 - beta2 ** step)
        p.sub_(lr * mh / (vh.sqrt() + eps)).clamp_(lo, hi)


def _make(ctx, seed=40, lr=0.05, steps=6):
    view = dpcs.DpcsView()
    view.Hc = view.Wc = view.Hp = view.Wp = 5
    return compensate.Compensation(ctx, 1, None, None, view, dpcs.DpcsParams(), 4, 2, steps, lr=lr, seed=seed,
                                   graph=False)


def _data():
    rng = np.random.default_rng(4)
    Ip0 = torch.from_numpy(rng.uniform(0.2, 0.8, (5, 5, 3)).astype(np.float32))
    target = torch.from_numpy(rng.uniform(0.1, 0.5, (5, 5, 3)).astype(np.float32))
    return Ip0, target


def test_steps_use_their_own_key_and_adam_step():
    ctx = FakeContext()
    comp = _make(ctx)
    Ip0, target = _data()
    P, hist = comp.run(Ip0, target)
    assert ctx.keys == [40 + k for k in range(6)]
    assert ctx.adam_steps == [1, 2, 3, 4, 5, 6]
    assert float(hist[-1]) < float(hist[0])
    assert float(P.min()) >= 0.0 and float(P.max()) <= 1.0


def test_checkpoint_resume_equals_an_uninterrupted_run(tmp_path):
    Ip0, target = _data()
    ref_ctx = FakeContext()
    ref = _make(ref_ctx)
    ref.start(Ip0, target)
    P_ref, hist_ref = ref.advance(6)

    ctx = FakeContext()
    a = _make(ctx)
    a.start(Ip0, target)
    a.advance(3)
    path = str(tmp_path / "comp.npz")
    a.save(path)
    b = _make(ctx)
    b.resume(path)
    P, hist = b.advance(3)
    assert ctx.keys == ref_ctx.keys and ctx.adam_steps == ref_ctx.adam_steps
    np.testing.assert_array_equal(P.numpy(), P_ref.numpy())
    np.testing.assert_array_equal(hist.numpy(), hist_ref.numpy())
    with pytest.raises(ValueError):
        b.advance(1)  # all six steps are done


@pytest.mark.parametrize("kw", [{"seed": 41}, {"lr": 0.04}])
def test_resume_refuses_another_seed_or_learning_rate(tmp_path, kw):
    Ip0, target = _data()
    a = _make(FakeContext())
    a.start(Ip0, target)
    a.advance(2)
    path = str(tmp_path / "comp.npz")
    a.save(path)
    with pytest.raises(ValueError, match="seed or learning rate"):
        _make(FakeContext(), **kw).resume(path)
