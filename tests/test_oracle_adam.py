"""Pins of the oracle's Adam step (the optimiser of the Eq. 13 compensation and
the Eq. 9 fit, followed by the range clamp of Sec. 3.2) against two things
outside it: PyTorch's own Adam run on the CPU in float64, and the closed form
of Adam's first step, where the bias corrections make the update
-lr g / (|g| + eps) whatever beta1 and beta2 are."""
import numpy as np
import pytest

import oracle


def _torch_adam_trajectory(p0, grads, lr, b1, b2, eps, lo, hi):
    torch = pytest.importorskip("torch")
    p = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=lr, betas=(b1, b2), eps=eps)
    out = []
    for g in grads:
        opt.zero_grad()
        p.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        with torch.no_grad():
            p.clamp_(lo, hi)
        out.append(p.detach().numpy().copy())
    return out


@pytest.mark.parametrize("lr,b1,b2,eps", [(1e-2, 0.9, 0.999, 1e-8), (0.05, 0.8, 0.99, 1e-6), (0.3, 0.5, 0.9, 1e-3)])
def test_adam_equals_torch_adam_in_float64(lr, b1, b2, eps):
    """Ten steps with varying gradients: the oracle's parameters equal those
    of torch.optim.Adam (float64, CPU) clamped to [lo, hi] after each step,
    to float64 rounding.  The clamp is active: the start sits near both bounds
    and the steps are large enough to cross them."""
    rng = np.random.default_rng(7)
    n = 500
    lo, hi = 0.0, 1.0
    p0 = rng.choice([0.001, 0.5, 0.999], n) + rng.uniform(-1e-3, 1e-3, n)
    p0 = np.clip(p0, lo, hi)
    grads = [rng.normal(size=n) * rng.choice([1e-4, 1.0, 30.0], n) for _ in range(10)]
    ref = _torch_adam_trajectory(p0, grads, lr, b1, b2, eps, lo, hi)
    p, m, v = p0.copy(), np.zeros(n), np.zeros(n)
    clamped = 0
    for k, g in enumerate(grads, start=1):
        oracle.adam_step(p, g.copy(), m, v, k, lr=lr, b1=b1, b2=b2, eps=eps, lo=lo, hi=hi)
        np.testing.assert_allclose(p, ref[k - 1], rtol=1e-13, atol=1e-15)
        clamped += int(np.sum((p == lo) | (p == hi)))
    assert clamped > 0


def test_adam_first_step_closed_form():
    """After one step m/(1-b1) = g and v/(1-b2) = g^2, so the update is
    -lr g / (|g| + eps) before the clamp, for any beta1, beta2."""
    rng = np.random.default_rng(3)
    g = rng.normal(size=1000) * np.exp(rng.uniform(-12, 3, 1000))
    for b1, b2 in ((0.9, 0.999), (0.5, 0.5), (0.0, 0.0)):
        p = np.full(1000, 0.5)
        m, v = np.zeros(1000), np.zeros(1000)
        oracle.adam_step(p, g, m, v, 1, lr=0.01, b1=b1, b2=b2, eps=1e-8, lo=-np.inf, hi=np.inf)
        np.testing.assert_allclose(p, 0.5 - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-14, atol=1e-16)
        np.testing.assert_allclose(m, (1.0 - b1) * g, rtol=1e-15)
        np.testing.assert_allclose(v, (1.0 - b2) * g * g, rtol=1e-15)
    # with the clamp: a step that would leave [0, 1] stops at the bound
    p = np.array([0.004, 0.996, 0.5])
    m, v = np.zeros(3), np.zeros(3)
    oracle.adam_step(p, np.array([1.0, -1.0, 2.0]), m, v, 1, lr=0.01)
    np.testing.assert_allclose(p, [0.0, 1.0, 0.5 - 0.01 * 2.0 / (2.0 + 1e-8)], rtol=1e-15)


def test_adam_second_step_closed_form():
    """Two steps with gradients g1, g2 (no clamp): m2 = b1 (1-b1) g1 + (1-b1) g2,
    v2 = b2 (1-b2) g1^2 + (1-b2) g2^2, update lr (m2/(1-b1^2)) / (sqrt(v2/(1-b2^2)) + eps)."""
    b1, b2, lr, eps = 0.9, 0.999, 0.02, 1e-8
    g1, g2 = np.array([0.3, -2.0, 1e-3]), np.array([-0.1, -1.0, 5.0])
    p, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    oracle.adam_step(p, g1, m, v, 1, lr=lr, b1=b1, b2=b2, eps=eps, lo=-np.inf, hi=np.inf)
    p1 = -lr * g1 / (np.abs(g1) + eps)
    oracle.adam_step(p, g2, m, v, 2, lr=lr, b1=b1, b2=b2, eps=eps, lo=-np.inf, hi=np.inf)
    m2 = b1 * (1 - b1) * g1 + (1 - b1) * g2
    v2 = b2 * (1 - b2) * g1 ** 2 + (1 - b2) * g2 ** 2
    p2 = p1 - lr * (m2 / (1 - b1 ** 2)) / (np.sqrt(v2 / (1 - b2 ** 2)) + eps)
    np.testing.assert_allclose(p, p2, rtol=1e-13)
