"""Pins of the oracle's Eq. 9 terms (L1 data term, total variation of the
BRDF maps) against closed forms and finite differences."""
import numpy as np
import pytest


def test_tv_of_a_ramp_is_its_closed_form(orc):
    """m(x, y, c) = a_c x + b_c y on an H x W grid: every right difference is
    a_c and every down difference b_c, so TV = sum_c |a_c| H (W-1) + |b_c| (H-1) W.
    Inside the grid each texel's four sign terms cancel."""
    H, W = 7, 11
    a, b = np.array([0.3, -0.2, 0.05]), np.array([-0.1, 0.4, 0.0])
    y, x = np.mgrid[0:H, 0:W]
    m = a * x[..., None] + b * y[..., None]
    loss, g = orc.tv_loss(m, weight=0.5)
    assert loss == pytest.approx(0.5 * np.sum(np.abs(a) * H * (W - 1) + np.abs(b) * (H - 1) * W), rel=1e-12)
    np.testing.assert_array_equal(g[1:-1, 1:-1], 0.0)
    # left column: only the right difference (m increases with x for a > 0) pulls it
    np.testing.assert_allclose(g[1:-1, 0, 0], -0.5 * np.sign(a[0]))
    np.testing.assert_allclose(g[0, 1:-1, 1], -0.5 * np.sign(b[1]))  # top row, channel 1: only the down difference
    # channel 2 has b = 0: no down term, so its top row only sees the x
    # differences, which cancel except at the two ends
    np.testing.assert_array_equal(g[0, 1:-1, 2], 0.0)
    assert g[0, 0, 2] == -0.5 and g[0, -1, 2] == 0.5


@pytest.mark.parametrize("shape", [(6, 9), (5, 4, 3)])
def test_tv_gradient_is_the_finite_difference(orc, shape):
    """Away from ties the TV is linear in each texel, so a central difference
    with a step below the smallest gap is exact."""
    rng = np.random.default_rng(1)
    m = rng.uniform(size=shape)
    _, g = orc.tv_loss(m, weight=0.7)
    gaps = np.concatenate([np.abs(np.diff(m, axis=0)).ravel(), np.abs(np.diff(m, axis=1)).ravel()])
    h = 0.25 * gaps.min()
    for idx in [tuple(rng.integers(0, s) for s in shape) for _ in range(12)]:
        mp, mm = m.copy(), m.copy()
        mp[idx] += h
        mm[idx] -= h
        fd = (orc.tv_loss(mp, weight=0.7)[0] - orc.tv_loss(mm, weight=0.7)[0]) / (2 * h)
        assert fd == pytest.approx(g[idx], abs=1e-9)


def test_l1_loss_value_and_gradient(orc):
    rng = np.random.default_rng(2)
    I = rng.uniform(size=(4, 5, 3))
    T = I + rng.choice([-0.2, 0.3], size=I.shape)
    T[0, 0, 0] = I[0, 0, 0]  # a tie: sign(0) = 0
    loss, g = orc.l1_loss(I, T, scale=0.25)
    assert loss == pytest.approx(0.25 * np.sum(np.abs(I - T)), rel=1e-12)
    assert g[0, 0, 0] == 0.0
    h = 1e-3
    for idx in [(1, 2, 0), (3, 4, 2)]:
        Ip, Im = I.copy(), I.copy()
        Ip[idx] += h
        Im[idx] -= h
        fd = (orc.l1_loss(Ip, T, 0.25)[0] - orc.l1_loss(Im, T, 0.25)[0]) / (2 * h)
        assert fd == pytest.approx(g[idx], abs=1e-9)
