"""The oracle's timing mode (a median-split FP64 BVH, used for the CPU
baseline) against its parity mode (brute force over every triangle): the
same closest hits bit for bit, including exact ties in t along shared
edges, and therefore the same images and gradients bit for bit."""
import numpy as np
import pytest

from paper_2503_12174_gb300 import scenes


def _rays(rng, n, origin_box, target_box):
    o = rng.uniform(*origin_box, size=(n, 3))
    tgt = rng.uniform(*target_box, size=(n, 3))
    d = tgt - o
    return o, d / np.linalg.norm(d, axis=1, keepdims=True)


@pytest.mark.parametrize("mesh", ["corner", "heightfield", "sphere"])
def test_bvh_closest_hits_equal_brute_force(orc, mesh):
    rng = np.random.default_rng(12)
    if mesh == "corner":
        v, t, _ = scenes.corner_mesh()
        o, d = _rays(rng, 20000, (-0.6, 0.7), (-0.6, 1.7))
        # rays through the camera's pixel centres: the seams of the corner
        # project onto image diagonals, where rays run along shared edges
        sc = scenes.corner(res=48)
        ys, xs = np.mgrid[0:48, 0:48]
        pc = np.stack([xs.ravel() + 0.5, ys.ravel() + 0.5, np.ones(48 * 48)], 1) @ np.linalg.inv(sc.Kc).T
        o = np.concatenate([o, np.zeros_like(pc)])
        d = np.concatenate([d, pc / np.linalg.norm(pc, axis=1, keepdims=True)])
    elif mesh == "heightfield":
        v, t, _ = scenes.heightfield_mesh(np.random.default_rng(4), n_vert=81)
        o, d = _rays(rng, 20000, (-1.2, 1.2), (-1.2, 1.2))
        o[:, 2] = rng.uniform(0.0, 1.0, len(o))
        tgt = np.stack([rng.uniform(-1, 1, len(o)), rng.uniform(-1, 1, len(o)), np.full(len(o), 1.5)], 1)
        d = tgt - o
        d /= np.linalg.norm(d, axis=1, keepdims=True)
    else:
        v, t = scenes.icosphere(3)[:2]
        o, d = _rays(rng, 20000, (-0.5, 0.5), (-2.0, 2.0))
    tb, ib = orc.closest(v, t, o, d)
    ta, ia = orc.closest(v, t, o, d, accel=True)
    assert (ib >= 0).mean() > 0.15
    np.testing.assert_array_equal(ia, ib)
    np.testing.assert_array_equal(ta, tb)


def test_bvh_breaks_exact_ties_like_brute_force(orc):
    """Two coincident copies of a quad: every hit is an exact tie in t, and
    both modes must return the lower triangle index."""
    v, t, _ = scenes.corner_mesh()
    t2 = np.concatenate([t, t])  # triangle i and i + T are the same triangle
    rng = np.random.default_rng(1)
    o, d = _rays(rng, 5000, (-0.4, 0.4), (-0.5, 1.6))
    tb, ib = orc.closest(v, t2, o, d)
    ta, ia = orc.closest(v, t2, o, d, accel=True)
    np.testing.assert_array_equal(ia, ib)
    np.testing.assert_array_equal(ta, tb)
    assert np.all(ib[ib >= 0] < len(t))


@pytest.mark.parametrize("case", ["corner", "heightfield_rr"])
def test_timing_mode_renders_the_same_image_and_gradient(orc, case):
    if case == "corner":
        sc = scenes.corner(res=24, tex=32, spp=4, bounces=3, seed=2)
    else:
        sc = scenes.heightfield(spp=2, cam=20, proj=(24, 32), tex=32, n_vert=41)
    Eb, Ib = orc.render(sc)
    Ea, Ia = orc.render(sc, accel=True)
    assert np.abs(Eb).max() > 0
    np.testing.assert_array_equal(Ea, Eb)
    np.testing.assert_array_equal(Ia, Ib)
    W = np.random.default_rng(3).normal(size=(sc.Hc, sc.Wc, 3))
    gb = orc.render_backward(sc, W)
    ga = orc.render_backward(sc, W, accel=True)
    # the same paths; the adjoint's sums over threads are taken in OpenMP's
    # schedule order, which changes the last bits between any two runs
    for k in gb:
        np.testing.assert_allclose(ga[k], gb[k], rtol=1e-12, atol=1e-14 * np.abs(gb[k]).max())
