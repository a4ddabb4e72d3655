"""Pins of the oracle's Eq. 11 denoiser and its guide features, against
closed forms and textbook filters rather than against itself."""
import numpy as np
import pytest

from paper_2503_12174_gb300 import scenes

ndimage = pytest.importorskip("scipy.ndimage")


def _prm(radius=3, sigma_s=1.5, sigma_albedo=0.0, sigma_normal=0.0, sigma_depth=0.0):
    return {"radius": radius, "sigma_s": sigma_s, "sigma_albedo": sigma_albedo, "sigma_normal": sigma_normal,
            "sigma_depth": sigma_depth}


def _random_guide(rng, H, W):
    g = np.zeros((H, W, 8))
    g[..., 0:3] = rng.uniform(0.2, 0.9, (H, W, 3))
    n = rng.normal(size=(H, W, 3))
    g[..., 3:6] = n / np.linalg.norm(n, axis=-1, keepdims=True)
    g[..., 6] = rng.uniform(1.0, 3.0, (H, W))
    g[..., 7] = 1.0
    return g


def test_gbuffer_plane_closed_form(orc):
    """A quad at z = 1 facing the camera: the ray through pixel centre (x, y)
    hits at Kc^-1 (x + 1/2, y + 1/2, 1), so the hit distance is that vector's
    length; the normal is -z and the albedo the texture's constant 0.5."""
    sc = scenes.plane(res=24)
    g = orc.gbuffer(sc)
    ys, xs = np.mgrid[0:sc.Hc, 0:sc.Wc]
    pix = np.stack([xs + 0.5, ys + 0.5, np.ones_like(xs, dtype=float)], axis=-1)
    v = pix @ np.linalg.inv(np.asarray(sc.Kc, np.float64)).T
    assert np.allclose(v[..., 2], 1.0)
    hit = g[..., 7] == 1.0
    assert hit.all()
    np.testing.assert_allclose(g[..., 6], np.linalg.norm(v, axis=-1), rtol=1e-12)
    np.testing.assert_allclose(g[..., 3:6], np.broadcast_to([0.0, 0.0, -1.0], g[..., 3:6].shape), atol=1e-12)
    np.testing.assert_allclose(g[..., 0:3], 0.5, rtol=1e-12)


def test_gbuffer_misses_are_zero_and_normals_face_the_camera(orc):
    sc = scenes.corner(res=32, tex=16, spp=1)
    g = orc.gbuffer(sc)
    hit = g[..., 7] == 1.0
    assert 0 < hit.sum() < hit.size  # the corner does not fill the view
    assert np.all(g[~hit] == 0.0)
    n = g[hit][:, 3:6]
    np.testing.assert_allclose(np.linalg.norm(n, axis=-1), 1.0, rtol=1e-12)
    ys, xs = np.nonzero(hit)
    pix = np.stack([xs + 0.5, ys + 0.5, np.ones(len(xs))], axis=-1)
    d = pix @ np.linalg.inv(np.asarray(sc.Kc, np.float64)).T
    assert np.all(np.sum(n * d, axis=-1) < 0.0)
    assert np.all(g[hit][:, 6] > 0.0)


def test_denoise_radius_zero_is_identity(orc):
    rng = np.random.default_rng(0)
    I = rng.uniform(size=(9, 11, 3))
    out, W = orc.denoise(I, _random_guide(rng, 9, 11), _prm(radius=0, sigma_albedo=0.1))
    np.testing.assert_array_equal(out, I)
    np.testing.assert_array_equal(W, 1.0)


def test_denoise_keeps_a_constant_image(orc):
    rng = np.random.default_rng(1)
    I = np.broadcast_to([0.3, 0.7, 1.9], (13, 10, 3))
    out, _ = orc.denoise(I, _random_guide(rng, 13, 10), _prm(radius=4, sigma_albedo=0.2, sigma_normal=0.5,
                                                             sigma_depth=0.3))
    np.testing.assert_allclose(out, I, rtol=1e-14)


@pytest.mark.parametrize("H,W,r,s", [(17, 23, 4, 1.7), (3, 5, 6, 2.5)])
def test_denoise_without_guide_terms_is_a_normalised_gaussian(orc, H, W, r, s):
    """All feature widths off: the filter is a Gaussian blur renormalised by
    the part of the window inside the image -- scipy's correlate of the image
    and of ones with zero padding, divided.  The second case has a window
    wider than the image."""
    rng = np.random.default_rng(2)
    I = rng.uniform(size=(H, W, 3))
    out, den = orc.denoise(I, _random_guide(rng, H, W), _prm(radius=r, sigma_s=s))
    yy, xx = np.mgrid[-r:r + 1, -r:r + 1]
    K = np.exp(-(xx * xx + yy * yy) / (2 * s * s))
    ones = ndimage.correlate(np.ones((H, W)), K, mode="constant", cval=0.0)
    np.testing.assert_allclose(den, ones, rtol=1e-12)
    for j in range(3):
        ref = ndimage.correlate(I[..., j], K, mode="constant", cval=0.0) / ones
        np.testing.assert_allclose(out[..., j], ref, rtol=1e-12)


@pytest.mark.parametrize("feature", ["albedo", "normal", "depth"])
def test_denoise_does_not_blur_across_a_guide_edge(orc, feature):
    """A guide edge in one feature only (albedo 0 | 1, normal -z | +x, depth
    1 | 3), with a narrow width for that feature and the other two off: each
    side is blurred with its own pixels only (the cross-bilateral property),
    i.e. a Gaussian blur of the masked image over the masked ones."""
    rng = np.random.default_rng(3)
    H, W, r, s = 12, 20, 3, 2.0
    I = rng.uniform(size=(H, W, 3))
    left = np.zeros((H, W), bool)
    left[:, :W // 2] = True
    g = np.zeros((H, W, 8))
    g[..., 3:6] = [0.0, 0.0, -1.0]
    g[..., 6] = 1.0
    g[..., 7] = 1.0
    if feature == "albedo":
        g[~left, 0:3] = 1.0
    elif feature == "normal":
        g[~left, 3:6] = [1.0, 0.0, 0.0]
    else:
        g[~left, 6] = 3.0
    out, _ = orc.denoise(I, g, _prm(radius=r, sigma_s=s, **{"sigma_" + feature: 0.01}))
    yy, xx = np.mgrid[-r:r + 1, -r:r + 1]
    K = np.exp(-(xx * xx + yy * yy) / (2 * s * s))
    for m in (left, ~left):
        den = ndimage.correlate(m.astype(float), K, mode="constant", cval=0.0)
        for j in range(3):
            num = ndimage.correlate(I[..., j] * m, K, mode="constant", cval=0.0)
            np.testing.assert_allclose(out[..., j][m], num[m] / den[m], rtol=1e-10)


def test_denoise_backward_is_the_adjoint(orc):
    """<D x, y> = <x, D^T y>: the scattered adjoint against the gathered
    forward, all feature terms on, a window clipped at every border."""
    rng = np.random.default_rng(4)
    H, W = 14, 9
    g = _random_guide(rng, H, W)
    prm = _prm(radius=5, sigma_s=2.5, sigma_albedo=0.3, sigma_normal=0.7, sigma_depth=0.5)
    x = rng.normal(size=(H, W, 3))
    y = rng.normal(size=(H, W, 3))
    Dx, _ = orc.denoise(x, g, prm)
    DTy = orc.denoise_backward(y, g, prm)
    assert abs(np.sum(Dx * y) - np.sum(x * DTy)) <= 1e-12 * np.sum(np.abs(Dx * y))


def test_denoise_backward_matches_finite_differences(orc):
    """D is linear in I, so one central difference per probed input is exact
    up to rounding; it checks single entries of D^T."""
    rng = np.random.default_rng(5)
    H, W = 8, 7
    g = _random_guide(rng, H, W)
    prm = _prm(radius=2, sigma_s=1.2, sigma_albedo=0.4, sigma_normal=0.0, sigma_depth=0.6)
    I = rng.uniform(size=(H, W, 3))
    y = rng.normal(size=(H, W, 3))
    dI = orc.denoise_backward(y, g, prm)
    h = 1e-3
    for (a, b, j) in ((0, 0, 0), (3, 4, 1), (7, 6, 2), (5, 1, 0)):
        Ip, Im = I.copy(), I.copy()
        Ip[a, b, j] += h
        Im[a, b, j] -= h
        fd = (np.sum(orc.denoise(Ip, g, prm)[0] * y) - np.sum(orc.denoise(Im, g, prm)[0] * y)) / (2 * h)
        assert abs(fd - dI[a, b, j]) <= 1e-9 * max(1.0, abs(fd))
