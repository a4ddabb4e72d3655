"""Pins for the oracle's Lambert + GGX BRDF, its sampling routine and pdf.

Checked against mathematics only: Helmholtz reciprocity, the normalisation
of the GGX distribution and of the sampling pdf (quadrature over the sphere),
the Monte Carlo identity E[g/pdf] = integral of g for directions produced by
the sampler, the exact Lambert sampling weight, and the roughness derivative
against central finite differences.
"""
import numpy as np
import pytest


def _rand_dir(rng, n, hemi=None):
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    if hemi is not None:
        v[v @ hemi < 0] *= -1
    return v


def _sphere_quad(nt=400, npph=800):
    """midpoint quadrature on the unit sphere: directions and solid-angle weights"""
    th = (np.arange(nt) + 0.5) * np.pi / nt
    ph = (np.arange(npph) + 0.5) * 2 * np.pi / npph
    T, P = np.meshgrid(th, ph, indexing="ij")
    d = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)
    w = (np.sin(T) * (np.pi / nt) * (2 * np.pi / npph)).ravel()
    return d, w


def test_reciprocity(orc):
    rng = np.random.default_rng(0)
    for _ in range(300):
        n = _rand_dir(rng, 1)[0]
        wo, wi = _rand_dir(rng, 2, hemi=n)
        rho = rng.random(3) * 0.9
        r = rng.uniform(0.05, 1.0)
        f1, _ = orc.bsdf_eval(n, wo, wi, rho, r, 1.0, 0.04)
        f2, _ = orc.bsdf_eval(n, wi, wo, rho, r, 1.0, 0.04)
        np.testing.assert_allclose(f1, f2, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("alpha", [0.01, 0.1, 0.36, 0.64, 1.0])
def test_ggx_D_normalised(orc, alpha):
    # integral of D(h) cos(theta_h) d omega = 1; with x = cos^2 it is pi * int_0^1 D(sqrt x) dx
    integrate = pytest.importorskip("scipy.integrate")
    a2 = alpha * alpha
    pts = sorted({max(0.0, 1 - k * a2) for k in (100.0, 10.0, 1.0, 0.1, 0.01)} - {0.0})
    val, err = integrate.quad(lambda x: np.pi * orc.ggx_D(np.sqrt(x), alpha), 0.0, 1.0, points=pts, limit=500,
                              epsabs=1e-12, epsrel=1e-10)
    assert abs(val - 1.0) < 1e-6


@pytest.mark.parametrize("ks,r", [(0.0, 0.5), (1.0, 0.3), (1.0, 0.6), (1.0, 0.9)])
def test_pdf_integrates_to_one(orc, ks, r):
    """The sampling density integrates to one minus the probability that the
    visible-normal sample reflects below the horizon (such samples end the
    path); for the cosine lobe alone it integrates to exactly one."""
    rng = np.random.default_rng(1)
    n = np.array([0.0, 0.0, 1.0])
    d, w = _sphere_quad(300, 600)
    for _ in range(3):
        wo = _rand_dir(rng, 1, hemi=n)[0]
        wo[2] = max(wo[2], 0.2)
        wo /= np.linalg.norm(wo)
        p = np.array([orc.bsdf_pdf(n, wo, di, r, ks) for di in d])
        ps = 0.5 if ks > 0 else 0.0
        N = 20000
        u = rng.random((N, 2))
        fail = np.mean([not orc.bsdf_sample(n, wo, r, ks, 0.0, a, b)[0] for a, b in u]) if ps else 0.0
        se = np.sqrt(max(fail * (1 - fail), 1e-12) / N)
        assert abs((p * w).sum() - (1.0 - ps * fail)) < 4 * ps * se + 2e-3


@pytest.mark.parametrize("r", [0.35, 0.6, 0.9])
def test_sampler_matches_pdf(orc, r):
    """E[g(wi) / pdf(wi)] over sampled wi equals the quadrature integral of g."""
    rng = np.random.default_rng(2)
    n = np.array([0.0, 0.0, 1.0])
    wo = np.array([0.3, -0.2, 0.9])
    wo /= np.linalg.norm(wo)
    d, w = _sphere_quad(200, 400)

    def g(v):
        return np.maximum(v[..., 2], 0) * (1.0 + 0.5 * v[..., 0]) ** 2

    exact = (g(d) * w).sum()
    N = 40000
    u = rng.random((N, 3))
    vals = np.zeros(N)
    for i in range(N):
        ok, wi = orc.bsdf_sample(n, wo, r, 1.0, *u[i])
        if ok:
            vals[i] = g(wi) / orc.bsdf_pdf(n, wo, wi, r, 1.0)
    est, se = vals.mean(), vals.std() / np.sqrt(N)
    assert abs(est - exact) < 4 * se + 1e-3 * exact


def test_lambert_weight_is_albedo(orc):
    rng = np.random.default_rng(3)
    for _ in range(200):
        n = _rand_dir(rng, 1)[0]
        wo = _rand_dir(rng, 1, hemi=n)[0]
        rho = rng.random(3)
        ok, wi = orc.bsdf_sample(n, wo, 0.5, 0.0, *rng.random(3))
        assert ok
        f, _ = orc.bsdf_eval(n, wo, wi, rho, 0.5, 0.0, 0.04)
        pdf = orc.bsdf_pdf(n, wo, wi, 0.5, 0.0)
        np.testing.assert_allclose(f * np.dot(n, wi) / pdf, rho, rtol=1e-12)


def test_mean_weight_is_directional_albedo(orc):
    rng = np.random.default_rng(4)
    n = np.array([0.0, 0.0, 1.0])
    wo = np.array([0.5, 0.1, 0.8])
    wo /= np.linalg.norm(wo)
    rho, r = np.array([0.3, 0.5, 0.7]), 0.5
    d, w = _sphere_quad(300, 600)
    fq = np.array([orc.bsdf_eval(n, wo, di, rho, r, 1.0, 0.04)[0] for di in d])
    albedo = (fq * np.maximum(d[:, 2], 0)[:, None] * w[:, None]).sum(0)
    N = 30000
    u = rng.random((N, 3))
    acc = np.zeros((N, 3))
    for i in range(N):
        ok, wi = orc.bsdf_sample(n, wo, r, 1.0, *u[i])
        if ok:
            f, _ = orc.bsdf_eval(n, wo, wi, rho, r, 1.0, 0.04)
            acc[i] = f * wi[2] / orc.bsdf_pdf(n, wo, wi, r, 1.0)
    se = acc.std(0) / np.sqrt(N)
    assert np.all(np.abs(acc.mean(0) - albedo) < 4 * se + 1e-3)
    assert np.all(albedo <= 1.0)  # energy: directional albedo <= 1 for rho <= 0.9


def test_roughness_derivative_fd(orc):
    rng = np.random.default_rng(5)
    for _ in range(100):
        n = _rand_dir(rng, 1)[0]
        wo, wi = _rand_dir(rng, 2, hemi=n)
        r = rng.uniform(0.1, 0.9)
        rho = rng.random(3)
        _, d = orc.bsdf_eval(n, wo, wi, rho, r, 1.0, 0.04)
        h = 1e-6
        fp, _ = orc.bsdf_eval(n, wo, wi, rho, r + h, 1.0, 0.04)
        fm, _ = orc.bsdf_eval(n, wo, wi, rho, r - h, 1.0, 0.04)
        fd = (fp[0] - fm[0]) / (2 * h)
        assert abs(fd - d) <= 1e-6 * max(1.0, abs(d))
