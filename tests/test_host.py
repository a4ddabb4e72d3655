"""Host-side logic that needs no GPU: the response-parameter vector of the
autograd wrapper and the fit, the posed projector extrinsics written into a
dpcs_view, and the seeded principled maps."""
import numpy as np

from paper_2503_12174_gb300 import autograd, dpcs, pose, scenes


def test_params_vector_round_trip():
    p = dpcs.make_params(scenes.corner(res=8, spp=1).params)
    v = [2.1, 2.2, 2.3, 1.4, 0.5, 0.6, 0.7, 1.8, 0.9, 1.1, 1.2]
    q = autograd.with_vector(p, v)
    np.testing.assert_allclose(autograd.params_vector(q), v, rtol=1e-7)
    # the other fields are copied, and p itself is untouched
    assert q.k_proj == p.k_proj and q.ks == p.ks and q.rr_start == p.rr_start
    np.testing.assert_allclose(autograd.params_vector(p), autograd.params_vector(
        dpcs.make_params(scenes.corner(res=8, spp=1).params)))


def test_posed_view_writes_the_posed_extrinsics():
    sc = scenes.corner(res=16, spp=1)
    v = dpcs.view_of(sc)
    R, t = pose.rotation([0.02, -0.05, 0.1]), np.array([0.01, 0.03, -0.02])
    pv = pose.posed_view(v, R, t)
    Rp2, tp2 = pose.posed_extrinsics(sc.Rp, sc.tp, R, t)
    np.testing.assert_allclose(np.array(pv.Rp[:]).reshape(3, 3), Rp2, atol=1e-7)
    np.testing.assert_allclose(np.array(pv.tp[:]), tp2, atol=1e-7)
    assert list(pv.Kc[:]) == list(v.Kc[:]) and list(pv.Kp[:]) == list(v.Kp[:])
    assert (pv.Hc, pv.Wc, pv.Hp, pv.Wp) == (v.Hc, v.Wc, v.Hp, v.Wp)
    # the projector centre -Rp'^T tp' is the moved centre R cp + t
    cp = -np.asarray(sc.Rp, np.float64).T @ np.asarray(sc.tp, np.float64)
    np.testing.assert_allclose(-Rp2.T @ tp2, R @ cp + t, atol=1e-12)
    # the identity pose changes nothing
    pv0 = pose.posed_view(v, np.eye(3), np.zeros(3))
    np.testing.assert_array_equal(np.array(pv0.Rp[:]), np.array(v.Rp[:]))
    np.testing.assert_array_equal(np.array(pv0.tp[:]), np.array(v.tp[:]))


def test_principled_maps_are_seeded_and_in_range():
    a = scenes.principled_maps(np.random.default_rng(3), 24, 20)
    b = scenes.principled_maps(np.random.default_rng(3), 24, 20)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    metallic, normal = a
    assert metallic.shape == (24, 20) and normal.shape == (24, 20, 3)
    assert metallic.min() >= 0.0 and metallic.max() <= 0.8 + 1e-6
    n = 2.0 * normal.astype(np.float64) - 1.0
    np.testing.assert_allclose(np.linalg.norm(n, axis=-1), 1.0, atol=1e-6)  # unit tangent-space normals
    assert n[..., 2].min() > 0.5  # tilted, but facing out of the surface


class _FakeSceneLib:
    """Stands in for libdpcs's context and scene entry points on the CPU."""

    def __init__(self):
        self.exports = 0

    def dpcs_create(self, device, budget, out):
        out._obj.value = 1
        return 0

    def dpcs_destroy(self, h):
        return 0

    def dpcs_last_error(self, h):
        return b""

    def dpcs_scene_upload(self, h, verts, V, tris, T, uv, stream, out):
        out._obj.value = 7
        return 0

    def dpcs_scene_free(self, h, scene):
        return 0

    def dpcs_scene_export(self, h, scene, codes, order, child, box):
        self.exports += 1
        return 0


def test_host_arrays_the_library_reads_or_fills_are_checked(monkeypatch):
    """The library fills export()'s host arrays for the scene's own triangle
    count, and reads V x 3 positions, T x 3 indices and V x 2 UVs at upload:
    the binding refuses other sizes before calling it."""
    import pytest

    from paper_2503_12174_gb300 import dpcs, scenes

    monkeypatch.setattr(dpcs, "_stream", lambda stream: None)  # no CUDA stream on the CPU
    lib = _FakeSceneLib()
    ctx = dpcs.Context(0, lib=lib)
    verts, tris, uv = scenes.corner_mesh()
    h = ctx.upload(verts, tris, uv)
    codes, order, child, box = ctx.export(h, len(tris))
    assert codes.shape == (len(tris),) and child.shape == (len(tris) - 1, 2) and lib.exports == 1
    for T in (len(tris) - 1, len(tris) + 1):
        with pytest.raises(ValueError):
            ctx.export(h, T)
    assert lib.exports == 1
    # the library reads V x 3, T x 3 and V x 2 values: other shapes never reach it
    for bad in ((verts.ravel(), tris, uv), (verts, tris[:, :2], uv), (verts, tris, uv[:-1]), (verts[:, :2], tris, uv)):
        with pytest.raises(ValueError):
            ctx.upload(*bad)
    with pytest.raises(ValueError):
        ctx.update(h, verts.ravel())
    ctx.free(h)
    ctx.close()
