"""GPU LBVH build vs the oracle's reference: Morton codes, sort order, radix
tree topology and child boxes must agree bit for bit (radix-tree builder);
closest hits through the BVH must match brute-force FP64 tests (both
builders)."""
import numpy as np
import pytest

from paper_2503_12174_gb300 import dpcs, scenes
from gpu_util import ctx, need_cuda

pytestmark = pytest.mark.gpu


def _meshes():
    rng = np.random.default_rng(3)
    sc = scenes.plane()
    yield "plane", sc.verts, sc.tris, sc.uv
    v, t, u = scenes.corner_mesh()
    yield "corner", v, t, u
    verts = rng.random((300, 3)).astype(np.float32)
    yield "random", verts, rng.integers(0, 300, (257, 3)).astype(np.int32), rng.random((300, 2)).astype(np.float32)
    base = rng.random((40, 3)).astype(np.float32)
    verts = np.concatenate([base, base, base]).astype(np.float32)
    tris = np.asarray([[i % 40, (i % 40) + 40, (i % 40) + 80] for i in range(200)], np.int32)
    yield "duplicates", verts, tris, np.zeros((120, 2), np.float32)
    v, t, u = scenes.heightfield_mesh(np.random.default_rng(4))
    yield "heightfield", v, t, u
    v, t, u = scenes.icosphere(4)
    yield "sphere", v, t, u


@pytest.mark.parametrize("case", list(range(6)))
def test_lbvh_bit_exact(orc, case):
    name, verts, tris, uv = list(_meshes())[case]
    c = ctx()
    c.set_bvh_builder(dpcs.DPCS_BVH_LBVH)
    try:
        h = c.upload(verts, tris, uv)
    finally:
        c.set_bvh_builder(dpcs.DPCS_BVH_PLOC)
    try:
        codes, order, child, box = c.export(h, len(tris))
        rc, ro, rch, rb = orc.lbvh(verts, tris)
        np.testing.assert_array_equal(codes, rc, err_msg=name)
        np.testing.assert_array_equal(order, ro, err_msg=name)
        np.testing.assert_array_equal(child, rch, err_msg=name)
        np.testing.assert_array_equal(box.view(np.uint32), rb.view(np.uint32), err_msg=name)
    finally:
        c.free(h)


@pytest.mark.parametrize("builder", [dpcs.DPCS_BVH_LBVH, dpcs.DPCS_BVH_PLOC])
@pytest.mark.parametrize("which", ["corner", "heightfield_small", "sphere"])
def test_closest_hit_vs_brute_force(orc, which, builder):
    torch = need_cuda()
    rng = np.random.default_rng(11)
    if which == "corner":
        verts, tris, uv = scenes.corner_mesh()
        o = np.zeros((20000, 3))
        d = rng.normal(size=(20000, 3)); d[:, 2] = np.abs(d[:, 2]) + 0.5
    elif which == "heightfield_small":
        verts, tris, uv = scenes.heightfield_mesh(np.random.default_rng(4), n_vert=81)
        o = rng.uniform(-0.5, 0.5, (20000, 3)); o[:, 2] = 0.0
        d = rng.normal(size=(20000, 3)); d[:, 2] = np.abs(d[:, 2]) + 0.3
    else:
        verts, tris, uv = scenes.icosphere(3)
        o = rng.uniform(-0.5, 0.5, (20000, 3))
        d = rng.normal(size=(20000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = o.astype(np.float32).astype(np.float64)
    d = d.astype(np.float32).astype(np.float64)
    c = ctx()
    c.set_bvh_builder(builder)
    try:
        h = c.upload(verts, tris, uv)
    finally:
        c.set_bvh_builder(dpcs.DPCS_BVH_PLOC)
    try:
        t, tri = c.trace(h, torch.from_numpy(o.astype(np.float32)).cuda(), torch.from_numpy(d.astype(np.float32)).cuda())
        c.sync()
        t, tri = t.cpu().numpy().astype(np.float64), tri.cpu().numpy()
    finally:
        c.free(h)
    rt, rtri = orc.closest(verts, tris, o, d)
    same = tri == rtri
    assert same.mean() >= 0.999, same.mean()
    hit = same & (rtri >= 0)
    assert hit.sum() > 1000
    np.testing.assert_allclose(t[hit], rt[hit], rtol=1e-5, atol=1e-6)
    # disagreements must be ties or near-ties in distance (edges between triangles)
    diff = ~same & (rtri >= 0) & (tri >= 0)
    if diff.any():
        np.testing.assert_allclose(t[diff], rt[diff], rtol=1e-4, atol=1e-5)
