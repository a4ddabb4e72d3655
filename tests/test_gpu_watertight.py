"""Watertight ray-triangle intersection on the GPU (Woop, Benthin, Wald 2013):
rays aimed exactly at the shared edges and vertices of a connected mesh, in
FP32, must hit it.  A Moller-Trumbore test in FP32 misses some of them (a ray
through a shared edge can fall outside both triangles by rounding), which lets
light leak through closed surfaces."""
import numpy as np
import pytest

from paper_2503_12174_gb300 import scenes
from gpu_util import ctx, need_cuda

pytestmark = pytest.mark.gpu


def _interior_targets(verts, tris):
    """Edges shared by two triangles (matched by the FP32 positions of their
    ends, so the seams between the corner's separately built walls count)
    and vertices all of whose edges are shared: points on the mesh that no
    ray can pass by."""
    v = verts.astype(np.float32)
    key = {}
    edges = []
    for t in tris:
        for e in range(3):
            a, b = v[t[e]].tobytes(), v[t[(e + 1) % 3]].tobytes()
            k = (a, b) if a < b else (b, a)
            key[k] = key.get(k, 0) + 1
            edges.append((k, t[e], t[(e + 1) % 3]))
    border_pos = set()
    for k, n in key.items():
        if n < 2:
            border_pos.update(k)
    mids = np.array([(v[i] + v[j]) * np.float32(0.5) for k, i, j in edges if key[k] >= 2], np.float32)
    corners = np.array([p for p in np.unique(v[tris.ravel()], axis=0) if p.tobytes() not in border_pos], np.float32)
    return np.unique(mids, axis=0), corners


def _aim(rng, targets, origins_box, n):
    tgt = targets[rng.integers(0, len(targets), n)]
    o = rng.uniform(*origins_box, size=(n, 3)).astype(np.float32)
    d = (tgt - o).astype(np.float64)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o, d.astype(np.float32), tgt


@pytest.mark.parametrize("mesh", ["grid", "heightfield", "corner"])
def test_rays_through_shared_edges_and_vertices_hit(mesh):
    torch = need_cuda()
    rng = np.random.default_rng(3)
    if mesh == "grid":
        verts, tris, uv = scenes._grid((-1.0, -1.0, 1.0), (2.0, 0, 0), (0, 2.0, 0), 64, (0.0, 0.0), (1.0, 1.0))
        box = (-0.3, 0.3)
    elif mesh == "heightfield":
        verts, tris, uv = scenes.heightfield_mesh(np.random.default_rng(4), n_vert=97)
        box = (-0.3, 0.3)
    else:
        verts, tris, uv = scenes.corner_mesh()
        box = (-0.1, 0.1)
    # targets on the walls only: seen from the camera side, the three walls
    # meet in concave seams, which a ray through them must hit; the box's
    # edges are convex silhouettes, where grazing the edge is a legitimate miss
    walls = tris[:3 * 338] if mesh == "corner" else tris
    mids, corners = _interior_targets(verts, walls)
    assert len(mids) > 100 and len(corners) > 20
    o1, d1, t1 = _aim(rng, mids, box, 20000)
    o2, d2, t2 = _aim(rng, corners, box, 20000)
    o, d, tgt = np.concatenate([o1, o2]), np.concatenate([d1, d2]), np.concatenate([t1, t2])
    c = ctx()
    h = c.upload(verts.astype(np.float32), tris.astype(np.int32), uv.astype(np.float32))
    try:
        t, tri = c.trace(h, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda())
        c.sync()
        t, tri = t.cpu().numpy(), tri.cpu().numpy()
    finally:
        c.free(h)
    miss = tri < 0
    assert not miss.any(), (int(miss.sum()), o[miss][:3], tgt[miss][:3])
    # the hit is where the ray was aimed, or nearer where the surface
    # occludes the target (the heightfield's bumps, the corner's box)
    dist = np.linalg.norm(tgt.astype(np.float64) - o, axis=1)
    assert np.all(t <= dist * (1 + 1e-5) + 1e-6)
    if mesh == "grid":
        np.testing.assert_allclose(t, dist, rtol=1e-5)
