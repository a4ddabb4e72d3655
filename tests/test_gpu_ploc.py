"""The clustered tree (PLOC over the Morton order, the default builder):
a valid binary tree over the same leaves, rooted at node 0, with exact
FP32 boxes, no deeper than the traversal stack, built the same way every
time; a lower surface-area cost than the radix tree; and closest hits, and
so renders, identical to the radix tree's."""
import numpy as np
import pytest

from paper_2503_12174_gb300 import dpcs, scenes
from gpu_util import GpuScene, ctx, need_cuda

pytestmark = pytest.mark.gpu


def _meshes():
    rng = np.random.default_rng(3)
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
    yield "three", rng.random((9, 3)).astype(np.float32), np.arange(9, dtype=np.int32).reshape(3, 3), \
        np.zeros((9, 2), np.float32)


def _upload(c, builder, verts, tris, uv):
    c.set_bvh_builder(builder)
    try:
        return c.upload(verts, tris, uv)
    finally:
        c.set_bvh_builder(dpcs.DPCS_BVH_PLOC)


def _area(b):
    d = np.maximum(b[..., 3:] - b[..., :3], 0.0)
    return 2.0 * (d[..., 0] * d[..., 1] + d[..., 1] * d[..., 2] + d[..., 2] * d[..., 0])


def _check_tree(verts, tris, order, child, box):
    """Every leaf once, every internal node but the root (0) once, child boxes
    exact: a leaf's = its triangle's min/max, an internal node's = the union
    of its children's.  Returns the depth and the summed internal-node area
    over the root's (the expected node visits of a random ray, up to a
    constant)."""
    T = len(tris)
    refs = child.ravel()
    leaves = np.sort(~refs[refs < 0])
    np.testing.assert_array_equal(leaves, np.arange(T))
    inner = np.sort(refs[refs >= 0])
    np.testing.assert_array_equal(inner, np.arange(1, T - 1))
    v = verts.astype(np.float32)[tris[order]]
    tb = np.concatenate([v.min(axis=1), v.max(axis=1)], axis=1)
    nb = np.concatenate([np.minimum(box[:, 0, :3], box[:, 1, :3]), np.maximum(box[:, 0, 3:], box[:, 1, 3:])], 1)
    for k in range(2):
        r = child[:, k]
        lf = r < 0
        np.testing.assert_array_equal(box[lf, k], tb[~r[lf]])
        np.testing.assert_array_equal(box[~lf, k], nb[r[~lf]])
    depth = np.zeros(T - 1, np.int64)
    depth[0] = 1
    parent = np.full(T - 1, -1)
    for i in range(T - 1):
        for k in range(2):
            if child[i, k] >= 0:
                parent[child[i, k]] = i
    order_nodes = [0]
    for i in order_nodes:
        for k in range(2):
            if child[i, k] >= 0:
                depth[child[i, k]] = depth[i] + 1
                order_nodes.append(child[i, k])
    return int(depth.max()), float(_area(nb).sum() / _area(nb[0]))


@pytest.mark.parametrize("case", list(range(6)))
def test_clustered_tree_is_valid_and_deterministic(orc, case):
    need_cuda()
    name, verts, tris, uv = list(_meshes())[case]
    c = ctx()
    hp = _upload(c, dpcs.DPCS_BVH_PLOC, verts, tris, uv)
    hq = _upload(c, dpcs.DPCS_BVH_PLOC, verts, tris, uv)
    hl = _upload(c, dpcs.DPCS_BVH_LBVH, verts, tris, uv)
    try:
        T = len(tris)
        codes, order, child, box = c.export(hp, T)
        codes2, order2, child2, box2 = c.export(hq, T)
        codesl, orderl, childl, boxl = c.export(hl, T)
    finally:
        for h in (hp, hq, hl):
            c.free(h)
    # the same codes and leaf order as the radix tree, the same tree on a repeat
    np.testing.assert_array_equal(codes, codesl)
    np.testing.assert_array_equal(order, orderl)
    np.testing.assert_array_equal(child2, child)
    np.testing.assert_array_equal(box2.view(np.uint32), box.view(np.uint32))
    depth, cost = _check_tree(verts, tris, order, child, box)
    assert depth <= 64, (name, depth)
    _, cost_l = _check_tree(verts, tris, orderl, childl, boxl)
    # walls meeting at seams and a displaced grid gain most; a closed,
    # uniformly tessellated sphere already suits the Morton order
    if name in ("corner", "heightfield"):
        assert cost < 0.85 * cost_l, (name, cost, cost_l)
    if name == "sphere":
        assert cost < cost_l, (name, cost, cost_l)


@pytest.mark.parametrize("which", ["corner", "heightfield"])
def test_renders_equal_across_builders(which):
    """Closest hits do not depend on the tree (ties go to the lowest triangle
    index), so images and gradients are the same bit for bit."""
    torch = need_cuda()
    if which == "corner":
        sc = scenes.corner(res=64, tex=64, spp=8, bounces=3, seed=3)
    else:
        v, t, u = scenes.heightfield_mesh(np.random.default_rng(4), n_vert=101)
        sc = scenes.corner(res=64, tex=64, spp=8, bounces=3, seed=3).replace(verts=v, tris=t, uv=u)
    out = {}
    for builder in (dpcs.DPCS_BVH_LBVH, dpcs.DPCS_BVH_PLOC):
        c = ctx()
        c.set_bvh_builder(builder)
        try:
            g = GpuScene(sc)
        finally:
            c.set_bvh_builder(dpcs.DPCS_BVH_PLOC)
        try:
            Ec, Ic = g.render()
            dIc = torch.ones_like(Ic)
            out[builder] = (Ec.cpu().numpy(), g.backward(Ec, Ic, dIc))
        finally:
            g.close()
    (e0, g0), (e1, g1) = out[dpcs.DPCS_BVH_LBVH], out[dpcs.DPCS_BVH_PLOC]
    np.testing.assert_array_equal(e1.view(np.uint32), e0.view(np.uint32))
    for k in g0:
        # the adjoint's float4 atomics add in a scheduling-dependent order
        np.testing.assert_allclose(g1[k], g0[k], rtol=1e-4, atol=1e-6 * max(np.abs(g0[k]).max(), 1e-30))


def test_builder_setting_is_checked():
    need_cuda()
    with pytest.raises(dpcs.DPCSError) as e:
        ctx().set_bvh_builder(7)
    assert e.value.status == dpcs.DPCS_ERR_INVALID_ARG


def test_tight_budget_keeps_the_radix_tree_and_failed_uploads_free_their_memory():
    """The clustering is an optimisation: a context whose budget holds the
    scene, its staging and the radix tree's scratch but not the clustering's
    still uploads, with the radix tree.  An upload that fails on the budget
    frees what it had taken."""
    need_cuda()
    verts, tris, uv = scenes.corner_mesh()
    T, V = len(tris), len(verts)
    ref = dpcs.Context(0)
    ref.set_bvh_builder(dpcs.DPCS_BVH_LBVH)
    h = ref.upload(verts, tris, uv)
    need = ref.memory_used
    _, _, child_l, box_l = ref.export(h, T)
    ref.free(h)
    ref.close()
    tight = dpcs.Context(0, hbm_budget_bytes=need + 4096)
    try:
        h = tight.upload(verts, tris, uv)  # the default builder, PLOC, cannot have its scratch
        _, _, child, box = tight.export(h, T)
        np.testing.assert_array_equal(child, child_l)
        np.testing.assert_array_equal(box.view(np.uint32), box_l.view(np.uint32))
        tight.free(h)
    finally:
        tight.close()
    scene_bytes = (T - 1) * 64 + T * 48 + T * 24 + T * 8 + T * 12 + V * 8 + V * 12
    probe = dpcs.Context(0)
    base = probe.memory_used  # the context's own status word and counters
    probe.close()
    small = dpcs.Context(0, hbm_budget_bytes=base + scene_bytes + 16)  # the scene fits, its staging does not
    try:
        assert small.memory_used == base
        with pytest.raises(dpcs.DPCSError) as e:
            small.upload(verts, tris, uv)
        assert e.value.status == dpcs.DPCS_ERR_OOM
        assert small.memory_used == base
    finally:
        small.close()
