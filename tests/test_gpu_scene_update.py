"""Moving an uploaded scene's vertices (dpcs_scene_update): the refit keeps
the tree and rewrites every box exactly as the min/max of what it holds;
closest hits and renders of the deformed scene match the oracle run on the
deformed mesh; restoring the original positions restores the original
boxes bit for bit."""
import numpy as np
import pytest

from paper_2503_12174_gb300 import dpcs, scenes
from gpu_util import GpuScene, crf_atol, ctx, need_cuda, pixel_parity

pytestmark = pytest.mark.gpu


def _deform(verts, amp=0.03):
    v = np.asarray(verts, np.float64)
    d = np.stack([np.sin(3.1 * v[:, 1] + 0.4), np.sin(2.7 * v[:, 2] + 1.1), np.sin(3.3 * v[:, 0] + 2.0)], axis=1)
    return (v + amp * d).astype(np.float32)


def _meshes():
    yield "corner", scenes.corner_mesh()
    yield "heightfield", scenes.heightfield_mesh(np.random.default_rng(4), n_vert=81)
    yield "sphere", scenes.icosphere(3)


def _check_boxes(verts, tris, order, child, box):
    """Every child box is exactly the min/max of its triangle's vertices (a
    leaf) or exactly the union of its node's two child boxes."""
    T = len(tris)
    tri_box = np.concatenate([verts[tris].min(axis=1), verts[tris].max(axis=1)], axis=1)  # original index
    for i in range(T - 1):
        for k in range(2):
            ref = child[i, k]
            if ref < 0:
                want = tri_box[order[~ref]]
            else:
                want = np.concatenate([np.minimum(box[ref, 0, :3], box[ref, 1, :3]),
                                       np.maximum(box[ref, 0, 3:], box[ref, 1, 3:])])
            np.testing.assert_array_equal(box[i, k], want, err_msg=f"node {i} child {k}")


@pytest.mark.parametrize("case", [0, 1, 2])
def test_refit_boxes_exact_and_topology_kept(case):
    need_cuda()
    name, (verts, tris, uv) = list(_meshes())[case]
    c = ctx()
    h = c.upload(verts, tris, uv)
    try:
        codes0, order0, child0, box0 = c.export(h, len(tris))
        moved = _deform(verts)
        c.update(h, moved)
        codes1, order1, child1, box1 = c.export(h, len(tris))
        np.testing.assert_array_equal(codes1, codes0)
        np.testing.assert_array_equal(order1, order0)
        np.testing.assert_array_equal(child1, child0)
        _check_boxes(moved, tris, order1, child1, box1)
        c.update(h, verts)  # back to the uploaded positions: the same boxes bit for bit
        _, _, _, box2 = c.export(h, len(tris))
        np.testing.assert_array_equal(box2.view(np.uint32), box0.view(np.uint32), err_msg=name)
    finally:
        c.free(h)


def test_closest_hits_after_update_match_brute_force(orc):
    torch = need_cuda()
    verts, tris, uv = scenes.heightfield_mesh(np.random.default_rng(4), n_vert=81)
    moved = _deform(verts, amp=0.05)
    rng = np.random.default_rng(12)
    o = rng.uniform(-0.5, 0.5, (20000, 3))
    o[:, 2] = -0.5
    d = rng.normal(size=(20000, 3))
    d[:, 2] = np.abs(d[:, 2]) + 0.3
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = o.astype(np.float32).astype(np.float64)
    d = d.astype(np.float32).astype(np.float64)
    c = ctx()
    h = c.upload(verts, tris, uv)
    try:
        c.update(h, moved)
        t, tri = c.trace(h, torch.from_numpy(o.astype(np.float32)).cuda(), torch.from_numpy(d.astype(np.float32)).cuda())
        c.sync()
        t, tri = t.cpu().numpy().astype(np.float64), tri.cpu().numpy()
    finally:
        c.free(h)
    rt, rtri = orc.closest(moved, tris, o, d)
    same = tri == rtri
    assert same.mean() >= 0.999, same.mean()
    hit = same & (rtri >= 0)
    assert hit.sum() > 1000
    np.testing.assert_allclose(t[hit], rt[hit], rtol=1e-5, atol=1e-6)


def test_render_after_update_matches_oracle(orc):
    """Relighting a deformed surface (Sec. 4.4): the GPU renders the
    refitted scene; the oracle renders the deformed mesh from scratch."""
    need_cuda()
    sc = scenes.corner(res=32, tex=16, spp=4, bounces=3, seed=2)
    moved = _deform(sc.verts, amp=0.02)
    g = GpuScene(sc)
    try:
        g.ctx.update(g.handle, moved)
        Ec, Ic = g.render()
        Ec, Ic = Ec.cpu().numpy(), Ic.cpu().numpy()
    finally:
        g.close()
    msc = sc.replace(verts=moved)
    rEc, rIc = orc.render(msc)
    ok, info = pixel_parity(Ec, rEc)
    assert ok, info
    ok, info = pixel_parity(Ic, rIc, atol=crf_atol(msc, rEc))
    assert ok, info


def test_update_refuses_bad_input():
    need_cuda()
    verts, tris, uv = scenes.corner_mesh()
    c = ctx()
    h = c.upload(verts, tris, uv)
    try:
        with pytest.raises(dpcs.DPCSError) as e:
            c.update(h, verts[:-1])
        assert e.value.status == dpcs.DPCS_ERR_INVALID_ARG
        bad = verts.copy()
        bad[3, 1] = np.nan
        with pytest.raises(dpcs.DPCSError) as e:
            c.update(h, bad)
        assert e.value.status == dpcs.DPCS_ERR_INVALID_ARG
        with pytest.raises(dpcs.DPCSError) as e:
            c.update(h + 12345, verts)
        assert e.value.status == dpcs.DPCS_ERR_NOT_FOUND
        c.update(h, verts)  # the scene still works
        c.sync()
    finally:
        c.free(h)


def test_compensation_on_a_deforming_surface(orc):
    """Compensation while the surface moves (Sec. 4.4 with Eq. 13): before
    each step the vertices take the frame's positions; each step's loss and
    Adam update follow the oracle run on that frame's mesh."""
    torch = need_cuda()
    sc = scenes.corner(res=20, tex=16, spp=4, bounces=2, seed=11)
    rng = np.random.default_rng(0)
    _, target = orc.render(sc, Ip=rng.random(sc.Ip.shape), seed=777)
    frames = [_deform(sc.verts, amp=0.01 * f) for f in range(3)]
    lr = 0.05
    g = GpuScene(sc)
    try:
        P = torch.full_like(g.Ip, 0.5)
        M, V, G = torch.zeros_like(P), torch.zeros_like(P), torch.zeros_like(P)
        tgt = torch.from_numpy(target.astype(np.float32)).cuda()
        loss = torch.zeros(1, device="cuda")
        losses = []
        for k, fv in enumerate(frames):
            g.ctx.update(g.handle, fv)
            G.zero_()
            g.ctx.render_loss_backward(g.handle, g.albedo, g.rough, P, g.view, g.params, sc.spp, sc.bounces,
                                       sc.seed + k, tgt, loss, loss_kind=0, dIp=G)
            losses.append(loss.item())
            g.ctx.adam(P, G, M, V, k + 1, lr=lr)
        g.ctx.sync()
        P = P.cpu().numpy().astype(np.float64)
    finally:
        g.close()
    Pr = np.full(sc.Ip.shape, 0.5)
    m, v = np.zeros_like(Pr), np.zeros_like(Pr)
    ref = []
    for k, fv in enumerate(frames):
        fsc = sc.replace(verts=fv)
        _, Ic = orc.render(fsc, Ip=Pr, seed=sc.seed + k)
        d = Ic - target
        ref.append(0.5 * np.sum(d * d))
        grad = orc.render_backward(fsc, d, Ip=Pr, seed=sc.seed + k)["dIp"]
        orc.adam_step(Pr, grad, m, v, k + 1, lr=lr)
    np.testing.assert_allclose(losses, ref, rtol=1e-3)
    np.testing.assert_allclose(P, Pr, rtol=0, atol=2e-3)
