"""Camera-pose refinement on the GPU (Sec. 3.2's Rc, tc): dpcs_scene_transform
moves the stored vertices rigidly and refits the tree (exact box unions, no
compounding, identity restores the upload); renders of the posed scene match
the oracle's render of the moved mesh; the central-difference pose gradient
matches the oracle's; and Adam on it pulls a perturbed pose back."""
import numpy as np
import pytest

from paper_2503_12174_gb300 import dpcs, pose, scenes
from gpu_util import GpuScene, crf_atol, need_cuda, pixel_parity

pytestmark = pytest.mark.gpu


def _posed_scene(sc, R, t):
    Rp2, tp2 = pose.posed_extrinsics(sc.Rp, sc.tp, R, t)
    verts = (sc.verts.astype(np.float64) @ np.asarray(R, np.float64).T + t).astype(np.float32)
    return sc.replace(verts=verts, Rp=Rp2.astype(np.float32), tp=tp2.astype(np.float32))


def test_transform_refits_exactly_without_compounding():
    need_cuda()
    sc = scenes.corner(res=16, tex=16, spp=2, bounces=2, seed=1)
    g = GpuScene(sc)
    try:
        T = len(sc.tris)
        _, _, child0, box0 = g.ctx.export(g.handle, T)
        R1, t1 = pose.rotation([0.05, -0.02, 0.1]), np.array([0.03, -0.01, 0.02])
        R2, t2 = pose.rotation([-0.03, 0.04, 0.0]), np.array([0.0, 0.02, -0.04])
        g.ctx.transform(g.handle, R1, t1)
        g.ctx.transform(g.handle, R2, t2)
        codes2, order2, child2, box2 = g.ctx.export(g.handle, T)
        np.testing.assert_array_equal(child2, child0)
        # internal boxes are exact unions of their children's boxes
        for i in range(T - 1):
            for k in range(2):
                ref = child2[i, k]
                if ref >= 0:
                    want = np.concatenate([np.minimum(box2[ref, 0, :3], box2[ref, 1, :3]),
                                           np.maximum(box2[ref, 0, 3:], box2[ref, 1, 3:])])
                    np.testing.assert_array_equal(box2[i, k], want)
        # leaves hold the moved triangles (FP32 transform, so to rounding)
        moved = sc.verts.astype(np.float64) @ R2.T + t2
        tb = np.concatenate([moved[sc.tris].min(axis=1), moved[sc.tris].max(axis=1)], axis=1)
        for i in range(T - 1):
            for k in range(2):
                if child2[i, k] < 0:
                    np.testing.assert_allclose(box2[i, k], tb[order2[~child2[i, k]]], atol=2e-6)
        # a fresh transform by (R2, t2) gives the same boxes: transforms map the stored positions
        g.ctx.transform(g.handle, R2, t2)
        _, _, _, box3 = g.ctx.export(g.handle, T)
        np.testing.assert_array_equal(box3.view(np.uint32), box2.view(np.uint32))
        g.ctx.transform(g.handle, np.eye(3), np.zeros(3))  # 1 x + 0 y + 0 z + 0 = x (up to the sign of zero)
        _, _, _, box4 = g.ctx.export(g.handle, T)
        np.testing.assert_array_equal(box4, box0)
        with pytest.raises(dpcs.DPCSError) as e:
            g.ctx.transform(g.handle, np.full((3, 3), np.nan), np.zeros(3))
        assert e.value.status == dpcs.DPCS_ERR_INVALID_ARG
    finally:
        g.close()


def test_posed_render_matches_oracle(orc):
    torch = need_cuda()
    sc = scenes.corner(res=32, tex=16, spp=4, bounces=3, seed=6)
    R, t = pose.rotation([0.03, -0.05, 0.02]), np.array([0.02, -0.015, 0.04])
    g = GpuScene(sc)
    try:
        g.ctx.transform(g.handle, R, t)
        v = pose.posed_view(g.view, R, t)
        Ec = torch.empty((sc.Hc, sc.Wc, 3), device=g.ctx.device)
        Ic, _ = g.ctx.render(g.handle, g.albedo, g.rough, g.Ip, v, g.params, sc.spp, sc.bounces, sc.seed, Ec=Ec)
        g.ctx.sync()
        Ec, Ic = Ec.cpu().numpy(), Ic.cpu().numpy()
    finally:
        g.close()
    psc = _posed_scene(sc, R, t)
    rEc, rIc = orc.render(psc)
    ok, info = pixel_parity(Ec, rEc)
    assert ok, info
    ok, info = pixel_parity(Ic, rIc, atol=crf_atol(psc, rEc))
    assert ok, info


def _pairs(orc, sc, rng, K, spp):
    Ips = [scenes.blob_image(rng, sc.Hp, sc.Wp) for _ in range(K)]
    caps = [orc.render(sc, Ip=Ips[i], spp=spp, seed=500 + i)[1] for i in range(K)]
    return Ips, caps


def test_pose_gradient_matches_oracle(orc):
    """The central-difference gradient of the mean L1 data term, GPU renders
    against oracle renders of the moved mesh with the same Philox keys."""
    torch = need_cuda()
    sc = scenes.corner(res=24, tex=16, spp=4, bounces=2, seed=7)
    rng = np.random.default_rng(8)
    K = 2
    Ips, caps = _pairs(orc, sc, rng, K, 16)
    xi0 = np.array([0.01, -0.008, 0.006, 0.01, -0.012, 0.02])
    g = GpuScene(sc)
    try:
        pairs = [(torch.from_numpy(Ips[i]).cuda(), torch.from_numpy(caps[i].astype(np.float32)).cuda())
                 for i in range(K)]
        pr = pose.PoseRefine(g.ctx, g.handle, g.view, g.params, g.albedo, g.rough, pairs, sc.spp, sc.bounces,
                             seed=sc.seed, xi0=xi0, h_rot=2e-3, h_trans=2e-3, lr=0.0, gradient="differences")
        L0 = pr.step()
        g.ctx.sync()
        grad = pr.g.cpu().numpy().astype(np.float64)
    finally:
        g.close()
    scale = 1.0 / (K * sc.Hc * sc.Wc * 3)

    def loss(x):
        R, t = pose.pose_of(x)
        psc = _posed_scene(sc, R, t)
        return sum(float(np.sum(np.abs(orc.render(psc, Ip=Ips[i], seed=sc.seed + i)[1] - caps[i]))) * scale
                   for i in range(K))

    ref = pose.central_differences(loss, xi0.astype(np.float32).astype(np.float64), pr.h)
    assert abs(L0 - loss(xi0.astype(np.float32).astype(np.float64))) <= 1e-3 * abs(L0)
    np.testing.assert_allclose(grad, ref, rtol=0.05, atol=0.02 * np.abs(ref).max())


def test_pose_refinement_recovers_the_pose(orc):
    """Captures rendered at the true pose (the identity); Adam on the
    central-difference gradient from a pose off by ~1 degree and ~2 cm
    shrinks the error."""
    torch = need_cuda()
    sc = scenes.corner(res=48, tex=32, spp=8, bounces=2, seed=9)
    rng = np.random.default_rng(10)
    K = 3
    Ips, caps = _pairs(orc, sc, rng, K, 32)
    xi0 = np.array([0.012, -0.01, 0.008, 0.015, -0.01, 0.02])
    g = GpuScene(sc)
    try:
        pairs = [(torch.from_numpy(Ips[i]).cuda(), torch.from_numpy(caps[i].astype(np.float32)).cuda())
                 for i in range(K)]
        pr = pose.PoseRefine(g.ctx, g.handle, g.view, g.params, g.albedo, g.rough, pairs, sc.spp, sc.bounces,
                             seed=3, xi0=xi0, h_rot=2e-3, h_trans=2e-3, lr=2e-3, gradient="differences")
        hist = [pr.step() for _ in range(40)]
        xi = pr.xi.cpu().numpy().astype(np.float64)
    finally:
        g.close()
    assert np.mean(hist[-5:]) < np.mean(hist[:3])
    assert np.linalg.norm(xi[:3]) < 0.5 * np.linalg.norm(xi0[:3]), xi
    assert np.linalg.norm(xi[3:]) < 0.5 * np.linalg.norm(xi0[3:]), xi
