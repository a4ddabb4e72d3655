"""The camera-pose gradient on the GPU (``dpcs_pose_backward``; Sec. 3.2
counts the pose Rc, tc among the scene parameters theta of Eq. 9).

Its three terms -- interior, pixel edges, silhouettes -- are compared with
the oracle's FP64 terms, which take every derivative of a smooth quantity by
central differences where the kernels use closed forms; both draw the same
Philox numbers, so they estimate the same sums sample for sample:
  - a glossy plane seen from a pose (no silhouette in view);
  - a quad hiding part of a wall (a silhouette in view);
  - the corner with its occluding box, three bounces and GGX lobes.
The oracle's gradient itself is pinned in tests/test_oracle_pose_gradient.py
(pixel quadrature of the plane's closed form; common-random-number
differences across an occluder).  Also: results repeat bit for bit and
accumulate, arguments are checked, and Adam on this gradient pulls a
perturbed pose back."""
import numpy as np
import pytest

from paper_2503_12174_gb300 import dpcs, pose, scenes
from gpu_util import GpuScene, need_cuda

pytestmark = pytest.mark.gpu

UNIT = np.eye(6)  # unit twists: the oracle's gradient along them is the wrench itself


def _posed(sc, xi, R0, t0):
    R, t = pose.pose_of(xi, R0, t0)
    Rp2, tp2 = pose.posed_extrinsics(sc.Rp, sc.tp, R, t)
    return sc.replace(verts=(sc.verts.astype(np.float64) @ R.T + t).astype(np.float32), Rp=Rp2.astype(np.float32),
                      tp=tp2.astype(np.float32))


def _plane():
    res = 16
    sc = scenes.plane(res=res)
    sc = sc.replace(Ip=np.full((res, res, 3), 0.6, np.float32), albedo=np.full((8, 8, 3), 0.5, np.float32),
                    rough=np.full((8, 8), 0.3, np.float32), Kp=scenes.intrinsics(res, res, 80.0), spp=64,
                    params=scenes.Params(gamma_p=(2.2,) * 3, gain_p=1.1, k_proj=1.3, ks=0.8, f0=0.04, jitter=1,
                                         gamma_c=(0.8, 0.9, 1.0)))
    return _posed(sc, np.array([0.01, 0.0, -0.02, 0.005, 0.0, 0.01]), pose.rotation([0.02, -0.03, 0.1]),
                  np.array([0.01, 0.02, 0.05]))


def _quad(c, half, z, rot_deg):
    cs, sn = np.cos(np.radians(rot_deg)), np.sin(np.radians(rot_deg))
    return np.array([[c[0] + cs * half * u - sn * half * v, c[1] + sn * half * u + cs * half * v, z]
                     for u, v in [(-1, -1), (1, -1), (1, 1), (-1, 1)]], np.float32)


def _occluder(res=24):
    """A quad at z = 1.2 (turned 20 degrees) in front of a wide quad at z = 2,
    both lit directly by a wide projector; Lambert, one bounce."""
    verts = np.concatenate([_quad((0.0, 0.0), 2.0, 2.0, 0.0), _quad((0.05, -0.03), 0.18, 1.2, 20.0)])
    tris = np.array([[0, 1, 2], [0, 2, 3], [4, 5, 6], [4, 6, 7]], np.int32)
    uv = np.array([[0, 0], [1, 0], [1, 1], [0, 1]] * 2, np.float32)
    return scenes.Scene(verts=verts, tris=tris, uv=uv, albedo=np.full((8, 8, 3), 0.6, np.float32),
                        rough=np.full((8, 8), 0.4, np.float32), Ip=np.full((16, 16, 3), 0.7, np.float32),
                        Kc=scenes.intrinsics(res, res, 40.0), Hc=res, Wc=res, Kp=scenes.intrinsics(16, 16, 80.0),
                        Rp=np.eye(3, dtype=np.float32), tp=np.array([-0.3, 0.1, 0.0], np.float32),
                        params=scenes.Params(gamma_p=(2.2,) * 3, k_proj=2.0, ks=0.0, jitter=1), spp=64, bounces=1,
                        seed=0, name="occluder")


def _corner():
    sc = scenes.corner(res=24, tex=16, spp=8, bounces=3, seed=4)
    return _posed(sc, np.array([0.02, -0.01, 0.015, 0.01, 0.02, -0.03]), np.eye(3), np.zeros(3))


def _gpu(sc, W, edge_spp, sil_spp, g=None):
    torch = need_cuda()
    own = g is None
    g = GpuScene(sc) if own else g
    try:
        Ec, Ic = g.render()
        dIc = torch.from_numpy(np.ascontiguousarray(W, np.float32)).to(g.ctx.device)
        w = g.ctx.pose_backward(g.handle, g.albedo, g.rough, g.Ip, g.view, g.params, sc.spp, sc.bounces, sc.seed, Ec,
                                Ic, dIc, edge_spp, sil_spp)
        g.ctx.sync()
        return w.cpu().numpy()
    finally:
        if own:
            g.close()


def _oracle(orc, sc, W, edge_spp, sil_spp):
    Ec, _ = orc.render(sc)
    return orc.pose_backward(sc, W * orc.crf_grad(Ec, sc.params), UNIT, edge_spp, sil_spp)


# Both sides sum the same samples.  The kernels' closed-form derivatives and
# FP32 paths differ from the oracle's FP64 differences by ~1e-5 relative per
# sample; the tolerance leaves room for the few samples whose path FP32
# resolves differently (a ray grazing an edge), each worth about 1/N of a term.
@pytest.mark.parametrize("case, edge_spp, sil_spp, rtol", [
    ("plane", 64, 64, 2e-3),
    ("occluder", 64, 64, 5e-3),
    ("corner", 16, 16, 1e-2),
])
def test_pose_wrench_matches_oracle(orc, case, edge_spp, sil_spp, rtol):
    sc = {"plane": _plane, "occluder": _occluder, "corner": _corner}[case]()
    W = np.random.default_rng(11).uniform(0.5, 1.5, (sc.Hc, sc.Wc, 3))
    got = _gpu(sc, W, edge_spp, sil_spp)
    ref = _oracle(orc, sc, W, edge_spp, sil_spp)
    scale = np.abs(ref).max()
    assert scale > 0.0
    for t, name in enumerate(("interior", "pixel edges", "silhouettes")):
        err = np.abs(got[t] - ref[t])
        assert np.all(err <= rtol * np.abs(ref[t]).max() + 1e-6 * scale), (name, got[t], ref[t])
    # the summed wrench, as a pose step uses it
    tot_g, tot_r = got.sum(0), ref.sum(0)
    assert np.all(np.abs(tot_g - tot_r) <= rtol * np.abs(tot_r).max()), (tot_g, tot_r)
    if case == "occluder":
        # the silhouette carries a visible share of the translations
        assert np.abs(ref[2, 3:]).max() > 0.05 * np.abs(ref[:, 3:].sum(0)).max()
    if case == "plane":
        assert np.all(got[2] == 0.0) and np.all(ref[2] == 0.0)  # no silhouette inside the image


def test_pose_wrench_repeats_and_accumulates():
    torch = need_cuda()
    sc = _occluder(16)
    W = np.random.default_rng(2).uniform(0.5, 1.5, (sc.Hc, sc.Wc, 3))
    g = GpuScene(sc)
    try:
        Ec, Ic = g.render()
        dIc = torch.from_numpy(W.astype(np.float32)).to(g.ctx.device)

        def call(edge_spp, sil_spp, wrench=None):
            return g.ctx.pose_backward(g.handle, g.albedo, g.rough, g.Ip, g.view, g.params, sc.spp, sc.bounces,
                                       sc.seed, Ec, Ic, dIc, edge_spp, sil_spp, wrench=wrench)
        a = call(16, 16).cpu().numpy()
        b = call(16, 16)
        call(16, 16, wrench=b)
        b = b.cpu().numpy()
        only_interior = call(0, 0).cpu().numpy()
        np.testing.assert_array_equal(b, 2.0 * a)  # every call adds the same sums
        np.testing.assert_array_equal(only_interior[0], a[0])
        assert np.all(only_interior[1:] == 0.0)
        for bad in [(-1, 4), (4, -1), (1 << 17, 4)]:
            with pytest.raises(dpcs.DPCSError) as e:
                call(*bad)
            assert e.value.status == dpcs.DPCS_ERR_INVALID_ARG
        skew = dpcs.view_of(sc.replace(Kc=np.array([[40.0, 0, 8], [0, 40.0, 8], [0.01, 0, 1]], np.float32)))
        with pytest.raises(dpcs.DPCSError) as e:
            g.ctx.pose_backward(g.handle, g.albedo, g.rough, g.Ip, skew, g.params, sc.spp, sc.bounces, sc.seed, Ec,
                                Ic, dIc, 4, 4)
        assert e.value.status == dpcs.DPCS_ERR_INVALID_ARG
        # the edge table survives a rigid transform: gradients at the moved pose
        # equal those of the same mesh uploaded already moved
        R, t = pose.rotation([0.01, 0.02, -0.01]), np.array([0.01, -0.02, 0.03])
        g.ctx.transform(g.handle, R, t)
        g.view = pose.posed_view(g.view, R, t)
        moved = g.ctx.pose_backward(g.handle, g.albedo, g.rough, g.Ip, g.view, g.params, sc.spp, sc.bounces, sc.seed,
                                    *g.render(), dIc, 16, 16)
    finally:
        g.close()
    ref = _gpu(sc.replace(verts=(sc.verts.astype(np.float64) @ np.asarray(R).T + t).astype(np.float32),
                          Rp=pose.posed_extrinsics(sc.Rp, sc.tp, R, t)[0].astype(np.float32),
                          tp=pose.posed_extrinsics(sc.Rp, sc.tp, R, t)[1].astype(np.float32)), W, 16, 16)
    # the two meshes differ by the rounding of the FP32 transform on the device
    np.testing.assert_allclose(moved.cpu().numpy(), ref, rtol=2e-3, atol=1e-4 * np.abs(ref).max())


def _pairs(orc, sc, rng, K, spp):
    Ips = [scenes.blob_image(rng, sc.Hp, sc.Wp) for _ in range(K)]
    caps = [orc.render(sc, Ip=Ips[i], spp=spp, seed=500 + i)[1] for i in range(K)]
    return Ips, caps


def test_adjoint_pose_refinement_recovers_the_pose(orc):
    """Captures rendered at the true pose (the identity); Adam on the adjoint
    pose gradient, one render and one pose adjoint per pair and step, from a
    pose off by ~1 degree and ~2.7 cm lowers the loss and the pose error.
    The bounds hold for an FP64 emulation of the same loop with the oracle's
    pose adjoint under several key sets (rotation and translation errors
    ending at 0.37-0.61 and 0.44-0.58 of their start): the adjoint is
    unbiased but noisier than common-random-number differences under an L1
    residual of 8-spp renders."""
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
                             seed=3, xi0=xi0, lr=2e-3, gradient="adjoint", edge_spp=64, sil_spp=16)
        hist = [pr.step() for _ in range(40)]
        xi = pr.xi.cpu().numpy().astype(np.float64)
    finally:
        g.close()
    assert np.mean(hist[-5:]) < 0.85 * np.mean(hist[:3])
    assert np.linalg.norm(xi[:3]) < 0.75 * np.linalg.norm(xi0[:3]), xi
    assert np.linalg.norm(xi[3:]) < 0.75 * np.linalg.norm(xi0[3:]), xi


def test_pose_wrench_at_the_benchmark_size(orc):
    """The pose step's configuration in the benchmark: the corner at
    256 x 256, 16 spp, 3 bounces, 16 samples per pixel edge and per
    silhouette edge, an L1 residual's sign for dLoss/dIc, carried through the
    corner's camera response (gamma_c 0.45-0.55).  The oracle runs in its timing mode, whose hits
    are the brute-force hits bit for bit."""
    torch = need_cuda()
    sc = scenes.corner(res=256, tex=256, spp=16, bounces=3, seed=6000)
    W = np.sign(np.random.default_rng(21).normal(size=(sc.Hc, sc.Wc, 3))) / (sc.Hc * sc.Wc * 3)
    got = _gpu(sc, W, 16, 16)
    Ec, _ = orc.render(sc, accel=True)
    ref = orc.pose_backward(sc, W * orc.crf_grad(Ec, sc.params), UNIT, 16, 16, accel=True)
    scale = np.abs(ref).max()
    assert scale > 0.0
    for t, name in enumerate(("interior", "pixel edges", "silhouettes")):
        err = np.abs(got[t] - ref[t])
        assert np.all(err <= 1e-2 * np.abs(ref[t]).max() + 1e-6 * scale), (name, got[t], ref[t])
    tot_g, tot_r = got.sum(0), ref.sum(0)
    assert np.all(np.abs(tot_g - tot_r) <= 1e-2 * np.abs(tot_r).max()), (tot_g, tot_r)


def test_pose_wrench_degenerate_cases():
    """A zero dLoss/dIc, and a scene without triangles, give a zero wrench."""
    torch = need_cuda()
    sc = _occluder(16)
    got = _gpu(sc, np.zeros((sc.Hc, sc.Wc, 3)), 8, 8)
    assert np.all(got == 0.0)
    empty = sc.replace(verts=np.zeros((0, 3), np.float32), tris=np.zeros((0, 3), np.int32),
                       uv=np.zeros((0, 2), np.float32))
    got = _gpu(empty, np.ones((sc.Hc, sc.Wc, 3)), 8, 8)
    assert np.all(got == 0.0)


def _gpu_pbr(sc, m, nm, W, edge_spp, sil_spp):
    torch = need_cuda()
    g = GpuScene(sc)
    try:
        dev = g.ctx.device
        mt = torch.from_numpy(np.ascontiguousarray(m, np.float32)).to(dev)
        nt = torch.from_numpy(np.ascontiguousarray(nm, np.float32)).to(dev)
        Ec = torch.empty((sc.Hc, sc.Wc, 3), dtype=torch.float32, device=dev)
        Ic, _ = g.ctx.render_principled(g.handle, g.albedo, g.rough, mt, nt, g.Ip, g.view, g.params, sc.spp,
                                        sc.bounces, sc.seed, Ec=Ec)
        dIc = torch.from_numpy(np.ascontiguousarray(W, np.float32)).to(dev)
        w = g.ctx.pose_backward_principled(g.handle, g.albedo, g.rough, mt, nt, g.Ip, g.view, g.params, sc.spp,
                                           sc.bounces, sc.seed, Ec, Ic, dIc, edge_spp, sil_spp)
        g.ctx.sync()
        return w.cpu().numpy()
    finally:
        g.close()


@pytest.mark.parametrize("case, rtol", [("plane", 2e-3), ("corner", 1e-2)])
def test_principled_pose_wrench_matches_oracle(orc, case, rtol):
    """The principled material (metallic and normal maps): the first
    vertex's BRDF is the principled lobe at the shading normal."""
    if case == "plane":
        sc = _plane()
        m = np.full((8, 8), 0.6, np.float32)
        nm = np.tile(np.array([0.62, 0.42, 0.9], np.float32), (8, 8, 1))
    else:
        sc = scenes.with_principled(_corner())
        m, nm = sc.metallic, sc.normal
    W = np.random.default_rng(12).uniform(0.5, 1.5, (sc.Hc, sc.Wc, 3))
    got = _gpu_pbr(sc, m, nm, W, 16, 16)
    Ec, _ = orc.render(sc, metallic=m, normal=nm)
    ref = orc.pose_backward(sc, W * orc.crf_grad(Ec, sc.params), UNIT, 16, 16, metallic=m, normal=nm)
    scale = np.abs(ref).max()
    assert scale > 0.0
    for t, name in enumerate(("interior", "pixel edges", "silhouettes")):
        err = np.abs(got[t] - ref[t])
        assert np.all(err <= rtol * np.abs(ref[t]).max() + 1e-6 * scale), (name, got[t], ref[t])
    # flat maps: the plain material's wrench
    if case == "plane":
        flat = _gpu_pbr(sc, np.zeros((8, 8)), np.tile([0.5, 0.5, 1.0], (8, 8, 1)), W, 16, 16)
        plain = _gpu(sc, W, 16, 16)
        np.testing.assert_allclose(flat, plain, rtol=1e-4, atol=1e-6 * np.abs(plain).max())
