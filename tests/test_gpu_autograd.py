"""The renderer as a torch.autograd.Function: its backward equals the direct
path-replay call, agrees with central finite differences of the GPU forward
on smooth parameters, and drives a torch optimiser; a camera pose given to it
gets the pose adjoint's gradient."""
import numpy as np
import pytest

from paper_2503_12174_gb300 import autograd, dpcs, scenes
from gpu_util import GpuScene, need_cuda

pytestmark = pytest.mark.gpu


def test_backward_equals_render_backward():
    torch = need_cuda()
    sc = scenes.corner(res=32, tex=16, spp=8, bounces=2, seed=2)
    g = GpuScene(sc)
    try:
        W = torch.from_numpy(np.random.default_rng(0).normal(size=(sc.Hc, sc.Wc, 3)).astype(np.float32)).cuda()
        A = g.albedo.clone().requires_grad_(True)
        R = g.rough.clone().requires_grad_(True)
        P = g.Ip.clone().requires_grad_(True)
        pv = torch.tensor(autograd.params_vector(g.params), device="cuda", requires_grad=True)
        Ic = autograd.render(g.ctx, g.handle, A, R, P, g.view, g.params, sc.spp, sc.bounces, sc.seed, pvec=pv)
        (Ic * W).sum().backward()
        Ec = torch.empty_like(W)
        Ic2, _ = g.ctx.render(g.handle, g.albedo, g.rough, g.Ip, g.view, g.params, sc.spp, sc.bounces, sc.seed, Ec=Ec)
        ref = {"dIp": torch.zeros_like(g.Ip), "dA": torch.zeros_like(g.albedo), "dR": torch.zeros_like(g.rough),
               "dP": torch.zeros(11, device="cuda")}
        g.ctx.render_backward(g.handle, g.albedo, g.rough, g.Ip, g.view, g.params, sc.spp, sc.bounces, sc.seed, Ec, Ic2,
                              W, dIp=ref["dIp"], dAlbedo=ref["dA"], dRough=ref["dR"], dParams=ref["dP"])
        g.ctx.sync()
        assert torch.equal(Ic.detach(), Ic2)
        for got, want in ((P.grad, ref["dIp"]), (A.grad, ref["dA"]), (R.grad, ref["dR"]), (pv.grad, ref["dP"])):
            a, b = got.cpu().numpy(), want.cpu().numpy()
            np.testing.assert_allclose(a, b, rtol=1e-4, atol=1e-6 * np.abs(b).max())
    finally:
        g.close()


def test_gradient_matches_central_differences_on_the_gpu():
    """Central differences of the GPU forward (fixed seed, so the same paths)
    for the projector gain, the camera gamma and two projector texels.  The
    forward is FP32, so the step is 1e-2 relative and the bar 2 %."""
    torch = need_cuda()
    sc = scenes.corner(res=48, tex=16, spp=16, bounces=2, seed=3)
    g = GpuScene(sc)
    try:
        W = torch.from_numpy(np.random.default_rng(1).uniform(0.5, 1.5, (sc.Hc, sc.Wc, 3)).astype(np.float32)).cuda()
        pv0 = torch.tensor(autograd.params_vector(g.params), device="cuda")

        def loss(P, pv):
            Ic = autograd.render(g.ctx, g.handle, g.albedo, g.rough, P, g.view, g.params, sc.spp, sc.bounces,
                                 sc.seed, pvec=pv)
            return (Ic * W).double().sum()

        P = g.Ip.clone().requires_grad_(True)
        pv = pv0.clone().requires_grad_(True)
        loss(P, pv).backward()
        gP, gv = P.grad.clone(), pv.grad.clone()
        with torch.no_grad():
            for k in (3, 5):  # Gp, gamma_c[1]
                h = 1e-2 * float(pv0[k])
                up, dn = pv0.clone(), pv0.clone()
                up[k] += h
                dn[k] -= h
                fd = (loss(g.Ip, up) - loss(g.Ip, dn)).item() / (2 * h)
                assert fd == pytest.approx(gv[k].item(), rel=2e-2), k
            flat = gP.reshape(-1).abs()
            for idx in torch.topk(flat, 2).indices.tolist():  # two strongly lit texels
                h = 1e-2
                up, dn = g.Ip.clone(), g.Ip.clone()
                up.view(-1)[idx] += h
                dn.view(-1)[idx] -= h
                fd = (loss(up, pv0) - loss(dn, pv0)).item() / (2 * h)
                assert fd == pytest.approx(gP.view(-1)[idx].item(), rel=2e-2), idx
    finally:
        g.close()


def test_torch_optimizer_compensates():
    """Projector compensation written with torch.optim.Adam over the
    autograd render: the loss against a target falls."""
    torch = need_cuda()
    sc = scenes.corner(res=32, tex=16, spp=8, bounces=2, seed=4)
    g = GpuScene(sc)
    try:
        target, _ = g.ctx.render(g.handle, g.albedo, g.rough,
                                 torch.from_numpy(np.random.default_rng(2).random(sc.Ip.shape, dtype=np.float32)).cuda(),
                                 g.view, g.params, 64, sc.bounces, 99)
        P = torch.full_like(g.Ip, 0.5).requires_grad_(True)
        opt = torch.optim.Adam([P], lr=0.05)
        hist = []
        for k in range(15):
            opt.zero_grad()
            Ic = autograd.render(g.ctx, g.handle, g.albedo, g.rough, P, g.view, g.params, sc.spp, sc.bounces, k)
            loss = 0.5 * ((Ic - target) ** 2).sum()
            loss.backward()
            opt.step()
            with torch.no_grad():
                P.clamp_(0.0, 1.0)
            hist.append(loss.item())
        assert np.mean(hist[-3:]) < 0.5 * hist[0]
    finally:
        g.close()


def test_principled_backward_equals_render_backward_principled():
    """With metallic and normal maps the Function routes to the principled
    calls; every gradient, the maps' included, equals the direct adjoint."""
    torch = need_cuda()
    sc = scenes.with_principled(scenes.corner(res=32, tex=16, spp=8, bounces=2, seed=4), seed=9)
    g = GpuScene(sc)
    try:
        W = torch.from_numpy(np.random.default_rng(2).normal(size=(sc.Hc, sc.Wc, 3)).astype(np.float32)).cuda()
        m0 = torch.from_numpy(sc.metallic).cuda()
        n0 = torch.from_numpy(sc.normal).cuda()
        A = g.albedo.clone().requires_grad_(True)
        M = m0.clone().requires_grad_(True)
        N = n0.clone().requires_grad_(True)
        Ic = autograd.render(g.ctx, g.handle, A, g.rough, g.Ip, g.view, g.params, sc.spp, sc.bounces, sc.seed,
                             metallic=M, normal=N)
        (Ic * W).sum().backward()
        Ec = torch.empty_like(W)
        Ic2, _ = g.ctx.render_principled(g.handle, g.albedo, g.rough, m0, n0, g.Ip, g.view, g.params, sc.spp,
                                         sc.bounces, sc.seed, Ec=Ec)
        ref = {"dA": torch.zeros_like(g.albedo), "dM": torch.zeros_like(m0), "dN": torch.zeros_like(n0)}
        g.ctx.render_backward_principled(g.handle, g.albedo, g.rough, m0, n0, g.Ip, g.view, g.params, sc.spp,
                                         sc.bounces, sc.seed, Ec, Ic2, W, dAlbedo=ref["dA"], dMetallic=ref["dM"],
                                         dNormal=ref["dN"])
        g.ctx.sync()
        assert torch.equal(Ic.detach(), Ic2)
        for got, want in ((A.grad, ref["dA"]), (M.grad, ref["dM"]), (N.grad, ref["dN"])):
            a, b = got.cpu().numpy(), want.cpu().numpy()
            assert np.abs(b).max() > 0
            np.testing.assert_allclose(a, b, rtol=1e-4, atol=1e-6 * np.abs(b).max())
    finally:
        g.close()


def test_pose_input_gradient_is_the_pose_adjoint():
    """A camera pose given to the wrapper: the forward renders the scene moved
    to it, and its gradient is the pose adjoint's wrench projected on the
    pose parameters' twists, under the adjoint's own key."""
    torch = need_cuda()
    from paper_2503_12174_gb300 import pose

    sc = scenes.corner(res=24, tex=16, spp=8, bounces=2, seed=3)
    R0, t0 = pose.rotation([0.01, -0.02, 0.015]), np.array([0.01, 0.0, -0.02])
    x0 = np.array([0.004, -0.003, 0.002, 0.005, 0.0, -0.004])
    W = torch.from_numpy(np.random.default_rng(9).uniform(0.5, 1.5, (sc.Hc, sc.Wc, 3)).astype(np.float32)).cuda()
    g = GpuScene(sc)
    try:
        xi = torch.tensor(x0, dtype=torch.float64, requires_grad=True)
        Ic = autograd.render(g.ctx, g.handle, g.albedo, g.rough, g.Ip, g.view, g.params, sc.spp, sc.bounces, sc.seed,
                             pose=xi, pose_R0=R0, pose_t0=t0, edge_spp=8, sil_spp=8)
        (Ic * W).sum().backward()
        got = xi.grad.numpy().copy()
        # the same by hand
        R, t = pose.pose_of(x0, R0, t0)
        g.ctx.transform(g.handle, R, t)
        v = pose.posed_view(g.view, R, t)
        Ec = torch.empty_like(Ic)
        Ic2, _ = g.ctx.render(g.handle, g.albedo, g.rough, g.Ip, v, g.params, sc.spp, sc.bounces, sc.seed, Ec=Ec)
        np.testing.assert_array_equal(Ic2.cpu().numpy(), Ic.detach().cpu().numpy())
        Wr = g.ctx.pose_backward(g.handle, g.albedo, g.rough, g.Ip, v, g.params, sc.spp, sc.bounces,
                                 pose.adjoint_key(sc.seed), Ec, Ic2, W, 8, 8)
        ref = pose.project(Wr.cpu().numpy(), pose.twists(x0, R0, t0))
    finally:
        g.close()
    assert np.abs(ref).max() > 0.0
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0.0)
