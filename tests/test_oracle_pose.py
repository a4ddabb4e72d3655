"""Pins of the camera-pose convention (Sec. 3.2's Rc, tc): the Rodrigues map
against scipy's rotation vectors, and the oracle's render of a posed plane
(mesh moved by (R, t), projector extrinsics by ``posed_extrinsics``)
against the direct-light closed form evaluated in the moved camera's frame;
the pose gradient by central differences against the same closed form."""
import math

import numpy as np
import pytest

from paper_2503_12174_gb300 import pose, scenes

Rotation = pytest.importorskip("scipy.spatial.transform").Rotation


def test_rotation_is_scipys_rotation_vector():
    rng = np.random.default_rng(0)
    for w in list(rng.normal(size=(20, 3))) + [np.array([1e-9, -2e-9, 0.5e-9]), np.zeros(3)]:
        np.testing.assert_allclose(pose.rotation(w), Rotation.from_rotvec(w).as_matrix(), atol=1e-14)
    R = pose.rotation([0.3, -0.2, 0.9])
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
    assert abs(np.linalg.det(R) - 1.0) < 1e-14


def _plane_closed_form(sc, R, t, c, gamma, k, gain, rho):
    """Ec of the plane z = 1 (normal -z) seen from a camera at pose (R, t):
    in the camera frame the plane passes through R (0,0,1) + t with normal
    R e_z, the projector centre is R cp + t and its axis R e_z."""
    Kinv = np.linalg.inv(np.asarray(sc.Kc, np.float64))
    ys, xs = np.mgrid[0:sc.Hc, 0:sc.Wc]
    d = np.stack([xs + 0.5, ys + 0.5, np.ones_like(xs, dtype=np.float64)], -1) @ Kinv.T
    n = R @ np.array([0.0, 0.0, 1.0])
    p0 = R @ np.array([0.0, 0.0, 1.0]) + t
    s = (p0 @ n) / (d @ n)
    x = d * s[..., None]
    cp_world = -np.asarray(sc.Rp, np.float64).T @ np.asarray(sc.tp, np.float64)
    cp = R @ cp_world + t
    axis = R @ np.array([0.0, 0.0, 1.0])
    v = cp - x
    r = np.linalg.norm(v, axis=-1)
    wp = v / r[..., None]
    nf = np.where(((d @ n) > 0)[..., None], -n, n)  # the normal turned towards the camera
    cos_s = np.sum(nf * wp, axis=-1)
    cos_p = ((x - cp) @ axis) / r
    pw = (x - t) @ R  # world coordinates R^T (x - t)
    q = (pw @ np.asarray(sc.Rp, np.float64).T + np.asarray(sc.tp, np.float64)) @ np.asarray(sc.Kp, np.float64).T
    u, vv = q[..., 0] / q[..., 2], q[..., 1] / q[..., 2]
    inside = (u >= 0) & (u < sc.Wp) & (vv >= 0) & (vv < sc.Hp) & (cos_s > 0)
    return np.where(inside, rho / math.pi * k * gain * c ** gamma * cos_p * cos_s / r ** 2, 0.0)


def _posed_scene(sc, R, t):
    Rp2, tp2 = pose.posed_extrinsics(sc.Rp, sc.tp, R, t)
    verts = (sc.verts.astype(np.float64) @ R.T + t).astype(np.float32)
    return sc.replace(verts=verts, Rp=Rp2.astype(np.float32), tp=tp2.astype(np.float32))


def _plane(c=0.6, gamma=2.2, k=1.3, gain=1.1, rho=0.55):
    sc = scenes.plane(res=40)
    return sc.replace(Ip=np.full((40, 40, 3), c, np.float32), albedo=np.full((8, 8, 3), rho, np.float32),
                      params=scenes.Params(gamma_p=(gamma,) * 3, gain_p=gain, k_proj=k, ks=0.0, jitter=0))


@pytest.mark.parametrize("omega,t", [((0.0, 0.0, 0.3), (0.02, -0.01, 0.1)), ((0.15, -0.1, 0.05), (0.0, 0.03, -0.05))])
def test_posed_plane_direct_light_closed_form(orc, omega, t):
    sc = _plane()
    R, t = pose.rotation(omega), np.asarray(t, np.float64)
    Ec, _ = orc.render(_posed_scene(sc, R, t))
    expect = _plane_closed_form(sc, R, t, float(np.float32(0.6)), 2.2, 1.3, 1.1, float(np.float32(0.55)))
    assert (expect > 0).mean() > 0.3
    lit = expect > 0
    # float32 vertices and extrinsics: the plane itself moves by ~1e-7
    np.testing.assert_allclose(Ec[..., 0][lit], expect[lit], rtol=2e-6)
    edge = np.abs(Ec[..., 0] - expect) > 2e-6 * np.abs(expect) + 1e-12
    assert edge.mean() < 0.01  # only pixels on the frustum border may flip


def test_pose_gradient_central_differences_follow_the_closed_form(orc):
    """The FD pose gradient of sum(W * Ec) through oracle renders equals the
    FD gradient of the closed form with the same steps, and both equal the
    closed form's gradient at a finer step.  W is zero near the projector
    frustum's border, where Ec jumps (the visibility terms): away from it
    the image is smooth in the pose."""
    ndimage = pytest.importorskip("scipy.ndimage")
    sc = _plane()
    rng = np.random.default_rng(3)
    R0, t0 = pose.rotation([0.02, -0.03, 0.1]), np.array([0.01, 0.02, 0.05])
    xi = np.array([0.01, 0.0, -0.02, 0.005, 0.0, 0.01])
    R, t = pose.pose_of(xi, R0, t0)
    inner = ndimage.binary_erosion(_plane_closed_form(sc, R, t, 0.6, 2.2, 1.3, 1.1, 0.55) > 0, iterations=3)
    assert inner.mean() > 0.2
    W = np.where(inner, rng.uniform(0.5, 1.5, (sc.Hc, sc.Wc)), 0.0)

    def closed(x):
        R, t = pose.pose_of(x, R0, t0)
        return float(np.sum(W * _plane_closed_form(sc, R, t, float(np.float32(0.6)), 2.2, 1.3, 1.1,
                                                   float(np.float32(0.55)))))

    def rendered(x):
        R, t = pose.pose_of(x, R0, t0)
        return float(np.sum(W * orc.render(_posed_scene(sc, R, t))[0][..., 0]))

    h = np.array([2e-3] * 3 + [2e-3] * 3)
    g_closed = pose.central_differences(closed, xi, h)
    g_render = pose.central_differences(rendered, xi, h)
    g_fine = pose.central_differences(closed, xi, h / 8)
    scale = np.abs(g_closed).max()
    assert scale > 0
    np.testing.assert_allclose(g_render, g_closed, atol=2e-3 * scale)
    np.testing.assert_allclose(g_closed, g_fine, atol=2e-3 * scale)
