"""Shared helpers of the GPU parity tests: upload a ``scenes.Scene``, render
through the C ABI, and compare with the FP64 oracle."""
import numpy as np
import pytest


def need_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    return torch


_CTX = None


def ctx():
    global _CTX
    torch = need_cuda()
    from paper_2503_12174_gb300 import dpcs

    if _CTX is None:
        _CTX = dpcs.Context(0)
    return _CTX


class GpuScene:
    """A scenes.Scene resident on the GPU."""

    def __init__(self, sc):
        torch = need_cuda()
        from paper_2503_12174_gb300 import dpcs

        self.sc = sc
        self.ctx = ctx()
        self.handle = self.ctx.upload(sc.verts, sc.tris, sc.uv)
        dev = self.ctx.device
        self.albedo = torch.from_numpy(np.ascontiguousarray(sc.albedo)).to(dev)
        self.rough = torch.from_numpy(np.ascontiguousarray(sc.rough)).to(dev)
        self.Ip = torch.from_numpy(np.ascontiguousarray(sc.Ip)).to(dev)
        self.view = dpcs.view_of(sc)
        self.params = dpcs.make_params(sc.params)

    def render(self, spp=None, bounces=None, seed=None, Ip=None, albedo=None, rough=None, params=None):
        torch = need_cuda()
        sc = self.sc
        Ec = torch.empty((sc.Hc, sc.Wc, 3), dtype=torch.float32, device=self.ctx.device)
        Ic, _ = self.ctx.render(self.handle, self.albedo if albedo is None else albedo,
                                self.rough if rough is None else rough, self.Ip if Ip is None else Ip, self.view,
                                self.params if params is None else params, spp or sc.spp,
                                sc.bounces if bounces is None else bounces, sc.seed if seed is None else seed, Ec=Ec)
        self.ctx.sync()
        return Ec, Ic

    def backward(self, Ec, Ic, dIc, spp=None, bounces=None):
        torch = need_cuda()
        sc = self.sc
        dev = self.ctx.device
        g = {"dIp": torch.zeros_like(self.Ip), "dalbedo": torch.zeros_like(self.albedo),
             "drough": torch.zeros_like(self.rough), "dparams": torch.zeros(11, dtype=torch.float32, device=dev)}
        self.ctx.render_backward(self.handle, self.albedo, self.rough, self.Ip, self.view, self.params,
                                 spp or sc.spp, sc.bounces if bounces is None else bounces, sc.seed, Ec, Ic, dIc,
                                 g["dIp"], g["dalbedo"], g["drough"], g["dparams"])
        self.ctx.sync()
        return {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}

    def close(self):
        self.ctx.free(self.handle)


def crf_atol(sc, Ec_ref, atol_E=1e-7):
    """Absolute tolerance of Ic implied by an absolute tolerance atol_E on Ec:
    |dIc/dEc| * atol_E with Ic = (Gc w Ec)^gamma_c (Eq. 5)."""
    p = sc.params
    E = np.asarray(Ec_ref, np.float64).reshape(-1, 3)
    g = np.asarray(p.gamma_c, np.float64)[None, :]
    a = p.gain_c * np.asarray(p.wb, np.float64)[None, :] * E
    with np.errstate(divide="ignore", invalid="ignore"):
        d = np.where(a > 0, g * np.power(np.maximum(a, 1e-300), g - 1) * p.gain_c * np.asarray(p.wb)[None, :], 0.0)
    return d * atol_E + 1e-12


def pixel_parity(gpu, ref, rtol=1e-4, atol=1e-7, frac=0.999, mean_rtol=1e-5):
    """North-star image gate: |g - r| <= rtol |r| + atol per channel on at
    least `frac` of the pixels (edge flips between FP32 and FP64 paths take
    the rest), and the image mean within mean_rtol.  ``atol`` may be an array
    of per-element tolerances."""
    gpu = np.asarray(gpu, np.float64).reshape(-1, 3)
    ref = np.asarray(ref, np.float64).reshape(-1, 3)
    atol = np.broadcast_to(np.asarray(atol, np.float64).reshape(-1, 3) if np.ndim(atol) else atol, ref.shape)
    ok = np.all(np.abs(gpu - ref) <= rtol * np.abs(ref) + atol, axis=1)
    n_bad = int((~ok).sum())
    allowed = int(np.floor((1.0 - frac) * len(ok)))
    m_g, m_r = gpu.mean(), ref.mean()
    mean_ok = abs(m_g - m_r) <= mean_rtol * abs(m_r) + 1e-12
    return n_bad <= allowed and mean_ok, {"bad_pixels": n_bad, "allowed": allowed, "n": len(ok),
                                          "mean_gpu": m_g, "mean_ref": m_r,
                                          "max_rel": float(np.max(np.abs(gpu - ref) / (np.abs(ref) + 1e-7))),
                                          "worst": [(int(i), gpu[i].tolist(), ref[i].tolist())
                                                    for i in np.argsort(-np.max(np.abs(gpu - ref) / (
                                                        np.abs(ref) + atol + 1e-30), axis=1))[:3]]}
