// denoise.cu -- the differentiable denoiser of Eq. 11, Ic' = D(Ic), as a
// cross-bilateral filter guided by noise-free first-hit features.
//
//   guide g(p): albedo (3), normal towards the camera (3), hit distance, hit
//               flag of the ray through pixel centre p (k_gbuffer);
//   D(I)(p)   = sum_q w(p,q) I(q) / W(p),   W(p) = sum_q w(p,q);
//   w(p,q)    = exp(-|p-q|^2 ks - |da|^2 ka - |dn|^2 kn - dt^2 kd),
//               k = 1 / (2 sigma^2), or 0 for a feature that is switched off,
//               q over the (2r+1)^2 window around p inside the image.
//
// The weights depend on the guide only, so D is linear in I and, because
// w(p,q) = w(q,p) over a symmetric window, its adjoint is the same gather
// applied to dD / W without the normalisation:
//   dI(q) = sum_p w(q,p) (dD(p) / W(p)).
// Both directions run one kernel: a 16 x 16 output tile per CTA with its
// (16 + 2r)^2 halo of guide and image staged in shared memory, so each input
// is read from HBM once per tile instead of (2r+1)^2 times; each thread
// computes a vertical strip of outputs that share the taps they load.
#include <cuda_runtime.h>
#include <stdint.h>

#include "device.cuh"
#include "internal.h"

#ifndef DPCS_DENOISE_STRIP
#define DPCS_DENOISE_STRIP 1  // 0: one output per thread (k_bilateral)
#endif

namespace dpcs {

namespace {

constexpr int kTile = 16;
constexpr int kMaxRadius = 8;  // (16 + 16)^2 pixels x 48 B = 48 KiB of shared memory

// First-hit guide through each camera pixel centre (a.jitter must be 0).
__global__ void k_gbuffer(const RenderArgs a, float4 *__restrict__ guide) {
    const int64_t pix = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (pix >= (int64_t)a.Hc * a.Wc) return;
    f3 o, d;
    camera_ray(a, (uint32_t)pix, 0u, o, d);
    const Ray ray = make_ray(o, d);
    Hit h;
    Cnt cnt;
    float4 g0 = make_float4(0.f, 0.f, 0.f, 0.f), g1 = g0;
    if (traverse(a.nodes, a.tris, a.root, a.T, ray, INFINITY, false, h, a.status, cnt)) {
        const Surf S = surface_at(a, h, ray.d);
        g0 = make_float4(S.rho.x, S.rho.y, S.rho.z, S.n.x);
        g1 = make_float4(S.n.y, S.n.z, h.t, 1.0f);
    }
    guide[2 * pix] = g0;
    guide[2 * pix + 1] = g1;
}

struct Widths {
    float ks, ka, kn, kd;  // 1 / (2 sigma^2) per term; 0 = term off
};

// kAdjoint = false: out = D(img), wsum = W (wsum may be null).
// kAdjoint = true : out += D^T(img), where img is dD and wsum the forward W.
template <bool kAdjoint>
__global__ void __launch_bounds__(kTile *kTile)
    k_bilateral(const float *__restrict__ img, const float4 *__restrict__ guide, const float *__restrict__ wsum_in,
                int H, int W, int r, Widths k, float *__restrict__ out, float *__restrict__ wsum_out) {
    extern __shared__ float4 smem[];
    const int S = kTile + 2 * r;
    float4 *sg0 = smem, *sg1 = smem + S * S, *si = smem + 2 * S * S;
    const int tid = threadIdx.y * kTile + threadIdx.x;
    const int y0 = blockIdx.y * kTile - r, x0 = blockIdx.x * kTile - r;
    for (int i = tid; i < S * S; i += kTile * kTile) {
        const int gy = y0 + i / S, gx = x0 + i % S;
        if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
            const int64_t p = (int64_t)gy * W + gx;
            sg0[i] = __ldg(guide + 2 * p);
            float4 g1 = __ldg(guide + 2 * p + 1);
            g1.w = 0.0f;  // inside the image
            sg1[i] = g1;
            float s = 1.0f;
            if (kAdjoint) s = 1.0f / __ldg(wsum_in + p);
            si[i] = make_float4(__ldg(img + 3 * p) * s, __ldg(img + 3 * p + 1) * s, __ldg(img + 3 * p + 2) * s, 0.0f);
        } else {
            sg1[i] = make_float4(0.f, 0.f, 0.f, -1.0f);  // outside: skipped
        }
    }
    __syncthreads();
    const int py = blockIdx.y * kTile + threadIdx.y, px = blockIdx.x * kTile + threadIdx.x;
    if (py >= H || px >= W) return;
    const int c = (threadIdx.y + r) * S + threadIdx.x + r;
    const float4 c0 = sg0[c], c1 = sg1[c];
    float ax = 0.f, ay = 0.f, az = 0.f, den = 0.f;
    for (int dy = -r; dy <= r; ++dy) {
        const int row = c + dy * S;
        for (int dx = -r; dx <= r; ++dx) {
            const int q = row + dx;
            const float4 q1 = sg1[q];
            if (q1.w < 0.0f) continue;
            const float4 q0 = sg0[q];
            const float da = (c0.x - q0.x) * (c0.x - q0.x) + (c0.y - q0.y) * (c0.y - q0.y) +
                             (c0.z - q0.z) * (c0.z - q0.z);
            const float dn = (c0.w - q0.w) * (c0.w - q0.w) + (c1.x - q1.x) * (c1.x - q1.x) +
                             (c1.y - q1.y) * (c1.y - q1.y);
            const float dt = (c1.z - q1.z) * (c1.z - q1.z);
            const float e = (float)(dx * dx + dy * dy) * k.ks + da * k.ka + dn * k.kn + dt * k.kd;
            const float w = expf(-e);
            const float4 v = si[q];
            ax += w * v.x;
            ay += w * v.y;
            az += w * v.z;
            den += w;
        }
    }
    const int64_t p = (int64_t)py * W + px;
    if (kAdjoint) {
        out[3 * p] += ax;
        out[3 * p + 1] += ay;
        out[3 * p + 2] += az;
    } else {
        const float inv = 1.0f / den;
        out[3 * p] = ax * inv;
        out[3 * p + 1] = ay * inv;
        out[3 * p + 2] = az * inv;
        if (wsum_out) wsum_out[p] = den;
    }
}

// The same filter with kStrip vertically stacked outputs per thread: each
// tap loaded from shared memory serves every output of the strip whose
// window contains it, so a thread issues (2r + kStrip) (2r + 1) tap loads
// for kStrip outputs instead of kStrip (2r + 1)^2.  Each output still sums
// its taps in the same order (rows, then columns), so the result is the one
// k_bilateral computes.
#ifndef DPCS_DENOISE_KSTRIP
#define DPCS_DENOISE_KSTRIP 2  // measured: 2 is 9-15 % faster than 1 output per thread, 4 is 15-40 % slower
#endif
constexpr int kStrip = DPCS_DENOISE_KSTRIP;

template <bool kAdjoint>
__global__ void __launch_bounds__(kTile *kTile / kStrip)
    k_bilateral_strip(const float *__restrict__ img, const float4 *__restrict__ guide,
                      const float *__restrict__ wsum_in, int H, int W, int r, Widths k, float *__restrict__ out,
                      float *__restrict__ wsum_out) {
    extern __shared__ float4 smem[];
    const int S = kTile + 2 * r;
    float4 *sg0 = smem, *sg1 = smem + S * S, *si = smem + 2 * S * S;
    constexpr int kThreads = kTile * kTile / kStrip;
    const int tid = threadIdx.y * kTile + threadIdx.x;
    const int y0 = blockIdx.y * kTile - r, x0 = blockIdx.x * kTile - r;
    for (int i = tid; i < S * S; i += kThreads) {
        const int gy = y0 + i / S, gx = x0 + i % S;
        if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
            const int64_t p = (int64_t)gy * W + gx;
            sg0[i] = __ldg(guide + 2 * p);
            float4 g1 = __ldg(guide + 2 * p + 1);
            g1.w = 0.0f;  // inside the image
            sg1[i] = g1;
            float s = 1.0f;
            if (kAdjoint) s = 1.0f / __ldg(wsum_in + p);
            si[i] = make_float4(__ldg(img + 3 * p) * s, __ldg(img + 3 * p + 1) * s, __ldg(img + 3 * p + 2) * s, 0.0f);
        } else {
            sg1[i] = make_float4(0.f, 0.f, 0.f, -1.0f);  // outside: skipped
        }
    }
    __syncthreads();
    const int px = blockIdx.x * kTile + threadIdx.x;
    if (px >= W) return;
    const int ry = threadIdx.y * kStrip;  // the strip's first output row in the tile
    float4 c0[kStrip], c1[kStrip];
    float ax[kStrip], ay[kStrip], az[kStrip], den[kStrip];
#pragma unroll
    for (int o = 0; o < kStrip; ++o) {
        const int c = (ry + o + r) * S + threadIdx.x + r;
        c0[o] = sg0[c];
        c1[o] = sg1[c];
        ax[o] = ay[o] = az[o] = den[o] = 0.f;
    }
    for (int j = -r; j < r + kStrip; ++j) {  // window rows, relative to the first output
        const int row = (ry + j + r) * S + threadIdx.x + r;
        for (int dx = -r; dx <= r; ++dx) {
            const int q = row + dx;
            const float4 q1 = sg1[q];
            if (q1.w < 0.0f) continue;
            const float4 q0 = sg0[q];
            const float4 v = si[q];
#pragma unroll
            for (int o = 0; o < kStrip; ++o) {
                const int dy = j - o;
                if (dy < -r || dy > r) continue;
                const float da = (c0[o].x - q0.x) * (c0[o].x - q0.x) + (c0[o].y - q0.y) * (c0[o].y - q0.y) +
                                 (c0[o].z - q0.z) * (c0[o].z - q0.z);
                const float dn = (c0[o].w - q0.w) * (c0[o].w - q0.w) + (c1[o].x - q1.x) * (c1[o].x - q1.x) +
                                 (c1[o].y - q1.y) * (c1[o].y - q1.y);
                const float dt = (c1[o].z - q1.z) * (c1[o].z - q1.z);
                const float e = (float)(dx * dx + dy * dy) * k.ks + da * k.ka + dn * k.kn + dt * k.kd;
                const float w = expf(-e);
                ax[o] += w * v.x;
                ay[o] += w * v.y;
                az[o] += w * v.z;
                den[o] += w;
            }
        }
    }
#pragma unroll
    for (int o = 0; o < kStrip; ++o) {
        const int py = blockIdx.y * kTile + ry + o;
        if (py >= H) break;
        const int64_t p = (int64_t)py * W + px;
        if (kAdjoint) {
            out[3 * p] += ax[o];
            out[3 * p + 1] += ay[o];
            out[3 * p + 2] += az[o];
        } else {
            const float inv = 1.0f / den[o];
            out[3 * p] = ax[o] * inv;
            out[3 * p + 1] = ay[o] * inv;
            out[3 * p + 2] = az[o] * inv;
            if (wsum_out) wsum_out[p] = den[o];
        }
    }
}

}  // namespace

}  // namespace dpcs

using namespace dpcs;

namespace {

dpcs_status check_denoise_args(dpcs_ctx *c, const float *img, const float *guide, int32_t Hc, int32_t Wc,
                               const dpcs_denoise_params *prm, const float *out, Widths &k) {
    if (!img || !guide || !out || !prm || Hc <= 0 || Wc <= 0)
        return ctx_fail(c, DPCS_ERR_INVALID_ARG, "denoise: null pointer or empty image");
    if (((uintptr_t)guide & 15u) != 0)
        return ctx_fail(c, DPCS_ERR_INVALID_ARG, "denoise: guide must be 16-byte aligned");
    if (prm->radius < 0 || prm->radius > kMaxRadius || !(prm->sigma_s > 0.0f))
        return ctx_fail(c, DPCS_ERR_INVALID_ARG, "denoise: radius must be in [0, 8] and sigma_s > 0");
    auto inv2 = [](float s) { return s > 0.0f ? 0.5f / (s * s) : 0.0f; };
    k.ks = inv2(prm->sigma_s);
    k.ka = inv2(prm->sigma_albedo);
    k.kn = inv2(prm->sigma_normal);
    k.kd = inv2(prm->sigma_depth);
    return cudaSetDevice(ctx_device(c)) == cudaSuccess ? DPCS_OK
                                                        : ctx_fail(c, DPCS_ERR_CUDA, "denoise: cudaSetDevice");
}

template <bool kAdjoint>
dpcs_status launch_bilateral(dpcs_ctx *c, const float *img, const float *guide, const float *wsum_in, int32_t Hc,
                             int32_t Wc, int r, const Widths &k, float *out, float *wsum_out, cudaStream_t st) {
    const int S = kTile + 2 * r;
    const size_t shm = (size_t)3 * S * S * sizeof(float4);
    const dim3 grid((Wc + kTile - 1) / kTile, (Hc + kTile - 1) / kTile);
#if DPCS_DENOISE_STRIP
    k_bilateral_strip<kAdjoint><<<grid, dim3(kTile, kTile / kStrip), shm, st>>>(img, (const float4 *)guide, wsum_in, Hc,
                                                                            Wc, r, k, out, wsum_out);
#else
    k_bilateral<kAdjoint><<<grid, dim3(kTile, kTile), shm, st>>>(img, (const float4 *)guide, wsum_in, Hc, Wc, r, k,
                                                                out, wsum_out);
#endif
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ctx_fail(c, DPCS_ERR_CUDA, cudaGetErrorString(e));
    ctx_add_launches(c, 1);
    return DPCS_OK;
}

}  // namespace

extern "C" {

dpcs_status dpcs_gbuffer(dpcs_ctx *c, dpcs_scene scene, const float *albedo, const float *rough, int32_t Ht,
                         int32_t Wt, const dpcs_view *view, float *guide, void *stream) {
    if (!c) return DPCS_ERR_INVALID_ARG;
    if (!guide || ((uintptr_t)guide & 15u) != 0)
        return ctx_fail(c, DPCS_ERR_INVALID_ARG, "gbuffer: guide must be a 16-byte aligned device pointer");
    dpcs_params prm{};
    prm.gamma_p[0] = prm.gamma_p[1] = prm.gamma_p[2] = 1.0f;
    prm.gamma_c[0] = prm.gamma_c[1] = prm.gamma_c[2] = 1.0f;
    prm.wb[0] = prm.wb[1] = prm.wb[2] = 1.0f;
    prm.gain_p = prm.gain_c = prm.k_proj = 1.0f;
    prm.rr_q = 1.0f;
    RenderArgs a;
    dpcs_status s = ctx_render_args(c, scene, albedo, rough, Ht, Wt, albedo, view, &prm, 1, 1, 0, a);
    if (s) return s;
    if (cudaSetDevice(ctx_device(c)) != cudaSuccess) return ctx_fail(c, DPCS_ERR_CUDA, "gbuffer: cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nt = (int64_t)Ht * Wt, npix = (int64_t)view->Hc * view->Wc;
    float4 *tex = nullptr;  // the packed texture, only for this call
    cudaError_t e = cudaMallocAsync((void **)&tex, (size_t)nt * 16, st);
    if (e != cudaSuccess) return ctx_fail(c, DPCS_ERR_OOM, "gbuffer: texture allocation failed");
    int nl = launch_pack_tex(albedo, rough, nt, tex, st);
    a.tex = tex;
    a.jitter = 0;  // rays through pixel centres
    a.counters = nullptr;
    k_gbuffer<<<(unsigned)((npix + 127) / 128), 128, 0, st>>>(a, (float4 *)guide);
    e = cudaGetLastError();
    cudaFreeAsync(tex, st);
    if (nl < 0 || e != cudaSuccess) return ctx_fail(c, DPCS_ERR_CUDA, "gbuffer: launch failed");
    ctx_add_launches(c, nl + 1);
    return DPCS_OK;
}

dpcs_status dpcs_denoise(dpcs_ctx *c, const float *Ic, const float *guide, int32_t Hc, int32_t Wc,
                         const dpcs_denoise_params *prm, float *out, float *wsum, void *stream) {
    if (!c) return DPCS_ERR_INVALID_ARG;
    Widths k;
    dpcs_status s = check_denoise_args(c, Ic, guide, Hc, Wc, prm, out, k);
    if (s) return s;
    if (out == Ic) return ctx_fail(c, DPCS_ERR_INVALID_ARG, "denoise: out must not alias the input");
    return launch_bilateral<false>(c, Ic, guide, nullptr, Hc, Wc, prm->radius, k, out, wsum, (cudaStream_t)stream);
}

dpcs_status dpcs_denoise_backward(dpcs_ctx *c, const float *dOut, const float *guide, const float *wsum, int32_t Hc,
                                  int32_t Wc, const dpcs_denoise_params *prm, float *dIc, void *stream) {
    if (!c) return DPCS_ERR_INVALID_ARG;
    Widths k;
    dpcs_status s = check_denoise_args(c, dOut, guide, Hc, Wc, prm, dIc, k);
    if (s) return s;
    if (!wsum) return ctx_fail(c, DPCS_ERR_INVALID_ARG, "denoise_backward: wsum from dpcs_denoise is required");
    if (dIc == dOut) return ctx_fail(c, DPCS_ERR_INVALID_ARG, "denoise_backward: dIc must not alias dOut");
    return launch_bilateral<true>(c, dOut, guide, wsum, Hc, Wc, prm->radius, k, dIc, nullptr, (cudaStream_t)stream);
}

}  // extern "C"
