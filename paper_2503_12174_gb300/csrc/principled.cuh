// principled.cuh -- device-side pieces of the principled material of
// Sec. 3.2 (metallic map m, normal map Vn) shared by its render and adjoint
// kernels (principled.cu) and the camera-pose adjoint (pose.cu): the GGX
// lobe at the shading normal with its derivatives, Schlick's Fresnel with
// F0_j = (1 - m) f0 + m rho_j, the surface interaction with the tangent
// frame and the normal map, next-event estimation to the projector, and the
// continuation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "device.cuh"
#include "internal.h"

namespace dpcs {

// GGX lobe of the principled BRDF at shading normal n, with its partial
// derivatives in roughness and in n (wo, wi and h held fixed):
//   d ln S / dn = (d ln D / d ch) h + (d ln G1(co) / d co - 1/co) wo
//               + (d ln G1(ci) / d ci - 1/ci) wi.
struct PLobe {
    float on;   // 1 when wo and wi are both above the shading hemisphere, else 0 (the whole BRDF is 0)
    float S;    // ks D G / (4 ci co)
    float dSr;  // dS / d roughness
    float s5;   // (1 - wo.h)^5 of Schlick's Fresnel
    f3 dSn;     // dS / dn
};
__device__ __forceinline__ void plobe(f3 n, f3 wo, f3 wi, float r, float ks, PLobe &L) {
    L.on = L.S = L.dSr = L.s5 = 0.0f;
    L.dSn = mk3(0.f, 0.f, 0.f);
    const float co = dot(n, wo), ci = dot(n, wi);
    if (co <= 0.0f || ci <= 0.0f) return;
    L.on = 1.0f;
    if (ks <= 0.0f) return;
    float dadr;
    const float a = alpha_of(r, dadr);
    const f3 h = normalize(wo + wi);
    const float ch = dot(n, h), a2 = a * a;
    const float t = sin2(n, h) + a2 * ch * ch;
    const float D = a2 / (DPCS_PI_F * t * t);
    const float si = sqrtf(a2 + (1.0f - a2) * ci * ci), so = sqrtf(a2 + (1.0f - a2) * co * co);
    const float G = (2.0f * ci / (ci + si)) * (2.0f * co / (co + so));
    const float S = ks * D * G / (4.0f * ci * co);
    const float dlnD = 2.0f / a - 4.0f * a * ch * ch / t;
    const float dlnG = -(a * (1.0f - ci * ci) / si) / (ci + si) - (a * (1.0f - co * co) / so) / (co + so);
    L.S = S;
    L.dSr = S * (dlnD + dlnG) * dadr;
    const float kh = -4.0f * ch * (a2 - 1.0f) / t;
    const float ko = -(1.0f + (1.0f - a2) * co / so) / (co + so);
    const float ki = -(1.0f + (1.0f - a2) * ci / si) / (ci + si);
    L.dSn = (h * kh + wo * ko + wi * ki) * S;
    const float m = fmaxf(0.0f, 1.0f - dot(wo, h));
    const float m2 = m * m;
    L.s5 = m2 * m2 * m;
}

// Schlick F_j for F0_j = (1 - m) f0 + m rho_j
__device__ __forceinline__ float pfresnel(float rho, float m, float f0, float s5) {
    const float F0 = (1.0f - m) * f0 + m * rho;
    return F0 + (1.0f - F0) * s5;
}

// f per channel from a lobe
__device__ __forceinline__ f3 pbrdf(f3 rho, float m, float f0, const PLobe &L) {
    const float kd = L.on * (1.0f - m) * DPCS_INV_PI_F;
    return mk3(kd * rho.x + L.S * pfresnel(rho.x, m, f0, L.s5), kd * rho.y + L.S * pfresnel(rho.y, m, f0, L.s5),
               kd * rho.z + L.S * pfresnel(rho.z, m, f0, L.s5));
}

// surface interaction with the principled maps
struct PSurf {
    f3 x, n, ns, wo, rho;  // n: geometric normal turned towards the incoming ray
    float rough, m;
    f3 T, B;               // tangent frame of the normal map
    float inv_ulen;        // 1 / |v| of the decoded normal-map vector (0: unperturbed)
    Bilin tb;
};
__device__ __forceinline__ PSurf psurface_at(const RenderArgs &a, const float4 *__restrict__ mat, const Hit &h, f3 d) {
    PSurf S;
    const float4 A = __ldg(a.tris + 3 * h.pos + 0);
    const float4 V1 = __ldg(a.tris + 3 * h.pos + 1);
    const float4 V2 = __ldg(a.tris + 3 * h.pos + 2);
    const f3 e1 = xyz(V1) - xyz(A), e2 = xyz(V2) - xyz(A);
    S.x = xyz(A) + e1 * h.u + e2 * h.v;
    S.n = normalize(cross(e1, e2));
    if (dot(S.n, d) > 0.0f) S.n = S.n * -1.0f;
    const float2 t0 = __ldg(a.tuv + 3 * h.pos + 0), t1 = __ldg(a.tuv + 3 * h.pos + 1),
                 t2 = __ldg(a.tuv + 3 * h.pos + 2);
    const float w0 = 1.0f - h.u - h.v;
    const float su = w0 * t0.x + h.u * t1.x + h.v * t2.x;
    const float sv = w0 * t0.y + h.u * t1.y + h.v * t2.y;
    S.tb = bilin_setup(su * (float)a.Wt, sv * (float)a.Ht, a.Wt, a.Ht);
    const float4 tex = bilin_fetch(a.tex, S.tb, a.Wt, a.Ht);
    const float4 mt = bilin_fetch(mat, S.tb, a.Wt, a.Ht);
    S.rho = mk3(tex.x, tex.y, tex.z);
    S.rough = tex.w;
    S.m = mt.x;
    S.wo = d * -1.0f;
    // tangent: dp/du from e1 = dp/du du1 + dp/dv dv1 and e2 likewise
    const float du1 = t1.x - t0.x, dv1 = t1.y - t0.y, du2 = t2.x - t0.x, dv2 = t2.y - t0.y;
    const float det = du1 * dv2 - du2 * dv1;
    bool ok = false;
    if (det != 0.0f) {
        const f3 dpdu = (e1 * dv2 - e2 * dv1) * (1.0f / det);
        const f3 t = dpdu - S.n * dot(S.n, dpdu);
        const float l2 = dot(t, t);
        if (l2 > 1e-12f * dot(dpdu, dpdu)) {
            S.T = t * rsqrtf(l2);
            ok = true;
        }
    }
    if (!ok) {
        f3 b;
        onb(S.n, S.T, b);
    }
    S.B = cross(S.n, S.T);
    const f3 u = S.T * (2.0f * mt.y - 1.0f) + S.B * (2.0f * mt.z - 1.0f) + S.n * (2.0f * mt.w - 1.0f);
    const float ul2 = dot(u, u);
    if (ul2 > 1e-24f) {
        S.inv_ulen = rsqrtf(ul2);
        S.ns = u * S.inv_ulen;
    } else {
        S.inv_ulen = 0.0f;
        S.ns = S.n;
    }
    return S;
}

// next-event estimation to the projector with the principled material
struct PNee {
    f3 so, sdir;
    float smax;
    Bilin pb;
    float4 ep;
    float G;
    PLobe L;
    f3 fp, wp_cs;
};
__device__ __forceinline__ bool pnee_prepare(const RenderArgs &a, const PSurf &S, PNee &N) {
    const f3 cp = mk3(a.cp[0], a.cp[1], a.cp[2]);
    const f3 X = mat3v(a.Rp, S.x) + mk3(a.tp[0], a.tp[1], a.tp[2]);
    const f3 q = mat3v(a.Kp, X);
    if (!(q.z > 0.0f && X.z > 0.0f)) return false;
    const float up = q.x / q.z, vp = q.y / q.z;
    if (!(up >= 0.0f && up < (float)a.Wp && vp >= 0.0f && vp < (float)a.Hp)) return false;
    const f3 v = cp - S.x;
    const float r2 = dot(v, v), dist = sqrtf(r2);
    const f3 wp = v * (1.0f / dist);
    const float cs = dot(S.ns, wp);
    if (!(cs > 0.0f && dot(S.n, wp) > 0.0f)) return false;
    const float cpz = X.z / sqrtf(dot(X, X));
    N.so = S.x + S.n * kRayEps;
    const f3 sv = cp - N.so;
    const float sd = sqrtf(dot(sv, sv));
    N.sdir = sv * (1.0f / sd);
    N.smax = sd - kRayEps;
    N.pb = bilin_setup(up, vp, a.Wp, a.Hp);
    N.ep = bilin_fetch(a.Ep, N.pb, a.Wp, a.Hp);
    N.G = a.k_proj * cpz * cs / r2;
    plobe(S.ns, S.wo, wp, S.rough, a.ks, N.L);
    N.fp = pbrdf(S.rho, S.m, a.f0, N.L);
    N.wp_cs = wp * (1.0f / cs);
    return true;
}

// continuation: BRDF sampling around ns, throughput, Russian roulette
struct PCont {
    f3 wi, w, wi_ci;
    float cw;
    PLobe L;
};
__device__ __forceinline__ bool pcontinue_prepare(const RenderArgs &a, uint32_t pix, uint32_t s, int b,
                                                  const PSurf &S, PCont &C) {
    float u[4];
    rand4(a.key0, a.key1, pix, s, (uint32_t)b, u);
    if (!bsdf_sample(S.ns, S.wo, S.rough, a.ks, u[0], u[1], u[2], C.wi)) return false;
    if (!(dot(S.n, C.wi) > 0.0f)) return false;  // below the geometric surface
    const float pdf = bsdf_pdf(S.ns, S.wo, C.wi, S.rough, a.ks);
    if (!(pdf > 0.0f)) return false;
    float qrr = 1.0f;
    if (a.rr_start > 0 && b >= a.rr_start) {
        if (u[3] >= a.rr_q) return false;
        qrr = a.rr_q;
    }
    plobe(S.ns, S.wo, C.wi, S.rough, a.ks, C.L);
    const float ci = dot(S.ns, C.wi);
    C.cw = ci / (pdf * qrr);
    C.wi_ci = C.wi * (1.0f / ci);
    C.w = pbrdf(S.rho, S.m, a.f0, C.L) * C.cw;
    return true;
}

}  // namespace dpcs
