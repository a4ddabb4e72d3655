// device.cuh -- device-side building blocks of the DPCS path tracer (sm_103a):
// Philox4x32-10, FP32 vector algebra, the Lambert+GGX BRDF, bilinear lookups,
// BVH traversal and the per-sample path (forward and replay record).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "internal.h"

namespace dpcs {

#define DPCS_PI_F 3.14159265358979323846f
#define DPCS_INV_PI_F 0.318309886183790671538f
constexpr float kRayEps = 1e-4f;   // origin offset along the shading normal
constexpr int kStack = 64;         // traversal stack depth

// Work counters of the DPCS_COUNTERS build (node visits, triangle tests,
// closest rays, shadow rays, vertices, lit NEE, continuations, paths, and
// two SIMT-efficiency counts: warp iterations of the traversal loop and of
// the one-ray-per-iteration path loop, each counted once per warp); in the
// normal build every increment compiles away.
enum { kCntNode = 0, kCntTri, kCntRay, kCntShadow, kCntVert, kCntLit, kCntCont, kCntPath, kCntTravWarpIter,
       kCntPathWarpIter, kCntN };
struct Cnt {
#ifdef DPCS_COUNTERS
    uint32_t v[kCntN];
    __device__ Cnt() {
        for (int i = 0; i < kCntN; ++i) v[i] = 0u;
    }
    __device__ __forceinline__ void add(int i, uint32_t k = 1u) { v[i] += k; }
    // once per warp: the lowest active lane counts
    __device__ __forceinline__ void add_warp(int i) {
        if ((int)(threadIdx.x & 31) == __ffs(__activemask()) - 1) v[i] += 1u;
    }
    __device__ __forceinline__ void flush(unsigned long long *out) {
        if (!out) return;
        for (int i = 0; i < kCntN; ++i) {
            unsigned long long x = v[i];
            for (int off = 16; off; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
            if ((threadIdx.x & 31) == 0 && x) atomicAdd(out + i, x);
        }
    }
#else
    __device__ __forceinline__ void add(int, uint32_t = 1u) {}
    __device__ __forceinline__ void add_warp(int) {}
    __device__ __forceinline__ void flush(unsigned long long *) {}
#endif
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 products
// with the key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4(uint32_t &c0, uint32_t &c1, uint32_t &c2, uint32_t &c3, uint32_t k0,
                                        uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
}

// four uniforms in [0,1) with 24 bits, exact in FP32, for counter (pix, s, b, 0)
__device__ __forceinline__ void rand4(uint32_t k0, uint32_t k1, uint32_t pix, uint32_t s, uint32_t b, float u[4]) {
    uint32_t c0 = pix, c1 = s, c2 = b, c3 = 0u;
    philox4(c0, c1, c2, c3, k0, k1);
    const float sc = 5.9604644775390625e-08f;  // 2^-24
    u[0] = (float)(c0 >> 8) * sc;
    u[1] = (float)(c1 >> 8) * sc;
    u[2] = (float)(c2 >> 8) * sc;
    u[3] = (float)(c3 >> 8) * sc;
}

// ---------------------------------------------------------------------------
// FP32 vectors
// ---------------------------------------------------------------------------
struct f3 {
    float x, y, z;
};
__device__ __forceinline__ f3 mk3(float x, float y, float z) { return f3{x, y, z}; }
__device__ __forceinline__ f3 operator+(f3 a, f3 b) { return mk3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ f3 operator-(f3 a, f3 b) { return mk3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ f3 operator*(f3 a, float s) { return mk3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ f3 operator*(f3 a, f3 b) { return mk3(a.x * b.x, a.y * b.y, a.z * b.z); }
__device__ __forceinline__ float dot(f3 a, f3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ f3 cross(f3 a, f3 b) {
    return mk3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ f3 normalize(f3 a) { return a * (1.0f / sqrtf(dot(a, a))); }
__device__ __forceinline__ f3 xyz(float4 v) { return mk3(v.x, v.y, v.z); }
__device__ __forceinline__ f3 mat3v(const float *M, f3 v) {
    return mk3(M[0] * v.x + M[1] * v.y + M[2] * v.z, M[3] * v.x + M[4] * v.y + M[5] * v.z,
               M[6] * v.x + M[7] * v.y + M[8] * v.z);
}

// ---------------------------------------------------------------------------
// Lambert + GGX BRDF (alpha = rough^2, rough clamped to [0.01, 1]),
// separable Smith masking, Schlick Fresnel.  spec terms include ks.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float alpha_of(float r, float &dadr) {
    float rc = r, d = 2.0f * r;
    if (rc < 0.01f) { rc = 0.01f; d = 0.0f; }
    if (rc > 1.0f) { rc = 1.0f; d = 0.0f; }
    dadr = d;
    return rc * rc;
}

// GGX D for cos(theta_h) = ch and sin^2(theta_h) = s2.  The denominator
// cos^2 (a^2 - 1) + 1 is formed as s2 + a^2 cos^2 with s2 = |n x h|^2: the
// textbook form cancels catastrophically in FP32 near the peak of sharp lobes.
__device__ __forceinline__ float ggx_D(float ch, float s2, float a) {
    const float a2 = a * a;
    const float t = s2 + a2 * ch * ch;
    return a2 / (DPCS_PI_F * t * t);
}
__device__ __forceinline__ float sin2(f3 n, f3 h) {
    const f3 c = cross(n, h);
    return dot(c, c);
}

__device__ __forceinline__ float ggx_G1(float c, float a) {
    const float a2 = a * a;
    return 2.0f * c / (c + sqrtf(a2 + (1.0f - a2) * c * c));
}

// ks * D G F / (4 ci co) and its derivative in roughness r (0 if ks == 0)
__device__ __forceinline__ float spec_eval(f3 n, f3 wo, f3 wi, float r, float ks, float f0, float &dspec_dr) {
    dspec_dr = 0.0f;
    const float co = dot(n, wo), ci = dot(n, wi);
    if (ks <= 0.0f || co <= 0.0f || ci <= 0.0f) return 0.0f;
    float dadr;
    const float a = alpha_of(r, dadr);
    const f3 h = normalize(wo + wi);
    const float ch = dot(n, h);
    const float a2 = a * a;
    const float t = sin2(n, h) + a2 * ch * ch;
    const float D = a2 / (DPCS_PI_F * t * t);
    const float si = sqrtf(a2 + (1.0f - a2) * ci * ci), so = sqrtf(a2 + (1.0f - a2) * co * co);
    const float G = (2.0f * ci / (ci + si)) * (2.0f * co / (co + so));
    float m = fmaxf(0.0f, 1.0f - dot(wo, h));
    const float m2 = m * m;
    const float F = f0 + (1.0f - f0) * (m2 * m2 * m);
    const float spec = ks * D * G * F / (4.0f * ci * co);
    const float dlnD = 2.0f / a - 4.0f * a * ch * ch / t;
    const float dlnG = -(a * (1.0f - ci * ci) / si) / (ci + si) - (a * (1.0f - co * co) / so) / (co + so);
    dspec_dr = spec * (dlnD + dlnG) * dadr;
    return spec;
}

// orthonormal basis around n (Duff et al., JCGT 2017) with its seam at
// n.z = -1/pi, away from the n.z = 0 of axis-aligned and symmetric facets
// whose sign FP32 rounding could otherwise flip
__device__ __forceinline__ void onb(f3 n, f3 &t, f3 &b) {
    const float sg = n.z >= -DPCS_INV_PI_F ? 1.0f : -1.0f;
    const float a = -1.0f / (sg + n.z);
    const float bb = n.x * n.y * a;
    t = mk3(1.0f + sg * n.x * n.x * a, sg * bb, -sg * n.x);
    b = mk3(bb, sg + n.y * n.y * a, -n.y);
}

__device__ __forceinline__ float spec_prob(float ks) { return ks > 0.0f ? 0.5f : 0.0f; }

__device__ __forceinline__ float bsdf_pdf(f3 n, f3 wo, f3 wi, float r, float ks) {
    const float ci = dot(n, wi), co = dot(n, wo);
    if (ci <= 0.0f || co <= 0.0f) return 0.0f;
    const float ps = spec_prob(ks);
    float p = (1.0f - ps) * ci * DPCS_INV_PI_F;
    if (ps > 0.0f) {
        float dadr;
        const float a = alpha_of(r, dadr);
        const f3 h = normalize(wo + wi);
        p += ps * ggx_G1(co, a) * ggx_D(dot(n, h), sin2(n, h), a) / (4.0f * co);
    }
    return p;
}

// u0 picks the lobe, (u1, u2) the direction: cosine hemisphere or GGX
// visible normals (Heitz, JCGT 2018).  false if wi is below the surface.
__device__ __forceinline__ bool bsdf_sample(f3 n, f3 wo, float r, float ks, float u0, float u1, float u2, f3 &wi) {
    f3 T, B;
    onb(n, T, B);
    f3 l;
    float sp, cp;
    sincospif(2.0f * u2, &sp, &cp);
    if (u0 >= spec_prob(ks)) {
        const float rr = sqrtf(u1);
        l = mk3(rr * cp, rr * sp, sqrtf(fmaxf(0.0f, 1.0f - u1)));
    } else {
        float dadr;
        const float a = alpha_of(r, dadr);
        const f3 wl = mk3(dot(wo, T), dot(wo, B), dot(wo, n));
        const f3 Vh = normalize(mk3(a * wl.x, a * wl.y, wl.z));
        const float lsq = Vh.x * Vh.x + Vh.y * Vh.y;
        const f3 T1 = lsq > 0.0f ? mk3(-Vh.y, Vh.x, 0.0f) * (1.0f / sqrtf(lsq)) : mk3(1.0f, 0.0f, 0.0f);
        const f3 T2 = cross(Vh, T1);
        const float rr = sqrtf(u1);
        const float t1 = rr * cp;
        float t2 = rr * sp;
        const float s = 0.5f * (1.0f + Vh.z);
        t2 = (1.0f - s) * sqrtf(fmaxf(0.0f, 1.0f - t1 * t1)) + s * t2;
        const f3 Nh = T1 * t1 + T2 * t2 + Vh * sqrtf(fmaxf(0.0f, 1.0f - t1 * t1 - t2 * t2));
        const f3 Ne = normalize(mk3(a * Nh.x, a * Nh.y, fmaxf(0.0f, Nh.z)));
        l = Ne * (2.0f * dot(wl, Ne)) - wl;
    }
    wi = T * l.x + B * l.y + n * l.z;
    return dot(n, wi) > 0.0f;
}

// ---------------------------------------------------------------------------
// bilinear lookup, texel centres at (i + 1/2), clamp to edge
// ---------------------------------------------------------------------------
struct Bilin {
    int x0, y0;
    float fx, fy;
};
__device__ __forceinline__ Bilin bilin_setup(float xp, float yp, int W, int H) {
    float x = xp - 0.5f, y = yp - 0.5f;
    x = fminf(fmaxf(x, -1.0f), (float)W);
    y = fminf(fmaxf(y, -1.0f), (float)H);
    const float fx0 = floorf(x), fy0 = floorf(y);
    Bilin b;
    b.fx = x - fx0;
    b.fy = y - fy0;
    b.x0 = (int)fx0;
    b.y0 = (int)fy0;
    return b;
}
__device__ __forceinline__ void bilin_taps(const Bilin &b, int W, int H, int idx[4], float w[4]) {
    const int xa = min(max(b.x0, 0), W - 1), xb = min(max(b.x0 + 1, 0), W - 1);
    const int ya = min(max(b.y0, 0), H - 1), yb = min(max(b.y0 + 1, 0), H - 1);
    idx[0] = ya * W + xa;
    idx[1] = ya * W + xb;
    idx[2] = yb * W + xa;
    idx[3] = yb * W + xb;
    w[0] = (1.0f - b.fx) * (1.0f - b.fy);
    w[1] = b.fx * (1.0f - b.fy);
    w[2] = (1.0f - b.fx) * b.fy;
    w[3] = b.fx * b.fy;
}
__device__ __forceinline__ float4 bilin_fetch(const float4 *__restrict__ img, const Bilin &b, int W, int H) {
    int idx[4];
    float w[4];
    bilin_taps(b, W, H, idx, w);
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 v = __ldg(img + idx[k]);
        r.x += w[k] * v.x;
        r.y += w[k] * v.y;
        r.z += w[k] * v.z;
        r.w += w[k] * v.w;
    }
    return r;
}

// ---------------------------------------------------------------------------
// BVH traversal.  Node = 4 float4: (l.lo.x, l.hi.x, l.lo.y, l.hi.y),
// (r.lo.x, r.hi.x, r.lo.y, r.hi.y), (l.lo.z, l.hi.z, r.lo.z, r.hi.z),
// (left ref, right ref, -, -) with refs >= 0 internal, < 0 leaf ~position.
// Triangle = 3 float4: (v0, original index), v1, v2.
// ---------------------------------------------------------------------------
#ifndef DPCS_SLAB_FMA
#define DPCS_SLAB_FMA 1  // slab distances as fma(lo, 1/d, -o/d) with a per-ray absolute error margin
#endif

struct Ray {
    f3 o, d, inv;
#if DPCS_SLAB_FMA
    f3 oinv;    // o / d per axis
    float err;  // bound on the extra rounding of the fused form
#endif
};
__device__ __forceinline__ Ray make_ray(f3 o, f3 d) {
    Ray r;
    r.o = o;
    r.d = d;
    const float e = 1e-20f;
    r.inv = mk3(1.0f / (fabsf(d.x) > e ? d.x : copysignf(e, d.x)), 1.0f / (fabsf(d.y) > e ? d.y : copysignf(e, d.y)),
                1.0f / (fabsf(d.z) > e ? d.z : copysignf(e, d.z)));
#if DPCS_SLAB_FMA
    r.oinv = mk3(o.x * r.inv.x, o.y * r.inv.y, o.z * r.inv.z);
    r.err = 4.8e-7f * fmaxf(fmaxf(fabsf(r.oinv.x), fabsf(r.oinv.y)), fabsf(r.oinv.z));
#endif
    return r;
}

#ifndef DPCS_SLAB_MINMAX3
#define DPCS_SLAB_MINMAX3 1  // three-input min/max (PTX ISA 8.8, sm_100+)
#endif

__device__ __forceinline__ float fmax3f(float a, float b, float c) {
#if DPCS_SLAB_MINMAX3
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
#else
    return fmaxf(fmaxf(a, b), c);
#endif
}

__device__ __forceinline__ float fmin3f(float a, float b, float c) {
#if DPCS_SLAB_MINMAX3
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
#else
    return fminf(fminf(a, b), c);
#endif
}

// slab test; the far bound is widened by a few ulps (Ize, JCGT 2013) so that
// flat boxes of axis-aligned walls are never missed by rounding
__device__ __forceinline__ bool slab(const Ray &r, float lx, float hx, float ly, float hy, float lz, float hz,
                                     float tmax, float &tnear) {
#if DPCS_SLAB_FMA
    // fused form: its rounding error is bounded by a few ulps of |t| plus a
    // few ulps of |o / d|, which r.err covers
    const float tx0 = fmaf(lx, r.inv.x, -r.oinv.x), tx1 = fmaf(hx, r.inv.x, -r.oinv.x);
    const float ty0 = fmaf(ly, r.inv.y, -r.oinv.y), ty1 = fmaf(hy, r.inv.y, -r.oinv.y);
    const float tz0 = fmaf(lz, r.inv.z, -r.oinv.z), tz1 = fmaf(hz, r.inv.z, -r.oinv.z);
    const float tn = fmax3f(fminf(tx0, tx1), fminf(ty0, ty1), fmaxf(fminf(tz0, tz1), 0.0f));
    const float tf = fmin3f(fmaxf(tx0, tx1), fmaxf(ty0, ty1), fminf(fmaxf(tz0, tz1), tmax));
    tnear = tn;
    return tn <= fmaf(tf, 1.0000004f, r.err);
#else
    const float tx0 = (lx - r.o.x) * r.inv.x, tx1 = (hx - r.o.x) * r.inv.x;
    const float ty0 = (ly - r.o.y) * r.inv.y, ty1 = (hy - r.o.y) * r.inv.y;
    const float tz0 = (lz - r.o.z) * r.inv.z, tz1 = (hz - r.o.z) * r.inv.z;
    const float tn = fmax3f(fminf(tx0, tx1), fminf(ty0, ty1), fmaxf(fminf(tz0, tz1), 0.0f));
    const float tf = fmin3f(fmaxf(tx0, tx1), fmaxf(ty0, ty1), fminf(fmaxf(tz0, tz1), tmax));
    tnear = tn;
    return tn <= tf * 1.0000004f;
#endif
}

#ifndef DPCS_MT_DETCHECK
// 0: a ray with determinant exactly 0 (in the triangle's plane) goes to the
// watertight test; 1: also rays within a scaled near-parallel bound (two
// more dot products and a square root per test: 3 % slower, measured)
#define DPCS_MT_DETCHECK 0
#endif
#ifndef DPCS_WATERTIGHT
// 1: Moller-Trumbore, with the watertight test deciding every ray that MT
//    finds within rounding of an edge of the triangle (crack-free);
// 2: the watertight test for every triangle; 0: Moller-Trumbore alone
#define DPCS_WATERTIGHT 1
#endif

// component k of v, by selects (no local-memory array)
__device__ __forceinline__ float comp(f3 v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }

// Watertight ray-triangle test (Woop, Benthin, Wald, JCGT 2013), two-sided,
// t in (0, tmax].  The ray is sheared so that it runs along +z through the
// origin; the three 2-D edge functions of the sheared vertices then decide
// containment.  A vertex shared by two triangles is sheared identically in
// both, and each edge function is a difference of two separately rounded
// products (no FMA contraction), so the function of a shared edge in one
// triangle is the exact negative of its function in the other: a ray
// through an edge hits at least one of the two triangles, never neither.
// When an edge function is exactly 0 it is recomputed in FP64, as the paper
// prescribes.  u, v are the barycentric weights of v1 and v2.
__device__ __forceinline__ bool tri_isect_wt(const Ray &r, f3 v0, f3 v1, f3 v2, float tmax, float &t, float &u,
                                             float &v) {
    const float ax = fabsf(r.d.x), ay = fabsf(r.d.y), az = fabsf(r.d.z);
    const int kz = ax > ay ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
    int kx = kz == 2 ? 0 : kz + 1, ky = kx == 2 ? 0 : kx + 1;
    if (comp(r.d, kz) < 0.0f) {
        const int tmp = kx;
        kx = ky;
        ky = tmp;
    }
    const float sz = 1.0f / comp(r.d, kz);
    const float sx = comp(r.d, kx) * sz, sy = comp(r.d, ky) * sz;
    const f3 A = v0 - r.o, B = v1 - r.o, C = v2 - r.o;
    const float Az = comp(A, kz), Bz = comp(B, kz), Cz = comp(C, kz);
    const float Ax = __fsub_rn(comp(A, kx), __fmul_rn(sx, Az)), Ay = __fsub_rn(comp(A, ky), __fmul_rn(sy, Az));
    const float Bx = __fsub_rn(comp(B, kx), __fmul_rn(sx, Bz)), By = __fsub_rn(comp(B, ky), __fmul_rn(sy, Bz));
    const float Cx = __fsub_rn(comp(C, kx), __fmul_rn(sx, Cz)), Cy = __fsub_rn(comp(C, ky), __fmul_rn(sy, Cz));
    float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
    if (U == 0.0f || V == 0.0f || W == 0.0f) {
        U = (float)__dsub_rn(__dmul_rn((double)Cx, (double)By), __dmul_rn((double)Cy, (double)Bx));
        V = (float)__dsub_rn(__dmul_rn((double)Ax, (double)Cy), __dmul_rn((double)Ay, (double)Cx));
        W = (float)__dsub_rn(__dmul_rn((double)Bx, (double)Ay), __dmul_rn((double)By, (double)Ax));
    }
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return false;
    const float det = U + V + W;
    if (det == 0.0f) return false;
    const float T = U * (sz * Az) + V * (sz * Bz) + W * (sz * Cz);
    const float inv = 1.0f / det;
    t = T * inv;
    u = V * inv;
    v = W * inv;
    return t > 0.0f && t <= tmax;
}

// out of line: the rare edge cases stay out of the traversal loop's code
static __device__ __noinline__ bool tri_isect_wt_call(const Ray &r, f3 v0, f3 v1, f3 v2, float tmax, float &t,
                                                      float &u, float &v) {
    return tri_isect_wt(r, v0, v1, v2, tmax, t, u, v);
}

// Moller-Trumbore, two-sided, t in (0, tmax].  near_edge reports a miss
// within kEdgeTol (in barycentric units) of the triangle -- or a ray nearly
// in its plane -- for the watertight test to decide.  MT's barycentrics
// carry an absolute error of a few ulps times |o - v0| / (edge length):
// about 2e-5 for the 200k-triangle heightfield seen from the camera, so
// 1e-4 leaves a margin of five.
__device__ __forceinline__ bool tri_isect_mt(const Ray &r, f3 v0, f3 v1, f3 v2, float tmax, float &t, float &u,
                                             float &v, bool &near_edge) {
    constexpr float kEdgeTol = 1e-4f;
    const f3 e1 = v1 - v0, e2 = v2 - v0;
    const f3 p = cross(r.d, e2);
    const float det = dot(e1, p);
    near_edge = false;
#if DPCS_MT_DETCHECK
    if (fabsf(det) <= 1e-12f * dot(e1, e1) * sqrtf(dot(e2, e2))) {
        near_edge = true;
        return false;
    }
#else
    if (det == 0.0f) {  // a ray in the triangle's plane: the watertight test decides
        near_edge = true;
        return false;
    }
#endif
    const float inv = 1.0f / det;
    const f3 s = r.o - v0;
    u = dot(s, p) * inv;
    if (u < -kEdgeTol || u > 1.0f + kEdgeTol) return false;
    const f3 q = cross(s, e1);
    v = dot(r.d, q) * inv;
    if (v < -kEdgeTol || u + v > 1.0f + kEdgeTol) return false;
    if (u < 0.0f || v < 0.0f || u + v > 1.0f) {
        near_edge = true;
        return false;
    }
    t = dot(e2, q) * inv;
    return t > 0.0f && t <= tmax;
}

__device__ __forceinline__ bool tri_isect(const Ray &r, f3 v0, f3 v1, f3 v2, float tmax, float &t, float &u,
                                          float &v) {
#if DPCS_WATERTIGHT == 2
    return tri_isect_wt(r, v0, v1, v2, tmax, t, u, v);
#elif DPCS_WATERTIGHT == 1
    bool near_edge;
    if (tri_isect_mt(r, v0, v1, v2, tmax, t, u, v, near_edge)) return true;
    return near_edge && tri_isect_wt_call(r, v0, v1, v2, tmax, t, u, v);
#else
    bool near_edge;
    return tri_isect_mt(r, v0, v1, v2, tmax, t, u, v, near_edge);
#endif
}

struct Hit {
    int pos;   // leaf (sorted) position, -1 = miss
    int orig;  // original triangle index
    float t, u, v;
};

// BVH traversal.  Node = 4 float4: (l.lo.x, l.hi.x, l.lo.y, l.hi.y),
// (r.lo.x, r.hi.x, r.lo.y, r.hi.y), (l.lo.z, l.hi.z, r.lo.z, r.hi.z),
// (left ref, right ref, -, -) with refs >= 0 internal, < 0 leaf ~position.
// Triangle = 3 float4: (v0, original index), v1, v2.  Both children's boxes
// are tested; the nearer hit child is visited next and the other pushed.
// any = true stops at the first hit with t < tmax (shadow rays); otherwise
// the closest hit is kept, ties in t to the lowest original triangle index.
// (A 4-wide collapse of this tree was measured slower on GB300: its child
// sorting and masking cost more ALU issue than the halved node visits save.)
//
// The traversal is resumable: its state (node, stack depth, visit count, best
// hit) lives in Trav, kept by the caller.  After at least one step the loop
// yields (returns false) when fewer than `min_active` lanes of the warp are
// still traversing; it returns true once the ray is resolved.  Every call
// advances by one or more steps, so a lane that keeps calling it finishes its
// ray within the visit cap.
struct Trav {
    int node, sp, visits;
    bool any;
    Hit h;
};

__device__ __forceinline__ void trav_begin(Trav &st, int32_t root, float tmax, bool any) {
    st.node = root;
    st.sp = 0;
    st.visits = 0;
    st.any = any;
    st.h.pos = -1;
    st.h.orig = 0x7fffffff;
    st.h.t = tmax;
}

__device__ __forceinline__ bool trav_resume(const float4 *__restrict__ nodes, const float4 *__restrict__ tris,
                                            int32_t root, int32_t T, const Ray &ray, Trav &st, int *stack,
                                            unsigned *status, Cnt &cnt, int min_active, int cap_override = 0) {
    if (root == kEmptyRoot) return true;
    // a correct tree needs at most T - 1 node and T leaf visits per ray
    const int cap = cap_override > 0 ? cap_override : 2 * T + 16;
    bool first = true;
    while (true) {
        if (min_active > 0 && !first && __popc(__activemask()) < min_active) return false;
        first = false;
        cnt.add_warp(kCntTravWarpIter);
        if (++st.visits > cap) {
            atomicOr(status, kStatusTraversalLimit);
            st.h.pos = -1;
            return true;
        }
        const int node = st.node;
#ifdef DPCS_CHECK
        // debug build: every node and leaf reference is checked against the
        // tree before it is read; a bad one ends the ray and is reported
        if (node >= T - 1 || (node < 0 && ~node >= T)) {
            atomicOr(status, kStatusBoundsCheck);
            st.h.pos = -1;
            return true;
        }
#endif
        if (node >= 0) {
            cnt.add(kCntNode);
            const float4 n0 = __ldg(nodes + 4 * node + 0);
            const float4 n1 = __ldg(nodes + 4 * node + 1);
            const float4 n2 = __ldg(nodes + 4 * node + 2);
            const float4 n3 = __ldg(nodes + 4 * node + 3);
            float tl, tr;
            const bool hl = slab(ray, n0.x, n0.y, n0.z, n0.w, n2.x, n2.y, st.h.t, tl);
            const bool hr = slab(ray, n1.x, n1.y, n1.z, n1.w, n2.z, n2.w, st.h.t, tr);
            const int cl = __float_as_int(n3.x), cr = __float_as_int(n3.y);
            if (hl && hr) {
                if (st.sp >= kStack) {
                    atomicOr(status, kStatusTraversalLimit);
                    st.h.pos = -1;
                    return true;
                }
                const bool lfirst = tl <= tr;
                stack[st.sp++] = lfirst ? cr : cl;
                st.node = lfirst ? cl : cr;
                continue;
            }
            if (hl) { st.node = cl; continue; }
            if (hr) { st.node = cr; continue; }
        } else {
            const int pos = ~node;
            cnt.add(kCntTri);
            const float4 a = __ldg(tris + 3 * pos + 0);
            const float4 b = __ldg(tris + 3 * pos + 1);
            const float4 c = __ldg(tris + 3 * pos + 2);
            float t, u, v;
            if (tri_isect(ray, xyz(a), xyz(b), xyz(c), st.h.t, t, u, v)) {
                const int orig = __float_as_int(a.w);
                if (t < st.h.t || (!st.any && t == st.h.t && orig < st.h.orig)) {
                    st.h.pos = pos;
                    st.h.orig = orig;
                    st.h.t = t;
                    st.h.u = u;
                    st.h.v = v;
                    if (st.any) return true;
                }
            }
        }
        if (st.sp == 0) return true;
        st.node = stack[--st.sp];
    }
}

// traversal to completion (no yielding)
__device__ __forceinline__ bool traverse(const float4 *__restrict__ nodes, const float4 *__restrict__ tris,
                                         int32_t root, int32_t T, const Ray &ray, float tmax, bool any, Hit &h,
                                         unsigned *status, Cnt &cnt) {
    Trav st;
    int stack[kStack];
    trav_begin(st, root, tmax, any);
    trav_resume(nodes, tris, root, T, ray, st, stack, status, cnt, 0);
    h = st.h;
    return h.pos >= 0;
}

// ---------------------------------------------------------------------------
// One camera path: Eq. 10 with next-event estimation to the pinhole
// projector; optionally records what the replay adjoint needs.
// ---------------------------------------------------------------------------
struct VRec {
    int tx0, ty0, px0, py0;
    float tfx, tfy, pfx, pfy;
    float beta[3];
    float Ep[3];
    float G;       // k cos_p cos_s / r^2 when projector light arrived, else 0
    float rho[3];
    float sp, dsp; // spec(wo, wp) and d/dr
    float si, dsi; // spec(wo, wi) and d/dr
    float cw;      // cos_i / (pdf q) when the path continued, else 0
    unsigned unc;  // bit j: channel j not clipped
};

constexpr int kRecWords = (int)(sizeof(VRec) / 4);  // VRec as 32-bit words (records kept in device memory)
static_assert(kRecWords == kRecWordsHost, "the host sizes kept records with kRecWordsHost");

// Kept records in device memory: each VRec as six 16-byte chunks (words
// 4c..4c+3 of the struct); chunk c of record v of sample k of thread t sits
// at chunk index ((c * spl + k) * bounces + v) * nthreads + t, so a warp's
// accesses to one chunk are contiguous.
constexpr int kKeptChunks = kRecWords / 4;
static_assert(kRecWords % 4 == 0, "VRec must be whole 16-byte chunks");
constexpr int kKeptGChunk = (int)(offsetof(VRec, G) / 16), kKeptGWord = (int)(offsetof(VRec, G) % 16) / 4;
static_assert(offsetof(VRec, G) == 14 * 4, "k_render_keep writes G as word 2 of chunk 3");
__device__ __forceinline__ int64_t kept_chunk(int c, int k, int v, int spl, int bounces, int64_t nthr, int64_t t) {
    return (((int64_t)c * spl + k) * bounces + v) * nthr + t;
}

// first camera ray of sample s of pixel pix (Eq. 6 with the Eq. 4 box filter)
__device__ __forceinline__ void camera_ray(const RenderArgs &a, uint32_t pix, uint32_t s, f3 &o, f3 &d) {
    float u[4];
    rand4(a.key0, a.key1, pix, s, 0u, u);
    const float fx = (float)(pix % (uint32_t)a.Wc) + (a.jitter ? u[0] : 0.5f);
    const float fy = (float)(pix / (uint32_t)a.Wc) + (a.jitter ? u[1] : 0.5f);
    o = mk3(0.f, 0.f, 0.f);
    d = normalize(mat3v(a.Kci, mk3(fx, fy, 1.0f)));
}

// surface interaction at a hit: position, two-sided normal, textures
struct Surf {
    f3 x, n, wo, rho;
    float rough;
    Bilin tb;
};
__device__ __forceinline__ Surf surface_at(const RenderArgs &a, const Hit &h, f3 d) {
    Surf S;
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
    S.rho = mk3(tex.x, tex.y, tex.z);
    S.rough = tex.w;
    S.wo = d * -1.0f;
    return S;
}

// next-event estimation towards the pinhole projector (Eqs. 1, 2, 3, 6)
// without the visibility test: the shadow ray and everything the
// contribution needs.  false if the projector cannot light the point.
struct Nee {
    f3 so, sdir;
    float smax;
    Bilin pb;
    float4 ep;
    float G, sp, dsp;
    f3 fp;
};
__device__ __forceinline__ bool nee_prepare(const RenderArgs &a, const Surf &S, Nee &N) {
    const f3 cp = mk3(a.cp[0], a.cp[1], a.cp[2]);
    const f3 X = mat3v(a.Rp, S.x) + mk3(a.tp[0], a.tp[1], a.tp[2]);
    const f3 q = mat3v(a.Kp, X);
    if (!(q.z > 0.0f && X.z > 0.0f)) return false;
    const float up = q.x / q.z, vp = q.y / q.z;
    if (!(up >= 0.0f && up < (float)a.Wp && vp >= 0.0f && vp < (float)a.Hp)) return false;
    const f3 v = cp - S.x;
    const float r2 = dot(v, v), dist = sqrtf(r2);
    const f3 wp = v * (1.0f / dist);
    const float cs = dot(S.n, wp);
    if (!(cs > 0.0f)) return false;
    const float cpz = X.z / sqrtf(dot(X, X));
    N.so = S.x + S.n * kRayEps;
    const f3 sv = cp - N.so;
    const float sd = sqrtf(dot(sv, sv));
    N.sdir = sv * (1.0f / sd);
    N.smax = sd - kRayEps;
    N.pb = bilin_setup(up, vp, a.Wp, a.Hp);
    N.ep = bilin_fetch(a.Ep, N.pb, a.Wp, a.Hp);
    N.G = a.k_proj * cpz * cs / r2;
    N.sp = spec_eval(S.n, S.wo, wp, S.rough, a.ks, a.f0, N.dsp);
    N.fp = mk3(S.rho.x * DPCS_INV_PI_F + N.sp, S.rho.y * DPCS_INV_PI_F + N.sp, S.rho.z * DPCS_INV_PI_F + N.sp);
    return true;
}

// contribution beta f Ep G of a visible projector, clipped per channel (Eq. 12)
__device__ __forceinline__ f3 nee_contrib(const RenderArgs &a, f3 beta, const Nee &N, unsigned &unc) {
    f3 c = beta * N.fp * mk3(N.ep.x, N.ep.y, N.ep.z) * N.G;
    unc = 7u;
    if (a.clip > 0.0f) {
        if (c.x > a.clip) { c.x = a.clip; unc &= ~1u; }
        if (c.y > a.clip) { c.y = a.clip; unc &= ~2u; }
        if (c.z > a.clip) { c.z = a.clip; unc &= ~4u; }
    }
    return c;
}

// continuation from vertex b: BRDF sampling, throughput weight, Russian
// roulette (Eq. 10).  false ends the path.
struct Cont {
    f3 wi, w;       // direction and throughput factor f cos / (pdf q)
    float cw, si, dsi;
};
__device__ __forceinline__ bool continue_prepare(const RenderArgs &a, uint32_t pix, uint32_t s, int b,
                                                 const Surf &S, Cont &C) {
    float u[4];
    rand4(a.key0, a.key1, pix, s, (uint32_t)b, u);
    if (!bsdf_sample(S.n, S.wo, S.rough, a.ks, u[0], u[1], u[2], C.wi)) return false;
    const float pdf = bsdf_pdf(S.n, S.wo, C.wi, S.rough, a.ks);
    if (!(pdf > 0.0f)) return false;
    float qrr = 1.0f;
    if (a.rr_start > 0 && b >= a.rr_start) {
        if (u[3] >= a.rr_q) return false;
        qrr = a.rr_q;
    }
    C.si = spec_eval(S.n, S.wo, C.wi, S.rough, a.ks, a.f0, C.dsi);
    C.cw = dot(S.n, C.wi) / (pdf * qrr);
    const f3 fi = mk3(S.rho.x * DPCS_INV_PI_F + C.si, S.rho.y * DPCS_INV_PI_F + C.si,
                      S.rho.z * DPCS_INV_PI_F + C.si);
    C.w = fi * C.cw;
    return true;
}

}  // namespace dpcs
