// pose.cu -- gradient of a loss on the camera image with respect to the
// camera pose (Sec. 3.2 counts the camera rotation Rc and translation tc
// among the scene parameters theta of Eq. 9).
//
// Renders keep the camera at the origin (Eq. 6), so a pose change moves the
// whole scene rigidly in the camera frame: a point y moves with velocity
// a x y + b, the twist (a, b) of the pose parameter.  The pixel mean of Eq. 4
// integrates the radiance over the pixel's square.  Pulled back onto the
// visible surfaces its integrand L(x) J(x) (J = image area per unit surface
// area) moves with the scene, and so do the shadow edges and the projector
// frustum's border on those surfaces: relative to the scene only the camera
// moves.  Differentiating each visible region's integral as its boundary
// moves leaves three terms, with g_P = dLoss/dEc of pixel P:
//   interior     per camera sample: the first vertex's BRDF change as its
//                direction to the camera turns, plus the whole path
//                contribution times d log J;
//   pixel edges  per pixel P: -g_P times the flux out of its square, the
//                integral over its four edges of L (V . n), V the image
//                velocity of the first hit seen on the edge and n the
//                outward normal (edge by edge the same sum as
//                L (V . n) (g_Q - g_P) over the edges between pixels P and
//                Q, but with the four edges' paths sharing their random
//                numbers, opposite edges give a low-variance difference);
//   silhouettes  where a mesh edge of a nearer surface F hides a surface B,
//                B's visible region ends at F's edge, which moves with F:
//                g_P L_B (V_F - V_B) . n, n turned towards F, along the
//                edge's image.
// Each term is linear in (a, b), so the kernels accumulate the six
// components of dLoss/d(a, b), a wrench; the derivative for any pose
// parameter is its twist's dot product with the wrench.
//
// The derivatives are analytic, in FP32: the GGX lobe's gradient in its
// outgoing direction; d log J = n.b / n.x - 3 (Kc v)_z / (Kc x)_z from
// J = |det Kc| |n.x| / (Kc x)_z^3; the image velocity M(y) (a x y + b) with
// M the Jacobian of the projection y -> (Kc y)_xy / (Kc y)_z.
//
// Work: one thread per item (a camera sample, a pixel's four edge samples
// or a silhouette sample) with a fixed grid stride, each path traced to its end
// by the same steps as the render (Eqs. 3, 6, 10).  Threads accumulate in
// FP32, blocks reduce in FP64 to one partial per block, and one block sums
// the partials in a fixed order: results repeat bit for bit.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "device.cuh"
#include "internal.h"
#include "pose.h"
#include "principled.cuh"

namespace dpcs {

namespace {

constexpr int kPoseBlock = 128;
// Blocks per SM in the grid-stride grids (4 fit at a time at these register
// counts; the rest balance the uneven paths).  Measured on the corner at
// 256 x 256, 16 spp: the interior kernel 0.75 / 0.73 / 0.87 ms at 8 / 16 /
// 32 blocks per SM, the pixel-edge kernel (16 samples) 2.53 / 2.24 / 1.88 ms.
constexpr int kPoseGridInterior = 16, kPoseGridEdges = 32, kPoseGridSil = 16;
constexpr int kPoseBlocksPerSM = 32;  // the largest of the three: the partial sums' stride
#ifndef DPCS_POSE_MINB
#define DPCS_POSE_MINB 4  // resident blocks per SM asked of ptxas for the path-tracing pose kernels
#endif

// Gradient of spec(wo, wi) = ks D G1(ci) G1(co) F / (4 ci co) in wo, wo
// taken as a free vector (its product with a direction tangent to the unit
// sphere is the directional derivative).  With h = (wo + wi) / |wo + wi|,
// D depends on ch = n.h through t = 1 + ch^2 (a^2 - 1); G1(co) / co =
// 2 / (co + sqrt(a^2 + (1 - a^2) co^2)); F = f0 + (1 - f0) (1 - wo.h)^5.
__device__ f3 spec_grad_wo(f3 n, f3 wo, f3 wi, float r, float ks, float f0) {
    const float co = dot(n, wo), ci = dot(n, wi);
    if (ks <= 0.0f || co <= 0.0f || ci <= 0.0f) return mk3(0.f, 0.f, 0.f);
    float dadr;
    const float a = alpha_of(r, dadr);
    const float a2 = a * a;
    const f3 hu = wo + wi;
    const float lh = sqrtf(dot(hu, hu));
    const float il = 1.0f / lh;
    const f3 h = hu * il;
    const float ch = dot(n, h);
    const float t = sin2(n, h) + a2 * ch * ch;
    const float D = a2 / (DPCS_PI_F * t * t);
    const float si = sqrtf(a2 + (1.0f - a2) * ci * ci), so = sqrtf(a2 + (1.0f - a2) * co * co);
    const float G = (2.0f * ci / (ci + si)) * (2.0f * co / (co + so));
    const float woh = dot(wo, h);
    const float m = fmaxf(0.0f, 1.0f - woh);
    const float m2 = m * m;
    const float F = f0 + (1.0f - f0) * (m2 * m2 * m);
    const float spec = ks * D * G * F / (4.0f * ci * co);
    // d ln D / d ch and d ch / d wo = (n - h ch) / |wo + wi|
    const float dlnD = -4.0f * ch * (a2 - 1.0f) / t;
    // d ln(G1(co) / co) / d co
    const float dlnGc = -(1.0f + (1.0f - a2) * co / so) / (co + so);
    f3 g = (n - h * ch) * (spec * dlnD * il) + n * (spec * dlnGc);
    if (m > 0.0f) {
        // d (wo.h) / d wo = h + (wo - h (wo.h)) / |wo + wi|
        const f3 dwoh = h + (wo - h * woh) * il;
        const float dF = -5.0f * (1.0f - f0) * (m2 * m2);
        g = g + dwoh * (ks * D * G * dF / (4.0f * ci * co));
    }
    return g;
}

// The principled lobe's pieces as functions of wo (a free vector), at the
// shading normal n: S = ks D G1(ci) G1(co) / (4 ci co) and s5 = (1 - wo.h)^5,
// so that f_j = (1 - m) rho_j / pi + S F_j with F_j = F0_j + (1 - F0_j) s5
// has grad f_j = F_j grad S + S (1 - F0_j) grad s5.  Zero where the lobe is
// off (wo or wi below the shading hemisphere) or ks = 0.
__device__ void plobe_grad_wo(f3 n, f3 wo, f3 wi, float r, float ks, f3 &gS, f3 &gs5) {
    gS = gs5 = mk3(0.f, 0.f, 0.f);
    const float co = dot(n, wo), ci = dot(n, wi);
    if (ks <= 0.0f || co <= 0.0f || ci <= 0.0f) return;
    float dadr;
    const float a = alpha_of(r, dadr);
    const float a2 = a * a;
    const f3 hu = wo + wi;
    const float il = 1.0f / sqrtf(dot(hu, hu));
    const f3 h = hu * il;
    const float ch = dot(n, h);
    const float t = sin2(n, h) + a2 * ch * ch;
    const float D = a2 / (DPCS_PI_F * t * t);
    const float si = sqrtf(a2 + (1.0f - a2) * ci * ci), so = sqrtf(a2 + (1.0f - a2) * co * co);
    const float S = ks * D * (2.0f * ci / (ci + si)) * (2.0f * co / (co + so)) / (4.0f * ci * co);
    const float dlnD = -4.0f * ch * (a2 - 1.0f) / t;                 // d ln D / d ch
    const float dlnGc = -(1.0f + (1.0f - a2) * co / so) / (co + so);  // d ln(G1(co) / co) / d co
    gS = (n - h * ch) * (S * dlnD * il) + n * (S * dlnGc);
    const float woh = dot(wo, h);
    const float m = 1.0f - woh;
    if (m > 0.0f) {
        const float m2 = m * m;
        gs5 = (h + (wo - h * woh) * il) * (-5.0f * m2 * m2);
    }
}

__device__ __forceinline__ f3 krow(const float *K, int r) { return mk3(K[3 * r], K[3 * r + 1], K[3 * r + 2]); }

// row c (0: x, 1: y) of the Jacobian of s = (K y)_xy / (K y)_z at y
__device__ __forceinline__ f3 proj_row(const float *K, f3 y, int c) {
    const f3 q = mat3v(K, y);
    const float iz = 1.0f / q.z;
    const float sc = (c == 0 ? q.x : q.y) * iz;
    return (krow(K, c) - krow(K, 2) * sc) * iz;
}

// What the pose terms keep of one path.  All terms: the first hit x and (for
// the pixel-edge and silhouette terms) the radiance L.  The interior term,
// whose pixel weight g = dLoss/dEc / spp is known before the path is traced,
// reduces the first vertex at once to the coefficients of the sample's
// wrench (A, B) = S (Acoef, Bcoef) + (0, [lit] Qp + Ai Pi):
//   S      sum over the path's lit vertices of g . contribution;
//   Acoef, Bcoef  d log J = a . Acoef + b . Bcoef at the first vertex;
//   Qp     the first vertex's light term's derivative along wo's turn,
//          counted when the projector sees that vertex (lit);
//   Ai, Pi the later vertices carry f(wo, wi) of the first one: Ai sums
//          g_j c_j / f_j(wo, wi) over their unclipped channels, and Pi is
//          the turn of wo applied to the gradient of f's GGX part.
// With the principled material grad f_j differs between channels (F_j and
// F0_j do), so Ai is kept per channel (Ai3) and the continuation's turn is
// kept as the turns of grad S and grad s5 (PiS, Pis5) with their channel
// weights F_j and S (1 - F0_j) at wi (cF, cS5).
struct Walk {
    int nv;        // vertices (0: the first ray left the scene)
    f3 x, L;
    float S, Ai;
    f3 Acoef, Bcoef, Qp, Pi, gf;  // gf_j = g_j / f_j(wo, wi) of the first vertex
    f3 Ai3, PiS, Pis5, cF, cS5;   // principled material
    bool lit;
};

// -(v - wo (v.wo)) / |x|: with the camera centre moving by -b relative to the
// scene, wo turns by dwo = -(b - wo (wo.b)) / |x|, and v . dwo = b . this
__device__ __forceinline__ f3 wo_turn(f3 v, f3 wo, float ilx) { return (v - wo * dot(v, wo)) * (-ilx); }

// The path of the ray (o, d): continuation b draws counter (pix, s, b, 0).
// One traversal per loop iteration -- the closest hit of the current ray or
// the shadow ray of the last vertex's light -- so that the lanes of a warp
// run the same traversal code whatever step their paths are at.
// kPbr: the principled material (mat = its packed maps); otherwise the
// plain Lambert + GGX material.
template <bool kInterior, bool kPbr>
__device__ void pose_trace(const RenderArgs &a, const float4 *__restrict__ mat, const float *Kc, float g0, float g1,
                           float g2, f3 o, f3 d, uint32_t pix, uint32_t s, Walk &W, Cnt &cnt) {
    const f3 zero = mk3(0.f, 0.f, 0.f);
    W.nv = 0;
    W.x = W.L = W.Acoef = W.Bcoef = W.Qp = W.Pi = W.gf = zero;
    W.Ai3 = W.PiS = W.Pis5 = W.cF = W.cS5 = zero;
    W.S = W.Ai = 0.0f;
    W.lit = false;
    f3 beta = mk3(1.f, 1.f, 1.f);
    Ray ray = make_ray(o, d);
    float tmax = INFINITY;
    bool shadow = false, has_ext = false, pfirst = false;
    f3 pc = zero, ext_o = zero, ext_d = zero;  // pending light contribution; next extension ray
    unsigned punc = 0u;
    int b = 1;
    for (int it = 0; it < 2 * a.bounces; ++it) {
        Hit h;
        const bool hit = traverse(a.nodes, a.tris, a.root, a.T, ray, tmax, shadow, h, a.status, cnt);
        if (shadow) {
            if (!hit) {  // the projector sees the vertex
                if constexpr (kInterior) {
                    W.S += g0 * pc.x + g1 * pc.y + g2 * pc.z;
                    if (pfirst)
                        W.lit = true;
                    else if constexpr (kPbr)
                        W.Ai3 = W.Ai3 + mk3((punc & 1u) ? W.gf.x * pc.x : 0.f, (punc & 2u) ? W.gf.y * pc.y : 0.f,
                                            (punc & 4u) ? W.gf.z * pc.z : 0.f);
                    else
                        W.Ai += ((punc & 1u) ? W.gf.x * pc.x : 0.f) + ((punc & 2u) ? W.gf.y * pc.y : 0.f) +
                                ((punc & 4u) ? W.gf.z * pc.z : 0.f);
                } else {
                    W.L = W.L + pc;
                }
            }
            shadow = false;
            if (!has_ext) break;
            ray = make_ray(ext_o, ext_d);
            tmax = INFINITY;
            has_ext = false;
            ++b;
            continue;
        }
        if (!hit) break;
        bool cand;
        f3 sh_o, sh_d;  // shadow ray of the vertex's light (when cand)
        float sh_max = 0.0f;
        if constexpr (kPbr) {
            const PSurf S = psurface_at(a, mat, h, ray.d);
            pfirst = W.nv == 0;
            ++W.nv;
            float ilx = 0.0f;
            if (pfirst) {
                W.x = S.x;
                if constexpr (kInterior) {
                    ilx = 1.0f / sqrtf(dot(S.x, S.x));
                    const f3 k2 = krow(Kc, 2);
                    const float w = 3.0f / dot(k2, S.x);
                    W.Acoef = cross(S.x, k2) * (-w);
                    W.Bcoef = S.n * (1.0f / dot(S.n, S.x)) - k2 * w;
                }
            }
            PNee N;
            cand = pnee_prepare(a, S, N);
            if (cand) {
                pc = beta * N.fp * mk3(N.ep.x, N.ep.y, N.ep.z) * N.G;
                punc = 7u;
                if (a.clip > 0.0f) {
                    if (pc.x > a.clip) { pc.x = a.clip; punc &= ~1u; }
                    if (pc.y > a.clip) { pc.y = a.clip; punc &= ~2u; }
                    if (pc.z > a.clip) { pc.z = a.clip; punc &= ~4u; }
                }
                sh_o = N.so;
                sh_d = N.sdir;
                sh_max = N.smax;
                if constexpr (kInterior) {
                    if (pfirst && N.L.on > 0.0f) {
                        // weights g_j unc_j Ep_j G of grad f_j = F_j grad S + S (1 - F0_j) grad s5
                        const f3 wgt = mk3((punc & 1u) ? g0 * N.ep.x : 0.f, (punc & 2u) ? g1 * N.ep.y : 0.f,
                                           (punc & 4u) ? g2 * N.ep.z : 0.f) * N.G;
                        const f3 F0 = S.rho * S.m + mk3(1.f, 1.f, 1.f) * ((1.0f - S.m) * a.f0);
                        const f3 F = F0 + (mk3(1.f, 1.f, 1.f) - F0) * N.L.s5;
                        const float cS = dot(wgt, F), cs5 = N.L.S * dot(wgt, mk3(1.f, 1.f, 1.f) - F0);
                        if (cS != 0.0f || cs5 != 0.0f) {
                            const f3 cp = mk3(a.cp[0], a.cp[1], a.cp[2]);
                            f3 gS, gs5;
                            plobe_grad_wo(S.ns, S.wo, normalize(cp - S.x), S.rough, a.ks, gS, gs5);
                            W.Qp = wo_turn(gS, S.wo, ilx) * cS + wo_turn(gs5, S.wo, ilx) * cs5;
                        }
                    }
                }
            }
            has_ext = false;
            if (b < a.bounces) {
                PCont C;
                if (pcontinue_prepare(a, pix, s, b, S, C)) {
                    if constexpr (kInterior) {
                        if (pfirst) {
                            const f3 fi = pbrdf(S.rho, S.m, a.f0, C.L);
                            W.gf = mk3(fi.x > 0.f ? g0 / fi.x : 0.f, fi.y > 0.f ? g1 / fi.y : 0.f,
                                       fi.z > 0.f ? g2 / fi.z : 0.f);
                            const f3 F0 = S.rho * S.m + mk3(1.f, 1.f, 1.f) * ((1.0f - S.m) * a.f0);
                            W.cF = (F0 + (mk3(1.f, 1.f, 1.f) - F0) * C.L.s5) * C.L.on;
                            W.cS5 = (mk3(1.f, 1.f, 1.f) - F0) * (C.L.S * C.L.on);
                            f3 gS, gs5;
                            plobe_grad_wo(S.ns, S.wo, C.wi, S.rough, a.ks, gS, gs5);
                            W.PiS = wo_turn(gS, S.wo, ilx);
                            W.Pis5 = wo_turn(gs5, S.wo, ilx);
                        }
                    }
                    beta = beta * C.w;
                    ext_o = S.x + S.n * kRayEps;
                    ext_d = C.wi;
                    has_ext = true;
                }
            }
        } else {
            const Surf S = surface_at(a, h, ray.d);
            pfirst = W.nv == 0;
            ++W.nv;
            float ilx = 0.0f;
            if (pfirst) {
                W.x = S.x;
                if constexpr (kInterior) {
                    ilx = 1.0f / sqrtf(dot(S.x, S.x));
                    // d log J = n.b / n.x - 3 k2.(a x x + b) / k2.x, k2 = Kc's third row
                    const f3 k2 = krow(Kc, 2);
                    const float w = 3.0f / dot(k2, S.x);
                    W.Acoef = cross(S.x, k2) * (-w);
                    W.Bcoef = S.n * (1.0f / dot(S.n, S.x)) - k2 * w;
                }
            }
            Nee N;
            cand = nee_prepare(a, S, N);
            if (cand) {
                pc = nee_contrib(a, beta, N, punc);
                if constexpr (kInterior) {
                    if (pfirst) {
                        const float Ap = (((punc & 1u) ? g0 * N.ep.x : 0.f) + ((punc & 2u) ? g1 * N.ep.y : 0.f) +
                                          ((punc & 4u) ? g2 * N.ep.z : 0.f)) * N.G;  // throughput 1 at the first vertex
                        if (Ap != 0.0f) {
                            const f3 cp = mk3(a.cp[0], a.cp[1], a.cp[2]);
                            const f3 v = spec_grad_wo(S.n, S.wo, normalize(cp - S.x), S.rough, a.ks, a.f0);
                            W.Qp = wo_turn(v, S.wo, ilx) * Ap;
                        }
                    }
                }
            }
            has_ext = false;
            if (b < a.bounces) {
                Cont C;
                if (continue_prepare(a, pix, s, b, S, C)) {
                    if constexpr (kInterior) {
                        if (pfirst) {
                            const float f0c = S.rho.x * DPCS_INV_PI_F + C.si, f1c = S.rho.y * DPCS_INV_PI_F + C.si,
                                        f2c = S.rho.z * DPCS_INV_PI_F + C.si;
                            W.gf = mk3(f0c > 0.f ? g0 / f0c : 0.f, f1c > 0.f ? g1 / f1c : 0.f, f2c > 0.f ? g2 / f2c : 0.f);
                            W.Pi = wo_turn(spec_grad_wo(S.n, S.wo, C.wi, S.rough, a.ks, a.f0), S.wo, ilx);
                        }
                    }
                    beta = beta * C.w;
                    ext_o = S.x + S.n * kRayEps;
                    ext_d = C.wi;
                    has_ext = true;
                }
            }
            if (cand) {
                sh_o = N.so;
                sh_d = N.sdir;
                sh_max = N.smax;
            }
        }
        if (cand) {
            shadow = true;
            ray = make_ray(sh_o, sh_d);
            tmax = sh_max;
        } else if (has_ext) {
            ray = make_ray(ext_o, ext_d);
            tmax = INFINITY;
            has_ext = false;
            ++b;
        } else {
            break;
        }
    }
}

__device__ __forceinline__ void add6(float acc[6], f3 A, f3 B) {
    acc[0] += A.x;
    acc[1] += A.y;
    acc[2] += A.z;
    acc[3] += B.x;
    acc[4] += B.y;
    acc[5] += B.z;
}

// the block's six sums in FP64, written to out[0..5] (every block writes)
__device__ void block_partial(const float acc[6], double *out) {
    __shared__ double red[6][kPoseBlock / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        double v = (double)acc[k];
        for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) red[k][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double s = 0.0;
        for (int j = 0; j < kPoseBlock / 32; ++j) s += red[threadIdx.x][j];
        out[threadIdx.x] = s;
    }
}

// Interior term, one item per camera sample (pixel i / spp, sample i % spp),
// the sample's path as the render traces it.
template <bool kPbr>
__global__ void __launch_bounds__(kPoseBlock, DPCS_POSE_MINB) k_pose_interior(const RenderArgs a, const PoseArgs p) {
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    Cnt cnt;
    const int64_t npix = (int64_t)a.Hc * a.Wc;
    const int64_t total = npix * a.spp;
    const float inv = 1.0f / (float)a.spp;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const int64_t pix = i / a.spp;
        const int s = (int)(i - pix * a.spp);
        const float g0 = a.gE[3 * pix] * inv, g1 = a.gE[3 * pix + 1] * inv, g2 = a.gE[3 * pix + 2] * inv;
        if (g0 == 0.0f && g1 == 0.0f && g2 == 0.0f) continue;
        f3 o, d;
        camera_ray(a, (uint32_t)pix, (uint32_t)s, o, d);
        Walk W;
        pose_trace<true, kPbr>(a, p.mat, p.Kc, g0, g1, g2, o, d, (uint32_t)pix, (uint32_t)s, W, cnt);
        if (W.nv == 0) continue;
        f3 Qi;  // the continuation's BRDF factor, turned with wo
        if constexpr (kPbr)
            Qi = W.PiS * dot(W.Ai3, W.cF) + W.Pis5 * dot(W.Ai3, W.cS5);
        else
            Qi = W.Pi * W.Ai;
        add6(acc, W.Acoef * W.S, W.Bcoef * W.S + (W.lit ? W.Qp : mk3(0.f, 0.f, 0.f)) + Qi);
    }
    block_partial(acc, p.partial + 6 * (int64_t)blockIdx.x);
}

// Pixel-edge term: -g_P times the flux out of pixel P's square.  Sample j
// of pixel p = (x0, y0) puts one point at t = (j + u0) / edge_spp along each
// of its edges -- right (x0 + 1, y0 + t), left (x0, y0 + t), bottom
// (x0 + t, y0 + 1), top (x0 + t, y0), outward normals +x, -x, +y, -y -- and
// the four paths share counter (Hc Wc + p, j, b, 0), so that the flux
// through opposite edges is a common-random-number difference across P.
template <bool kPbr>
__global__ void __launch_bounds__(kPoseBlock, DPCS_POSE_MINB) k_pose_edges(const RenderArgs a, const PoseArgs p) {
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    Cnt cnt;
    const int64_t npix = (int64_t)a.Hc * a.Wc;
    const int64_t total = npix * p.edge_spp;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const float inv = 1.0f / (float)p.edge_spp;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const int64_t pix = i / p.edge_spp;
        const int j = (int)(i - pix * p.edge_spp);
        const float g0 = a.gE[3 * pix], g1 = a.gE[3 * pix + 1], g2 = a.gE[3 * pix + 2];
        if (g0 == 0.0f && g1 == 0.0f && g2 == 0.0f) continue;
        const float x0 = (float)(pix % a.Wc), y0 = (float)(pix / a.Wc);
        const uint32_t vpix = (uint32_t)(npix + pix);
        float u[4];
        rand4(a.key0, a.key1, vpix, (uint32_t)j, 0u, u);
        const float t = ((float)j + u[0]) * inv;
#pragma unroll 1
        for (int k = 0; k < 4; ++k) {
            const float sx = k == 0 ? x0 + 1.0f : (k == 1 ? x0 : x0 + t);
            const float sy = k < 2 ? y0 + t : (k == 2 ? y0 + 1.0f : y0);
            const f3 d = normalize(mat3v(a.Kci, mk3(sx, sy, 1.0f)));
            Walk W;
            pose_trace<false, kPbr>(a, p.mat, p.Kc, 0.f, 0.f, 0.f, mk3(0.f, 0.f, 0.f), d, vpix, (uint32_t)j, W, cnt);
            if (W.nv == 0) continue;
            // -(outward sign) g . L / edge_spp times V . n = m . (a x x + b),
            // m the Jacobian row across the edge
            const float gl = (W.L.x * g0 + W.L.y * g1 + W.L.z * g2) * ((k & 1) ? inv : -inv);
            if (gl == 0.0f) continue;
            const f3 m = proj_row(p.Kc, W.x, k < 2 ? 0 : 1);
            add6(acc, cross(W.x, m) * gl, m * gl);
        }
    }
    block_partial(acc, p.partial + 6 * (int64_t)blockIdx.x);
}

// Silhouette term.  Mesh edge k (PoseEdge order) is a silhouette when its
// triangles all lie on one side of the plane through the camera centre and
// the edge.  Sample j sits at t = (j + u0) / sil_spp from the lower-numbered
// vertex, u from counter (2 Hc Wc + k, j, 0, 0); it counts if
// it lies in front of the camera, inside the image and in view, and the path
// continuing behind it (B) draws the same counter's later bounces.
template <bool kPbr>
__global__ void __launch_bounds__(kPoseBlock, DPCS_POSE_MINB) k_pose_sil(const RenderArgs a, const PoseArgs p) {
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    Cnt cnt;
    const int64_t Hc = a.Hc, Wc = a.Wc, npix = Hc * Wc;
    const int64_t vbase = 2 * npix;
    const int64_t total = p.nedges * p.sil_spp;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const int64_t k = i / p.sil_spp;
        const int j = (int)(i - k * p.sil_spp);
        const PoseEdge E = p.edges[k];
        if (E.x < 0) continue;  // more than two triangles share the edge
        const float4 *tA = a.tris + 3 * (int64_t)E.x;
        const f3 P0 = xyz(tA[E.y & 3]), P1 = xyz(tA[(E.y >> 2) & 3]), P2 = xyz(tA[(E.y >> 4) & 3]);
        const f3 mplane = cross(P0, P1);
        const float sa = dot(mplane, P2);
        if (sa == 0.0f) continue;
        if (E.z >= 0) {
            const float sb = dot(mplane, xyz(a.tris[3 * (int64_t)E.z + E.w]));
            if (!(sa > 0.0f ? sb > 0.0f : sb < 0.0f)) continue;
        }
        const uint32_t vpix = (uint32_t)(vbase + k);
        float u[4];
        rand4(a.key0, a.key1, vpix, (uint32_t)j, 0u, u);
        const float t = ((float)j + u[0]) / (float)p.sil_spp;
        const f3 de = P1 - P0;
        const f3 pe = P0 + de * t;
        if (!(pe.z > 0.0f)) continue;
        const f3 q = mat3v(p.Kc, pe);
        const float sx = q.x / q.z, sy = q.y / q.z;
        if (!(sx >= 0.0f && sx < (float)Wc && sy >= 0.0f && sy < (float)Hc)) continue;
        const float dist = sqrtf(dot(pe, pe));
        const f3 d = pe * (1.0f / dist);
        Hit hs;
        const Ray vr = make_ray(mk3(0.f, 0.f, 0.f), d);
        if (traverse(a.nodes, a.tris, a.root, a.T, vr, dist * (1.0f - 1e-4f), true, hs, a.status, cnt)) continue;
        Walk W;
        pose_trace<false, kPbr>(a, p.mat, p.Kc, 0.f, 0.f, 0.f, d * (dist * (1.0f + 1e-4f)), d, vpix, (uint32_t)j, W, cnt);
        if (W.nv == 0) continue;
        const int64_t px = (int64_t)floorf(sy) * Wc + (int64_t)floorf(sx);
        const float gl = W.L.x * a.gE[3 * px] + W.L.y * a.gE[3 * px + 1] + W.L.z * a.gE[3 * px + 2];
        if (gl == 0.0f) continue;
        // the edge's image tangent per unit t, its normal turned towards F
        // (the image of the third vertex's side), and the two velocities
        // across it: V_F of the edge point, V_B of B's first hit
        const f3 mx = proj_row(p.Kc, pe, 0), my = proj_row(p.Kc, pe, 1);
        const float tx = dot(mx, de), ty = dot(my, de);
        const float tl = sqrtf(tx * tx + ty * ty);
        if (!(tl > 0.0f)) continue;
        float nx = -ty / tl, ny = tx / tl;
        const f3 dF = P2 - pe;
        if (nx * dot(mx, dF) + ny * dot(my, dF) < 0.0f) {
            nx = -nx;
            ny = -ny;
        }
        const f3 uf = mx * nx + my * ny;
        const f3 ub = proj_row(p.Kc, W.x, 0) * nx + proj_row(p.Kc, W.x, 1) * ny;
        const float w = gl * tl / (float)p.sil_spp;
        add6(acc, (cross(pe, uf) - cross(W.x, ub)) * w, (uf - ub) * w);
    }
    block_partial(acc, p.partial + 6 * (int64_t)blockIdx.x);
}

// wrench[6 term + c] += the sum of the term's block partials of component
// c: one warp per (term, c), lane l adding blocks l, l + 32, ... in order,
// then a fixed shuffle tree (the same order on every call)
__global__ void k_pose_reduce(const double *__restrict__ partial, int gmax, int g0, int g1, int g2,
                              double *__restrict__ wrench) {
    const int t = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (t >= 18) return;
    const int term = t / 6, c = t % 6;
    const int g = term == 0 ? g0 : (term == 1 ? g1 : g2);
    double s = 0.0;
    for (int b = lane; b < g; b += 32) s += partial[((int64_t)term * gmax + b) * 6 + c];
    for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) wrench[t] += s;
}

}  // namespace

int pose_grid(int device) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0) return 0;
    return sms * kPoseBlocksPerSM;
}

int launch_pose(const RenderArgs &a, const PoseArgs &p, int device, double *wrench, cudaStream_t st) {
    const int gmax = pose_grid(device);
    if (gmax <= 0) return DPCS_ERR_CUDA;
    const int64_t npix = (int64_t)a.Hc * a.Wc;
    const int64_t total[3] = {npix * a.spp, npix * p.edge_spp, p.edges ? p.nedges * p.sil_spp : 0};
    const int per_sm[3] = {kPoseGridInterior, kPoseGridEdges, kPoseGridSil};
    int g[3];
    for (int k = 0; k < 3; ++k) {
        const int64_t need = (total[k] + kPoseBlock - 1) / kPoseBlock;
        const int64_t cap = (int64_t)gmax / kPoseBlocksPerSM * per_sm[k];
        g[k] = (int)(need < cap ? need : cap);
    }
    int nl = 0;
    PoseArgs q = p;
    const bool pbr = p.mat != nullptr;
    if (g[0] > 0) {
        q.partial = p.partial;
        if (pbr)
            k_pose_interior<true><<<g[0], kPoseBlock, 0, st>>>(a, q);
        else
            k_pose_interior<false><<<g[0], kPoseBlock, 0, st>>>(a, q);
        ++nl;
    }
    if (g[1] > 0) {
        q.partial = p.partial + (size_t)gmax * 6;
        if (pbr)
            k_pose_edges<true><<<g[1], kPoseBlock, 0, st>>>(a, q);
        else
            k_pose_edges<false><<<g[1], kPoseBlock, 0, st>>>(a, q);
        ++nl;
    }
    if (g[2] > 0) {
        q.partial = p.partial + (size_t)2 * gmax * 6;
        if (pbr)
            k_pose_sil<true><<<g[2], kPoseBlock, 0, st>>>(a, q);
        else
            k_pose_sil<false><<<g[2], kPoseBlock, 0, st>>>(a, q);
        ++nl;
    }
    k_pose_reduce<<<1, 18 * 32, 0, st>>>(p.partial, gmax, g[0], g[1], g[2], wrench);
    return nl + 1;
}

}  // namespace dpcs
