// principled.cu -- the principled material of Sec. 3.2 on the GPU: the
// scene parameters m (a BRDF with a metallic map) and Vn (a normal map) on
// top of the Lambert + GGX path tracer, forward and path-replay adjoint.
//
// Material (Burley 2012's metallic workflow; the normal map in Mitsuba's
// convention, the paper's stated reference):
//   f_j = (1 - m) rho_j / pi + S F_j,  S = ks D G / (4 ci co),
//   F_j = F0_j + (1 - F0_j) (1 - wo.h)^5,  F0_j = (1 - m) f0 + m rho_j;
//   v = 2 Vn - 1 in the triangle's tangent frame (T = dp/du made orthogonal
//   to the geometric normal N, B = N x T), shading normal ns = v / |v|.
// ns replaces N in the BRDF, its sampling and pdf, cos_s of the NEE and
// cos_i of the continuation; N keeps the ray offsets, and light or
// continuations below the geometric surface are dropped.  metallic 0 and
// Vn = (0.5, 0.5, 1) give the plain material.
//
// Kernels: k_pack_mat interleaves (metallic, Vn) into one float4 per texel;
// k_render_pbr is k_render's loop (same thread mapping, same sample rounds,
// same xor-shuffle pixel sum) with this material; k_replay_pbr re-traces the
// paths, records each vertex and runs the reverse sweep with the material's
// derivatives (detached sampling: sampled directions and pdfs fixed);
// k_render_grad_pbr traces once for losses that act on each pixel alone (as
// k_render_grad does for the plain material): forward with records, the
// pixel's loss gradient through Eq. 5, then the sweeps; k_render_keep_pbr and
// k_sweep_kept_pbr keep the records in device memory for losses that couple
// pixels (the Eq. 11 filter), as k_render_keep / k_sweep_kept do;
// k_mat_backward adds the metallic and normal-map gradients to the caller's
// buffers.
#include <cuda_runtime.h>
#include <stdint.h>

#include "device.cuh"
#include "internal.h"
#include "principled.cuh"

namespace dpcs {

#ifndef DPCS_ALIGN_SHADOW
// 1: a vertex without projector light takes an empty shadow step, so the
// lanes of a warp trace extension rays and shadow rays in the same
// iterations (as in render.cu)
#define DPCS_ALIGN_SHADOW 1
#endif

namespace {

constexpr int kPBlock = 128;
#ifndef DPCS_YIELD_MIN
#define DPCS_YIELD_MIN 0  // as in render.cu: traversal does not yield
#endif
#ifndef DPCS_PBR_MINB
#define DPCS_PBR_MINB 8  // resident blocks per SM asked of ptxas (64 registers)
#endif

__device__ __forceinline__ void atomic_add4p(float4 *p, float4 v) { atomicAdd(p, v); }

// what the principled sweep needs of one vertex (52 words)
struct PRec {
    Bilin tb, pb;
    float beta[3], Ep[3], G;
    float rho[3], m;
    unsigned unc;  // bits 0-2: channel j not clipped; bit 3 / 4: the NEE / continuation BRDF is on
    float cw;
    float Sp, dSrp, s5p;
    f3 dSnp, wp_cs;
    float Si, dSri, s5i;
    f3 dSni, wi_ci;
    f3 T, B, N, ns;
    float inv_ulen;
};

// reverse sweep of one recorded path (the replay's recursion A_c = [lit]
// f(wp) Ep G + f(wi) cw A_{c+1}) with the principled derivatives:
//   d/d rho_j: (1 - m)/pi + S (1 - s5) m            (per lobe)
//   d/d m:     -rho_j/pi + S (1 - s5) (rho_j - f0)
//   d/d r:     dS/dr F_j
//   d/d ns:    ln_e (F_j dS/dn + f_j wp / cs) + cont (F_j dS/dn + f_j wi / ci),
// then ns = u / |u|, u = v_x T + v_y B + v_z N, v = 2 Vn - 1.
__device__ __forceinline__ void psweep(const RenderArgs &a, float4 *__restrict__ dmat, const PRec *rec, int nv,
                                       const float gb_in[3]) {
    float A[3] = {0.f, 0.f, 0.f};
    for (int c = nv - 1; c >= 0; --c) {
        const PRec &R = rec[c];
        float ga[3], dEp[3];
        float dr = 0.0f, dm = 0.0f;
        f3 gn = mk3(0.f, 0.f, 0.f);
        const float kdp = (R.unc & 8u) ? (1.0f - R.m) * DPCS_INV_PI_F : 0.0f;
        const float kdi = (R.unc & 16u) ? (1.0f - R.m) * DPCS_INV_PI_F : 0.0f;
        const float onp = (R.unc & 8u) ? 1.0f : 0.0f, oni = (R.unc & 16u) ? 1.0f : 0.0f;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float An = A[j];
            const float gb = gb_in[j] * R.beta[j];
            const bool lit = R.G > 0.0f && ((R.unc >> j) & 1u);
            const float ln_e = lit ? R.Ep[j] * R.G : 0.0f;
            const float cont = R.cw * An;
            const float Fp = pfresnel(R.rho[j], R.m, a.f0, R.s5p), Fi = pfresnel(R.rho[j], R.m, a.f0, R.s5i);
            const float fp = kdp * R.rho[j] + R.Sp * Fp, fi = kdi * R.rho[j] + R.Si * Fi;
            dEp[j] = lit ? gb * fp * R.G : 0.0f;
            ga[j] = gb * (ln_e * (kdp + R.Sp * (1.0f - R.s5p) * R.m) + cont * (kdi + R.Si * (1.0f - R.s5i) * R.m));
            dr += gb * (R.dSrp * Fp * ln_e + R.dSri * Fi * cont);
            dm += gb * (ln_e * (-onp * R.rho[j] * DPCS_INV_PI_F + R.Sp * (1.0f - R.s5p) * (R.rho[j] - a.f0)) +
                        cont * (-oni * R.rho[j] * DPCS_INV_PI_F + R.Si * (1.0f - R.s5i) * (R.rho[j] - a.f0)));
            gn = gn + (R.dSnp * Fp + R.wp_cs * fp) * (gb * ln_e) + (R.dSni * Fi + R.wi_ci * fi) * (gb * cont);
            A[j] = fp * ln_e + fi * cont;
        }
        int idx[4];
        float w[4];
        bilin_taps(R.tb, a.Wt, a.Ht, idx, w);
        if (a.dtex) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                atomic_add4p(a.dtex + idx[k], make_float4(ga[0] * w[k], ga[1] * w[k], ga[2] * w[k], dr * w[k]));
        }
        if (dmat) {
            f3 gv = mk3(0.f, 0.f, 0.f);
            if (R.inv_ulen > 0.0f) {
                const f3 gu = (gn - R.ns * dot(R.ns, gn)) * R.inv_ulen;
                gv = mk3(2.0f * dot(R.T, gu), 2.0f * dot(R.B, gu), 2.0f * dot(R.N, gu));
            }
#pragma unroll
            for (int k = 0; k < 4; ++k)
                atomic_add4p(dmat + idx[k], make_float4(dm * w[k], gv.x * w[k], gv.y * w[k], gv.z * w[k]));
        }
        if (R.G > 0.0f && (dEp[0] != 0.0f || dEp[1] != 0.0f || dEp[2] != 0.0f)) {
            bilin_taps(R.pb, a.Wp, a.Hp, idx, w);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                atomic_add4p(a.dEp + idx[k], make_float4(dEp[0] * w[k], dEp[1] * w[k], dEp[2] * w[k], 0.0f));
        }
    }
}

__device__ __forceinline__ void prec_vertex(PRec &R, const PSurf &S, f3 beta) {
    R.tb = S.tb;
    R.pb.x0 = R.pb.y0 = 0;
    R.pb.fx = R.pb.fy = 0.0f;
    R.beta[0] = beta.x; R.beta[1] = beta.y; R.beta[2] = beta.z;
    R.Ep[0] = R.Ep[1] = R.Ep[2] = 0.0f;
    R.G = 0.0f;
    R.rho[0] = S.rho.x; R.rho[1] = S.rho.y; R.rho[2] = S.rho.z;
    R.m = S.m;
    R.unc = 0u;
    R.cw = 0.0f;
    R.Sp = R.dSrp = R.s5p = R.Si = R.dSri = R.s5i = 0.0f;
    R.dSnp = R.wp_cs = R.dSni = R.wi_ci = mk3(0.f, 0.f, 0.f);
    R.T = S.T;
    R.B = S.B;
    R.N = S.n;
    R.ns = S.ns;
    R.inv_ulen = S.inv_ulen;
}

// NV floats summed over the block into FP64 accumulators
template <int NV>
__device__ __forceinline__ void pblock_reduce_add(float (&v)[NV], double *acc) {
    __shared__ float red[NV][kPBlock / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int off = 16; off; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) red[k][w] = v[k];
    __syncthreads();
    if (threadIdx.x < NV) {
        float s = 0.0f;
        for (int j = 0; j < (int)(blockDim.x >> 5); ++j) s += red[threadIdx.x][j];
        if (s != 0.0f) atomicAdd(acc + threadIdx.x, (double)s);
    }
}

__device__ __forceinline__ float pcrf(float ec, float gain, float wb, float gamma) {
    const float v = gain * wb * ec;
    return v > 0.0f ? powf(v, gamma) : 0.0f;
}

// One warp-synchronous pass over a lane's samples, as k_render and k_replay
// run them: each iteration traces one ray (extension or shadow) per lane,
// and the warp starts its next samples together.  kMode 0: sum the lit
// contributions and write Ec / Ic; 1: record the vertices and sweep each
// path with the pixel's dLoss/dEc from a.gE; 2: record the vertices of up to
// kFusedSamples samples, then form the pixel's loss gradient (loss l) and
// sweep them all; 3: as 0, and store every vertex record to the kept buffer
// (kchunks, 16-byte chunks laid out as the plain kept records, kernel
// k_sweep_kept_pbr) and each sample's vertex count to knvs.
constexpr int kModeRender = 0, kModeReplay = 1, kModeFused = 2, kModeKeep = 3;
template <int kMode>
__device__ __forceinline__ void pbr_lanes(const RenderArgs &a, const float4 *__restrict__ mat,
                                          float4 *__restrict__ dmat, int64_t pix, int sl, bool valid,
                                          const LossArgs *l, uint4 *__restrict__ kchunks = nullptr,
                                          uint8_t *__restrict__ knvs = nullptr) {
    constexpr bool kReplay = kMode != kModeRender;  // vertices are recorded
    constexpr int kPChunks = (int)(sizeof(PRec) / 16);
    constexpr int kGChunk = (int)(offsetof(PRec, G) / 16), kGWord = (int)(offsetof(PRec, G) % 16) / 4;
    const int L = 1 << a.log2L;
    Cnt cnt;
    f3 sum = mk3(0.f, 0.f, 0.f);
    float gb_in[3] = {0.f, 0.f, 0.f};
    bool any = true;
    int k = 0;  // samples this lane has finished (kModeFused)
    int nvs[kMode == kModeFused ? kFusedSamples : 1];
    if (kMode == kModeReplay) {
        const float inv = 1.0f / (float)a.spp;
        if (valid) {
            gb_in[0] = a.gE[3 * pix] * inv;
            gb_in[1] = a.gE[3 * pix + 1] * inv;
            gb_in[2] = a.gE[3 * pix + 2] * inv;
        }
        any = gb_in[0] != 0.0f || gb_in[1] != 0.0f || gb_in[2] != 0.0f;
    }
    int s = (valid && any) ? sl : a.spp;
    int b = 1, nv = 0;
    bool shadow = false, has_ext = false, pending = false, nulls = false;
    f3 beta = mk3(0.f, 0.f, 0.f), c = beta, ed = beta;
    Ray ray;
    ray.o = ray.d = ray.inv = beta;
    float tmax = INFINITY;
    Trav st;
    int stack[kStack];
    PRec rec[(kMode == kModeRender || kMode == kModeKeep) ? 1
                                                           : (kMode == kModeReplay ? DPCS_MAX_BOUNCES : kFusedRecs)];
    const int64_t nthr = ((int64_t)a.Hc * a.Wc) << a.log2L, gt = (pix << a.log2L) + sl;  // kModeKeep
    const int spl = (a.spp + L - 1) / L;
    if (s < a.spp && a.bounces > 0) {
        f3 o, d;
        camera_ray(a, (uint32_t)pix, (uint32_t)s, o, d);
        ray = make_ray(o, d);
        beta = mk3(1.f, 1.f, 1.f);
        cnt.add(kCntPath);
    } else {
        s = a.spp;
    }
    const int64_t max_iter = ((int64_t)(a.spp / L + 1) * (2 * a.bounces + 1)) * (2 * (int64_t)a.T + 18);
    int64_t iter = 0;
    while (s < a.spp) {
        // this sample's records (the host keeps k < kFusedSamples and k * bounces + nv < kFusedRecs)
        PRec *rs = rec + (kMode == kModeFused ? min(k, kFusedSamples - 1) * a.bounces : 0);
        while (true) {
            if (++iter > max_iter) {
                atomicOr(a.status, kStatusTraversalLimit);
                s = a.spp;
                nv = 0;
                break;
            }
            if (!pending) {
                if (!nulls) cnt.add(shadow ? kCntShadow : kCntRay);
                trav_begin(st, a.root, shadow ? tmax : INFINITY, shadow);
                pending = true;
            }
            // the min_active argument in the form render.cu's kernels pass it:
            // there a literal 0 (the same value) cost a 3.2x slowdown
            const int alive = DPCS_YIELD_MIN > 0 ? __popc(__activemask()) : 0;
            if (!trav_resume(a.nodes, a.tris, nulls ? kEmptyRoot : a.root, a.T, ray, st, stack, a.status, cnt,
                             min(DPCS_YIELD_MIN, alive), a.visit_cap))
                continue;
            pending = false;
            const bool hit = st.h.pos >= 0;
            bool end = false;
            if (shadow) {
                if (hit) {
                    if (kMode == kModeKeep) {  // occluded: clear G of the stored record
                        if (valid)
                            __stcs(reinterpret_cast<unsigned *>(kchunks + kept_chunk(kGChunk, k, nv - 1, spl, a.bounces,
                                                                                     nthr, gt)) + kGWord, 0u);
                    } else if (kReplay) {
                        rs[nv - 1].G = 0.0f;  // occluded
                    }
                } else if (!nulls) {
                    if (kMode != kModeReplay) sum = sum + c;
                    cnt.add(kCntLit);
                }
                shadow = false;
                nulls = false;
                if (has_ext) {
                    ray = make_ray(ray.o, ed);
                    ++b;
                } else {
                    end = true;
                }
            } else if (!hit) {
                end = true;
            } else {
                cnt.add(kCntVert);
                const PSurf S = psurface_at(a, mat, st.h, ray.d);
                PRec *R = kReplay ? &rs[kMode == kModeKeep ? 0 : nv] : nullptr;
                if (kReplay) ++nv;
                if (kReplay) prec_vertex(*R, S, beta);
                PNee N;
                const bool cand = pnee_prepare(a, S, N);
                if (cand) {
                    c = beta * N.fp * mk3(N.ep.x, N.ep.y, N.ep.z) * N.G;
                    unsigned unc = 7u;
                    if (a.clip > 0.0f) {
                        if (c.x > a.clip) { c.x = a.clip; unc &= ~1u; }
                        if (c.y > a.clip) { c.y = a.clip; unc &= ~2u; }
                        if (c.z > a.clip) { c.z = a.clip; unc &= ~4u; }
                    }
                    if (kReplay) {
                        R->pb = N.pb;
                        R->Ep[0] = N.ep.x; R->Ep[1] = N.ep.y; R->Ep[2] = N.ep.z;
                        R->G = N.G;
                        R->unc = unc | (N.L.on > 0.0f ? 8u : 0u);
                        R->Sp = N.L.S; R->dSrp = N.L.dSr; R->s5p = N.L.s5; R->dSnp = N.L.dSn;
                        R->wp_cs = N.wp_cs;
                    }
                }
                has_ext = false;
                if (b < a.bounces) {
                    PCont C;
                    if (pcontinue_prepare(a, (uint32_t)pix, (uint32_t)s, b, S, C)) {
                        cnt.add(kCntCont);
                        beta = beta * C.w;
                        ed = C.wi;
                        has_ext = true;
                        if (kReplay) {
                            R->cw = C.cw;
                            R->unc |= C.L.on > 0.0f ? 16u : 0u;
                            R->Si = C.L.S; R->dSri = C.L.dSr; R->s5i = C.L.s5; R->dSni = C.L.dSn;
                            R->wi_ci = C.wi_ci;
                        }
                    }
                }
                if (kMode == kModeKeep && valid) {  // the record, complete but for a later occlusion
                    const uint4 *src = reinterpret_cast<const uint4 *>(R);
#pragma unroll
                    for (int q = 0; q < kPChunks; ++q)
                        __stcs(kchunks + kept_chunk(q, k, nv - 1, spl, a.bounces, nthr, gt), src[q]);
                }
                if (cand) {
                    shadow = true;
                    ray = make_ray(N.so, N.sdir);
                    tmax = N.smax;
                } else if (has_ext) {
#if DPCS_ALIGN_SHADOW
                    // no projector light here: an empty shadow step (no
                    // traversal) keeps the lane in phase with the others
                    shadow = true;
                    nulls = true;
                    ray.o = S.x + S.n * kRayEps;
#else
                    ray = make_ray(S.x + S.n * kRayEps, ed);
                    ++b;
#endif
                } else {
                    end = true;
                }
            }
            if (end) break;
        }
        if (kMode == kModeKeep && valid) knvs[(int64_t)k * nthr + gt] = (uint8_t)nv;
        if (kMode == kModeReplay) psweep(a, dmat, rec, nv, gb_in);
        if (kMode == kModeFused) nvs[k < kFusedSamples ? k : kFusedSamples - 1] = nv;
        ++k;
        nv = 0;
        s += L;
        if (s < a.spp) {
            f3 o, d;
            camera_ray(a, (uint32_t)pix, (uint32_t)s, o, d);
            ray = make_ray(o, d);
            beta = mk3(1.f, 1.f, 1.f);
            b = 1;
            shadow = false;
            nulls = false;
            has_ext = false;
            cnt.add(kCntPath);
        }
    }
    cnt.flush(a.counters);
    if (kMode == kModeFused) {
        // every lane of a pixel ends with the pixel's sum (the tree below)
        for (int off = L >> 1; off > 0; off >>= 1) {
            sum.x += __shfl_xor_sync(0xffffffffu, sum.x, off);
            sum.y += __shfl_xor_sync(0xffffffffu, sum.y, off);
            sum.z += __shfl_xor_sync(0xffffffffu, sum.z, off);
        }
        const float inv = 1.0f / (float)a.spp;
        const float ec[3] = {sum.x * inv, sum.y * inv, sum.z * inv};
        float v[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // gamma_c(3), Gc, wb(3), loss
        if (valid) {
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float ic = pcrf(ec[j], a.gain_c, a.wb[j], a.gamma_c[j]);
                if (sl == 0) {
                    if (a.Ec) a.Ec[3 * pix + j] = ec[j];
                    a.Ic[3 * pix + j] = ic;
                }
                const float d = ic - l->target[3 * pix + j];
                const float g = l->kind == 0 ? l->scale * d : (d > 0.0f ? l->scale : (d < 0.0f ? -l->scale : 0.0f));
                const float w = a.gain_c * a.wb[j] * ec[j];
                if (w > 0.0f) {
                    const float da = a.gamma_c[j] * powf(w, a.gamma_c[j] - 1.0f);
                    gb_in[j] = g * da * a.gain_c * a.wb[j] * inv;
                    if (sl == 0) {
                        v[j] += g * ic * logf(w);
                        v[3] += g * da * a.wb[j] * ec[j];
                        v[4 + j] += g * da * a.gain_c * ec[j];
                    }
                }
                if (sl == 0) v[7] += l->kind == 0 ? 0.5f * l->scale * d * d : l->scale * fabsf(d);
            }
        }
        pblock_reduce_add<8>(v, l->acc + 4);  // acc[4..10]: gamma_c, Gc, wb; acc[11]: the loss
        if (gb_in[0] != 0.0f || gb_in[1] != 0.0f || gb_in[2] != 0.0f)
            for (int i = 0; i < k && i < kFusedSamples; ++i) psweep(a, dmat, rec + i * a.bounces, nvs[i], gb_in);
    }
    if (kMode == kModeRender || kMode == kModeKeep) {
        for (int off = L >> 1; off > 0; off >>= 1) {
            sum.x += __shfl_xor_sync(0xffffffffu, sum.x, off);
            sum.y += __shfl_xor_sync(0xffffffffu, sum.y, off);
            sum.z += __shfl_xor_sync(0xffffffffu, sum.z, off);
        }
        if (valid && sl == 0) {
            const float inv = 1.0f / (float)a.spp;
            const float ex = sum.x * inv, ey = sum.y * inv, ez = sum.z * inv;
            if (a.Ec) {
                a.Ec[3 * pix] = ex;
                a.Ec[3 * pix + 1] = ey;
                a.Ec[3 * pix + 2] = ez;
            }
            const float e3[3] = {ex, ey, ez};
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float v = a.gain_c * a.wb[j] * e3[j];
                a.Ic[3 * pix + j] = v > 0.0f ? powf(v, a.gamma_c[j]) : 0.0f;
            }
        }
    }
}

__global__ void __launch_bounds__(kPBlock, DPCS_PBR_MINB) k_render_pbr(const RenderArgs a, const float4 *__restrict__ mat) {
    const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t pix = gt >> a.log2L;
    pbr_lanes<kModeRender>(a, mat, nullptr, pix, (int)(gt & ((1 << a.log2L) - 1)), pix < (int64_t)a.Hc * a.Wc,
                           nullptr);
}

// render + per-pixel loss + adjoint in one trace; the host calls it only
// when ceil(spp / L) <= kFusedSamples and ceil(spp / L) * bounces <= kFusedRecs
__global__ void __launch_bounds__(kPBlock, DPCS_PBR_MINB)
    k_render_grad_pbr(const RenderArgs a, const float4 *__restrict__ mat, float4 *__restrict__ dmat,
                      const LossArgs l) {
    const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t pix = gt >> a.log2L;
    pbr_lanes<kModeFused>(a, mat, dmat, pix, (int)(gt & ((1 << a.log2L) - 1)), pix < (int64_t)a.Hc * a.Wc, &l);
}

__global__ void __launch_bounds__(kPBlock, DPCS_PBR_MINB) k_replay_pbr(const RenderArgs a, const float4 *__restrict__ mat,
                                                        float4 *__restrict__ dmat) {
    const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t pix = gt >> a.log2L;
    pbr_lanes<kModeReplay>(a, mat, dmat, pix, (int)(gt & ((1 << a.log2L) - 1)), pix < (int64_t)a.Hc * a.Wc,
                           nullptr);
}

// the render of k_render_pbr, keeping every vertex record for k_sweep_kept_pbr
__global__ void __launch_bounds__(kPBlock, DPCS_PBR_MINB)
    k_render_keep_pbr(const RenderArgs a, const float4 *__restrict__ mat, uint4 *__restrict__ chunks,
                      uint8_t *__restrict__ nvs) {
    const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t pix = gt >> a.log2L;
    pbr_lanes<kModeKeep>(a, mat, nullptr, pix, (int)(gt & ((1 << a.log2L) - 1)), pix < (int64_t)a.Hc * a.Wc,
                         nullptr, chunks, nvs);
}

// the principled adjoint from the kept records: the sweeps of k_replay_pbr
// without tracing again
__global__ void __launch_bounds__(kPBlock) k_sweep_kept_pbr(const RenderArgs a, const uint4 *__restrict__ chunks,
                                                            const uint8_t *__restrict__ nvs, float4 *__restrict__ dmat) {
    constexpr int kPChunks = (int)(sizeof(PRec) / 16);
    const int L = 1 << a.log2L;
    const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t pix = gt >> a.log2L;
    const int64_t nthr = ((int64_t)a.Hc * a.Wc) << a.log2L;
    if (pix >= (int64_t)a.Hc * a.Wc) return;
    const float inv = 1.0f / (float)a.spp;
    const float gb_in[3] = {a.gE[3 * pix] * inv, a.gE[3 * pix + 1] * inv, a.gE[3 * pix + 2] * inv};
    if (gb_in[0] == 0.0f && gb_in[1] == 0.0f && gb_in[2] == 0.0f) return;
    const int sl = (int)(gt & (L - 1));
    const int spl = (a.spp + L - 1) / L;
    PRec rec[DPCS_MAX_BOUNCES];
    for (int k = 0; k < spl && sl + k * L < a.spp; ++k) {
        const int nv = nvs[(int64_t)k * nthr + gt];
        for (int v = 0; v < nv; ++v) {
            uint4 *dst = reinterpret_cast<uint4 *>(&rec[v]);
#pragma unroll
            for (int q = 0; q < kPChunks; ++q) dst[q] = __ldcs(chunks + kept_chunk(q, k, v, spl, a.bounces, nthr, gt));
        }
        psweep(a, dmat, rec, nv, gb_in);
    }
}

__global__ void k_pack_mat(const float *__restrict__ metallic, const float *__restrict__ normal, int64_t ntex,
                           float4 *__restrict__ mat) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= ntex) return;
    mat[t] = make_float4(metallic ? metallic[t] : 0.0f, normal ? normal[3 * t] : 0.5f, normal ? normal[3 * t + 1] : 0.5f,
                         normal ? normal[3 * t + 2] : 1.0f);
}

__global__ void k_mat_backward(const float4 *__restrict__ dmat, int64_t ntex, float *__restrict__ dMetallic,
                               float *__restrict__ dNormal) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= ntex) return;
    const float4 g = dmat[t];
    if (dMetallic) dMetallic[t] += g.x;
    if (dNormal) {
        dNormal[3 * t] += g.y;
        dNormal[3 * t + 1] += g.z;
        dNormal[3 * t + 2] += g.w;
    }
}

inline unsigned grid1(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

}  // namespace

int launch_pack_mat(const float *metallic, const float *normal, int64_t ntex, float4 *mat, cudaStream_t st) {
    if (ntex <= 0) return 0;
    k_pack_mat<<<grid1(ntex, 256), 256, 0, st>>>(metallic, normal, ntex, mat);
    return 1;
}

int launch_render_pbr(const RenderArgs &a, const float4 *mat, cudaStream_t st) {
    const int64_t threads = ((int64_t)a.Hc * a.Wc) << a.log2L;
    if (threads <= 0) return 0;
    k_render_pbr<<<grid1(threads, kPBlock), kPBlock, 0, st>>>(a, mat);
    return 1;
}

int launch_replay_pbr(const RenderArgs &a, const float4 *mat, float4 *dmat, cudaStream_t st) {
    const int64_t threads = ((int64_t)a.Hc * a.Wc) << a.log2L;
    if (threads <= 0) return 0;
    k_replay_pbr<<<grid1(threads, kPBlock), kPBlock, 0, st>>>(a, mat, dmat);
    return 1;
}

int launch_render_grad_pbr(const RenderArgs &a, const float4 *mat, float4 *dmat, const LossArgs &l,
                           cudaStream_t st) {
    const int64_t threads = ((int64_t)a.Hc * a.Wc) << a.log2L;
    if (threads <= 0) return 0;
    k_render_grad_pbr<<<grid1(threads, kPBlock), kPBlock, 0, st>>>(a, mat, dmat, l);
    return 1;
}

static_assert(sizeof(PRec) == 4 * kPRecWordsHost, "the host sizes kept principled records with kPRecWordsHost");
static_assert(sizeof(PRec) % 16 == 0, "PRec must be whole 16-byte chunks");

int launch_render_keep_pbr(const RenderArgs &a, const float4 *mat, void *chunks, uint8_t *nvs, cudaStream_t st) {
    const int64_t threads = ((int64_t)a.Hc * a.Wc) << a.log2L;
    if (threads <= 0) return 0;
    k_render_keep_pbr<<<grid1(threads, kPBlock), kPBlock, 0, st>>>(a, mat, (uint4 *)chunks, nvs);
    return 1;
}

int launch_sweep_kept_pbr(const RenderArgs &a, const void *chunks, const uint8_t *nvs, float4 *dmat, cudaStream_t st) {
    const int64_t threads = ((int64_t)a.Hc * a.Wc) << a.log2L;
    if (threads <= 0) return 0;
    k_sweep_kept_pbr<<<grid1(threads, kPBlock), kPBlock, 0, st>>>(a, (const uint4 *)chunks, nvs, dmat);
    return 1;
}

int launch_mat_backward(const float4 *dmat, int64_t ntex, float *dMetallic, float *dNormal, cudaStream_t st) {
    if (ntex <= 0 || (!dMetallic && !dNormal)) return 0;
    k_mat_backward<<<grid1(ntex, 256), 256, 0, st>>>(dmat, ntex, dMetallic, dNormal);
    return 1;
}

}  // namespace dpcs
