// render.cu -- forward rendering and its path-replay adjoint.
//
// Forward (Eq. 7): k_prf maps the projector image through the PRF (Eq. 1),
// k_pack_tex interleaves albedo and roughness into one float4 per texel, and
// k_render traces every camera path (Eqs. 3, 6, 10) and applies the camera
// response (Eqs. 4, 5) in its epilogue.
//
// Adjoint: k_crf_backward turns dLoss/dIc into dLoss/dEc (Eq. 5), k_replay
// re-traces each path from its Philox counters and scatters gradients into
// the projector and texture accumulators, k_prf_backward applies Eq. 1's
// derivative, and k_tex_backward / k_finalize add the results to the
// caller's buffers.
//
// Thread mapping: L = 2^log2L consecutive lanes of a warp share one camera
// pixel; lane l traces samples l, l+L, l+2L, ... and the L partial sums are
// combined by a fixed xor-shuffle tree, so a pixel's result does not depend
// on scheduling.
#include <cuda_runtime.h>
#include <stdint.h>

#include "device.cuh"
#include "internal.h"

namespace dpcs {

namespace {

constexpr int kRenderBlock = 128;
#ifndef DPCS_YIELD_MIN
// Traversal yields when fewer lanes of the warp are still traversing.  Off
// (0): on GB300 yielding at 8..24 lanes cost 1.6-2x more than it recovered.
#define DPCS_YIELD_MIN 0
#endif
#ifndef DPCS_BATCH_MINB
#define DPCS_BATCH_MINB 8  // resident blocks per SM for the batched render: it reads its arguments from shared memory and needs the registers
#endif
#ifndef DPCS_ALIGN_SHADOW
// 1: a vertex without projector light takes an empty shadow step, so the
// lanes of a warp trace extension rays and shadow rays in the same
// iterations and shade together; 0: it goes straight to its extension ray
#define DPCS_ALIGN_SHADOW 1
#endif
#ifndef DPCS_RENDER_MINB
// minimum resident blocks per SM requested from ptxas for k_render: 8 (64
// registers) against 10 (48 registers, with spills) measured 2 % faster on
// the corner and 2 % slower on the 200k-triangle heightfield
#define DPCS_RENDER_MINB 8
#endif
#ifndef DPCS_GRAD_MINB
// the same for the kernels that keep vertex records (replay, fused step,
// kept records): 8 blocks (64 registers) measured 3-5 % faster than 10
#define DPCS_GRAD_MINB 8
#endif

__device__ __forceinline__ void atomic_add4(float4 *p, float4 v) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
    atomicAdd(p, v);
#else
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
    atomicAdd(&p->z, v.z);
    atomicAdd(&p->w, v.w);
#endif
}

#ifndef DPCS_WARP_PREREDUCE
// Combine same-texel gradient scatters of a warp before the atomic.  Off: on
// GB300 the vote and warp syncs inside the divergent sweep cost more (replay
// +14 % at 16 spp, +23 % at 64 spp) than the float4 atomics they save (the
// atomics take 5-7 % of the replay).
#define DPCS_WARP_PREREDUCE 0
#endif

// Gradient scatter with warp pre-reduction: when every lane taking part adds
// to the same texel (typical at a pixel's first vertex, where the L lanes of
// the pixel hit nearly the same point), the lanes sum their values through a
// per-warp shared-memory row and one lane issues the float4 atomic;
// otherwise each lane adds its own value.  `row` is this warp's 32 float4.
__device__ __forceinline__ void scatter_add4(float4 *base, int key, float4 v, float4 *row) {
#if DPCS_WARP_PREREDUCE
    const unsigned active = __activemask();
    int same = 0;
    __match_all_sync(active, key, &same);
    if (same && (active & (active - 1u)) != 0u) {
        const int lane = threadIdx.x & 31;
        row[lane] = v;
        __syncwarp(active);
        if (lane == __ffs(active) - 1) {
            float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
            for (unsigned m = active; m; m &= m - 1u) {
                const float4 o = row[__ffs(m) - 1];
                t.x += o.x;
                t.y += o.y;
                t.z += o.z;
                t.w += o.w;
            }
            atomic_add4(base + key, t);
        }
        __syncwarp(active);  // the row is reused by the next scatter
        return;
    }
#else
    (void)row;
#endif
    atomic_add4(base + key, v);
}

__global__ void k_prf(const float *__restrict__ Ip, int64_t ntex, float g0, float g1, float g2, float gain,
                      float4 *__restrict__ Ep) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= ntex) return;
    const float a = Ip[3 * t], b = Ip[3 * t + 1], c = Ip[3 * t + 2];
    Ep[t] = make_float4(a > 0.0f ? gain * powf(a, g0) : 0.0f, b > 0.0f ? gain * powf(b, g1) : 0.0f,
                        c > 0.0f ? gain * powf(c, g2) : 0.0f, 0.0f);
}

__global__ void k_pack_tex(const float *__restrict__ albedo, const float *__restrict__ rough, int64_t ntex,
                           float4 *__restrict__ tex) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= ntex) return;
    tex[t] = make_float4(albedo[3 * t], albedo[3 * t + 1], albedo[3 * t + 2], rough[t]);
}

__device__ __forceinline__ float crf(float ec, float gain, float wb, float gamma) {
    const float a = gain * wb * ec;
    return a > 0.0f ? powf(a, gamma) : 0.0f;
}

// Forward megakernel.  Every loop iteration traces exactly one ray per lane --
// the extension ray of the current vertex or its shadow ray towards the
// projector -- through the same traversal loop, then advances that lane's
// path.  A lane whose path ends leaves the inner loop and waits there until
// every path of the warp has ended; then the warp starts its next samples
// together.  Starting a lane's next camera ray while the others are deep in
// their paths (path regeneration) was measured 20-28 % slower: the mixed
// warp loses the coherence of its first bounces.  Each lane adds its lit
// vertices' contributions to its pixel sum in sample-then-vertex order; the
// per-vertex arithmetic (surface_at, nee_prepare, continue_prepare) is
// shared with k_replay.
//
// The L lanes (L = 2^log2L, a divisor of 32) that share camera pixel `pix`:
// lane `sl` traces samples sl, sl+L, ...; the lanes then combine their sums
// and lane 0 writes Ec and Ic.  Every lane of the warp must call this (the
// reduction shuffles over the full warp); lanes with valid == false only
// take part in the shuffles.
__device__ __forceinline__ void render_lanes(const RenderArgs &a, int64_t pix, int sl, bool valid) {
    const int L = 1 << a.log2L;
    f3 sum = mk3(0.f, 0.f, 0.f);
    Cnt cnt;
    int s = valid ? sl : a.spp;
    int b = 1;
    bool shadow = false, has_ext = false, pending = false, nulls = false;
    // throughput, pending NEE contribution, extension direction; each lit
    // vertex's contribution goes straight into the lane's pixel sum
    f3 beta = mk3(0.f, 0.f, 0.f), c = beta, ed = beta;
    Ray ray;
    ray.o = ray.d = ray.inv = beta;
    float tmax = INFINITY;
    Trav st;
    int stack[kStack];
    if (s < a.spp && a.bounces > 0) {
        f3 o, d;
        camera_ray(a, (uint32_t)pix, (uint32_t)s, o, d);
        ray = make_ray(o, d);
        beta = mk3(1.f, 1.f, 1.f);
        cnt.add(kCntPath);
    } else {
        s = a.spp;
    }
    // defensive bound on loop iterations: every iteration either advances a
    // traversal by at least one node or consumes a finished ray
    const int64_t max_iter = ((int64_t)(a.spp / L + 1) * (2 * a.bounces + 1)) * (2 * (int64_t)a.T + 18);
    int64_t iter = 0;
    while (s < a.spp) {
        while (true) {  // the lane's current path; the warp starts its next samples together
            if (++iter > max_iter) {
                atomicOr(a.status, kStatusTraversalLimit);
                s = a.spp;
                break;
            }
            cnt.add_warp(kCntPathWarpIter);
            // yield only while some live lane of the warp could take a new ray
            const int alive = DPCS_YIELD_MIN > 0 ? __popc(__activemask()) : 0;
            if (!pending) {
                if (!nulls) cnt.add(shadow ? kCntShadow : kCntRay);
                trav_begin(st, a.root, shadow ? tmax : INFINITY, shadow);
                pending = true;
            }
            if (!trav_resume(a.nodes, a.tris, nulls ? kEmptyRoot : a.root, a.T, ray, st, stack, a.status, cnt, min(DPCS_YIELD_MIN, alive), a.visit_cap))
                continue;
            pending = false;
            const bool hit = st.h.pos >= 0;
            bool end = false;
            if (shadow) {
                if (!hit && !nulls) {
                    sum = sum + c;
                    cnt.add(kCntLit);
                }
                shadow = false;
                nulls = false;
                if (has_ext) {  // the extension ray starts where the shadow ray did (x + n eps)
                    ray = make_ray(ray.o, ed);
                    ++b;
                } else {
                    end = true;
                }
            } else if (!hit) {
                end = true;
            } else {
                cnt.add(kCntVert);
                const Surf S = surface_at(a, st.h, ray.d);
                Nee N;
                const bool cand = nee_prepare(a, S, N);
                if (cand) {
                    unsigned unc;
                    c = nee_contrib(a, beta, N, unc);
                }
                has_ext = false;
                if (b < a.bounces) {
                    Cont C;
                    if (continue_prepare(a, (uint32_t)pix, (uint32_t)s, b, S, C)) {
                        cnt.add(kCntCont);
                        beta = beta * C.w;
                        ed = C.wi;
                        has_ext = true;
                    }
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
        a.Ic[3 * pix] = crf(ex, a.gain_c, a.wb[0], a.gamma_c[0]);
        a.Ic[3 * pix + 1] = crf(ey, a.gain_c, a.wb[1], a.gamma_c[1]);
        a.Ic[3 * pix + 2] = crf(ez, a.gain_c, a.wb[2], a.gamma_c[2]);
    }
}

__global__ void __launch_bounds__(kRenderBlock, DPCS_RENDER_MINB) k_render(const RenderArgs a) {
    const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t pix = gt >> a.log2L;
    render_lanes(a, pix, (int)(gt & ((1 << a.log2L) - 1)), pix < (int64_t)a.Hc * a.Wc);
}

// Batched persistent render: CTAs pull virtual blocks from a device counter;
// virtual block vb belongs to the segment whose range [vb_begin, vb_begin +
// ceil(npix L / 128)) holds it, and covers that segment's pixels from
// pix_begin on.  A segment is a pixel range of one request whose arguments
// are descs[slot].  Per pixel the computation is render_lanes, exactly as in
// k_render.  The loop ends when the counter passes the last virtual block:
// there is no waiting on other CTAs.
__global__ void __launch_bounds__(kRenderBlock, DPCS_BATCH_MINB)
    k_render_batch(const RenderArgs *__restrict__ descs, const BatchSeg *__restrict__ segs, int nseg,
                   int64_t total_vb, unsigned long long *counter) {
    __shared__ RenderArgs sa;
    __shared__ int64_t s_vb;
    __shared__ int s_seg;
    while (true) {
        if (threadIdx.x == 0) {
            const int64_t vb = (int64_t)atomicAdd(counter, 1ull);
            int lo = 0, hi = nseg - 1;  // last segment with vb_begin <= vb
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (segs[mid].vb_begin <= vb) lo = mid; else hi = mid - 1;
            }
            s_vb = vb;
            s_seg = lo;
        }
        __syncthreads();
        const int64_t vb = s_vb;
        if (vb >= total_vb) break;
        const BatchSeg sg = segs[s_seg];
        {
            const int *src = reinterpret_cast<const int *>(descs + sg.slot);
            int *dst = reinterpret_cast<int *>(&sa);
            for (int i = threadIdx.x; i < (int)(sizeof(RenderArgs) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
        }
        __syncthreads();
        const int64_t lt = (vb - sg.vb_begin) * kRenderBlock + threadIdx.x;  // thread index within the segment
        const int64_t lp = lt >> sa.log2L;
        render_lanes(sa, sg.pix_begin + lp, (int)(lt & ((1 << sa.log2L) - 1)), lp < sg.npix);
        __syncthreads();
    }
}

__global__ void k_trace(const float4 *__restrict__ nodes, const float4 *__restrict__ tris, int32_t root, int32_t T,
                        const float *__restrict__ o, const float *__restrict__ d, int64_t n, float *__restrict__ tout,
                        int32_t *__restrict__ triout, unsigned *status) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    Hit h;
    Cnt cnt;
    const Ray r = make_ray(mk3(o[3 * i], o[3 * i + 1], o[3 * i + 2]), mk3(d[3 * i], d[3 * i + 1], d[3 * i + 2]));
    const bool hit = traverse(nodes, tris, root, T, r, INFINITY, false, h, status, cnt);
    tout[i] = hit ? h.t : INFINITY;
    triout[i] = hit ? h.orig : -1;
}

// ---------------------------------------------------------------------------
// block reduction of NV floats into FP64 accumulators
// ---------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_reduce_add(float (&v)[NV], double *acc) {
    __shared__ float red[NV][32];
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

// Eq. 5 adjoint.  acc layout: [gamma_p(3), Gp, gamma_c(3), Gc, wb(3)]
__global__ void k_crf_backward(const float *__restrict__ dIc, const float *__restrict__ Ec,
                               const float *__restrict__ Ic, int64_t npix, float gc0, float gc1, float gc2,
                               float gain, float w0, float w1, float w2, float *__restrict__ gE, double *acc) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float v[7] = {0, 0, 0, 0, 0, 0, 0};  // gamma_c(3), Gc, wb(3)
    if (p < npix) {
        const float gcs[3] = {gc0, gc1, gc2}, wbs[3] = {w0, w1, w2};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float ec = Ec[3 * p + j];
            const float a = gain * wbs[j] * ec;
            float ge = 0.0f;
            if (a > 0.0f) {
                const float g = dIc[3 * p + j];
                const float da = gcs[j] * powf(a, gcs[j] - 1.0f);
                ge = g * da * gain * wbs[j];
                v[j] += g * Ic[3 * p + j] * logf(a);
                v[3] += g * da * wbs[j] * ec;
                v[4 + j] += g * da * gain * ec;
            }
            gE[3 * p + j] = ge;
        }
    }
    block_reduce_add<7>(v, acc + 4);
}

// reverse sweep over the recorded vertices of one path: with A the
// derivative of the path radiance with respect to the throughput entering
// the next vertex (A_c = [lit] f(wp) Ep G + f(wi) cw A_{c+1}), scatter
// dLoss/dEp, dLoss/dalbedo and dLoss/droughness into the accumulators:
// packed float4 atomics, or (F64) one FP64 atomic per component, whose sums
// do not depend on the order of the adds beyond FP64 rounding.
template <bool F64>
__device__ __forceinline__ void replay_sweep(const RenderArgs &a, const VRec *rec, int nv, const float gb_in[3],
                                             float4 *row) {
    float A[3] = {0.f, 0.f, 0.f};
    for (int c = nv - 1; c >= 0; --c) {
        const VRec &R = rec[c];
        float ga[3], dEp[3];
        float dr = 0.0f;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float An = A[j];
            const float gb = gb_in[j] * R.beta[j];
            const bool lit = R.G > 0.0f && ((R.unc >> j) & 1u);
            const float ln_e = lit ? R.Ep[j] * R.G : 0.0f;  // radiance / f along wp
            const float cont = R.cw * An;                  // w / f times downstream A
            const float fp = R.rho[j] * DPCS_INV_PI_F + R.sp;
            const float fi = R.rho[j] * DPCS_INV_PI_F + R.si;
            dEp[j] = lit ? gb * fp * R.G : 0.0f;
            ga[j] = gb * (ln_e + cont) * DPCS_INV_PI_F;
            dr += gb * (R.dsp * ln_e + R.dsi * cont);
            A[j] = fp * ln_e + fi * cont;
        }
        int idx[4];
        float w[4];
        if (F64 ? a.dtex64 != nullptr : a.dtex != nullptr) {  // null when the caller wants no texture gradient
            Bilin tb;
            tb.x0 = R.tx0; tb.y0 = R.ty0; tb.fx = R.tfx; tb.fy = R.tfy;
            bilin_taps(tb, a.Wt, a.Ht, idx, w);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if constexpr (F64) {
                    double *p = a.dtex64 + 4 * (int64_t)idx[k];
                    atomicAdd(p + 0, (double)ga[0] * (double)w[k]);
                    atomicAdd(p + 1, (double)ga[1] * (double)w[k]);
                    atomicAdd(p + 2, (double)ga[2] * (double)w[k]);
                    atomicAdd(p + 3, (double)dr * (double)w[k]);
                } else {
                    scatter_add4(a.dtex, idx[k], make_float4(ga[0] * w[k], ga[1] * w[k], ga[2] * w[k], dr * w[k]),
                                 row);
                }
            }
        }
        if (R.G > 0.0f && (dEp[0] != 0.0f || dEp[1] != 0.0f || dEp[2] != 0.0f)) {
            Bilin pb;
            pb.x0 = R.px0; pb.y0 = R.py0; pb.fx = R.pfx; pb.fy = R.pfy;
            bilin_taps(pb, a.Wp, a.Hp, idx, w);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if constexpr (F64) {
                    double *p = a.dEp64 + 3 * (int64_t)idx[k];
                    atomicAdd(p + 0, (double)dEp[0] * (double)w[k]);
                    atomicAdd(p + 1, (double)dEp[1] * (double)w[k]);
                    atomicAdd(p + 2, (double)dEp[2] * (double)w[k]);
                } else {
                    scatter_add4(a.dEp, idx[k], make_float4(dEp[0] * w[k], dEp[1] * w[k], dEp[2] * w[k], 0.0f), row);
                }
            }
        }
    }
}

// Path-replay adjoint.  Same thread mapping and loops as k_render: each lane
// re-traces its paths from their Philox counters one ray per iteration and
// records every vertex; once every path of the warp has ended, the lanes run
// their reverse sweeps together and start their next samples.
template <bool F64>
__global__ void __launch_bounds__(kRenderBlock, DPCS_GRAD_MINB) k_replay(const RenderArgs a) {
    const int L = 1 << a.log2L;
    const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t pix = gt >> a.log2L;
    const int sl = (int)(gt & (L - 1));
    const int64_t npix = (int64_t)a.Hc * a.Wc;
    Cnt cnt;
    const float inv = 1.0f / (float)a.spp;
    float gb_in[3] = {0.f, 0.f, 0.f};
    if (pix < npix) {
        gb_in[0] = a.gE[3 * pix] * inv;
        gb_in[1] = a.gE[3 * pix + 1] * inv;
        gb_in[2] = a.gE[3 * pix + 2] * inv;
    }
    const bool any = gb_in[0] != 0.0f || gb_in[1] != 0.0f || gb_in[2] != 0.0f;
    __shared__ float4 s_row[kRenderBlock];  // per-warp rows for scatter_add4
    int s = (pix < npix && any) ? sl : a.spp;
    int b = 1, nv = 0;
    bool shadow = false, has_ext = false, pending = false, nulls = false;
    f3 beta = mk3(0.f, 0.f, 0.f), ed = beta;
    Ray ray;
    ray.o = ray.d = ray.inv = beta;
    float tmax = INFINITY;
    Trav st;
    int stack[kStack];
    VRec rec[DPCS_MAX_BOUNCES];
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
        while (true) {  // the lane's current path; the warp sweeps and starts its next samples together
            if (++iter > max_iter) {
                atomicOr(a.status, kStatusTraversalLimit);
                s = a.spp;
                nv = 0;
                break;
            }
            const int alive = DPCS_YIELD_MIN > 0 ? __popc(__activemask()) : 0;
            if (!pending) {
                if (!nulls) cnt.add(shadow ? kCntShadow : kCntRay);
                trav_begin(st, a.root, shadow ? tmax : INFINITY, shadow);
                pending = true;
            }
            if (!trav_resume(a.nodes, a.tris, nulls ? kEmptyRoot : a.root, a.T, ray, st, stack, a.status, cnt, min(DPCS_YIELD_MIN, alive), a.visit_cap))
                continue;
            pending = false;
            const bool hit = st.h.pos >= 0;
            bool end = false;
            if (shadow) {
                if (hit) rec[nv - 1].G = 0.0f;  // occluded: no projector light at this vertex
                else if (!nulls) cnt.add(kCntLit);
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
                const Surf S = surface_at(a, st.h, ray.d);
                VRec *R = &rec[nv++];
                R->tx0 = S.tb.x0; R->ty0 = S.tb.y0; R->tfx = S.tb.fx; R->tfy = S.tb.fy;
                R->beta[0] = beta.x; R->beta[1] = beta.y; R->beta[2] = beta.z;
                R->rho[0] = S.rho.x; R->rho[1] = S.rho.y; R->rho[2] = S.rho.z;
                R->G = 0.0f; R->cw = 0.0f; R->unc = 0u; R->sp = R->dsp = R->si = R->dsi = 0.0f;
                Nee N;
                const bool cand = nee_prepare(a, S, N);
                if (cand) {
                    unsigned unc;
                    nee_contrib(a, beta, N, unc);
                    R->px0 = N.pb.x0; R->py0 = N.pb.y0; R->pfx = N.pb.fx; R->pfy = N.pb.fy;
                    R->Ep[0] = N.ep.x; R->Ep[1] = N.ep.y; R->Ep[2] = N.ep.z;
                    R->G = N.G; R->sp = N.sp; R->dsp = N.dsp; R->unc = unc;
                }
                has_ext = false;
                if (b < a.bounces) {
                    Cont C;
                    if (continue_prepare(a, (uint32_t)pix, (uint32_t)s, b, S, C)) {
                        cnt.add(kCntCont);
                        beta = beta * C.w;
                        ed = C.wi;
                        has_ext = true;
                        R->si = C.si; R->dsi = C.dsi; R->cw = C.cw;
                    }
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
        replay_sweep<F64>(a, rec, nv, gb_in, &s_row[threadIdx.x & ~31]);
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
}

// Forward render, per-pixel loss and path-replay adjoint in one pass, for
// losses that act on each pixel alone (the L2 loss of Eq. 13, the L1 term of
// Eq. 9).  Each lane traces its samples as k_render does -- the same rounds,
// the same per-lane sum, the same xor-shuffle tree, so Ec and Ic are those of
// k_render bit for bit -- and records every vertex as k_replay does.  Once
// the warp holds its pixels' Ec, every lane knows its pixel's dLoss/dEc
// (the loss's gradient through Eq. 5), and runs the reverse sweeps over the
// vertices it recorded: the paths are traced once, not twice.  The host
// calls it only when ceil(spp / L) <= kFusedSamples and ceil(spp / L) *
// bounces <= kFusedRecs.
template <bool F64>
__global__ void __launch_bounds__(kRenderBlock, DPCS_GRAD_MINB) k_render_grad(const RenderArgs a, const LossArgs l) {
    const int L = 1 << a.log2L;
    const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t pix = gt >> a.log2L;
    const int sl = (int)(gt & (L - 1));
    const bool valid = pix < (int64_t)a.Hc * a.Wc;
    Cnt cnt;
    __shared__ float4 s_row[kRenderBlock];  // per-warp rows for scatter_add4
    int s = valid ? sl : a.spp;
    int b = 1, nv = 0, k = 0;
    bool shadow = false, has_ext = false, pending = false, nulls = false;
    f3 sum = mk3(0.f, 0.f, 0.f);
    f3 beta = sum, c = sum, ed = sum;
    Ray ray;
    ray.o = ray.d = ray.inv = beta;
    float tmax = INFINITY;
    Trav st;
    int stack[kStack];
    VRec rec[kFusedRecs];
    int nvs[kFusedSamples];
#pragma unroll
    for (int i = 0; i < kFusedSamples; ++i) nvs[i] = 0;
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
        VRec *rs = rec + k * a.bounces;  // this sample's records
        while (true) {  // the lane's current path; the warp starts its next samples together
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
            // the same call as in k_render and k_replay: passing a literal 0 for
            // min_active instead (the same value) made this kernel 3.2x slower
            const int alive = DPCS_YIELD_MIN > 0 ? __popc(__activemask()) : 0;
            if (!trav_resume(a.nodes, a.tris, nulls ? kEmptyRoot : a.root, a.T, ray, st, stack, a.status, cnt, min(DPCS_YIELD_MIN, alive),
                             a.visit_cap))
                continue;
            pending = false;
            const bool hit = st.h.pos >= 0;
            bool end = false;
            if (shadow) {
                if (hit) {
                    rs[nv - 1].G = 0.0f;  // occluded: no projector light at this vertex
                } else if (!nulls) {
                    sum = sum + c;
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
                const Surf S = surface_at(a, st.h, ray.d);
                VRec *R = &rs[nv++];
                R->tx0 = S.tb.x0; R->ty0 = S.tb.y0; R->tfx = S.tb.fx; R->tfy = S.tb.fy;
                R->beta[0] = beta.x; R->beta[1] = beta.y; R->beta[2] = beta.z;
                R->rho[0] = S.rho.x; R->rho[1] = S.rho.y; R->rho[2] = S.rho.z;
                R->G = 0.0f; R->cw = 0.0f; R->unc = 0u; R->sp = R->dsp = R->si = R->dsi = 0.0f;
                Nee N;
                const bool cand = nee_prepare(a, S, N);
                if (cand) {
                    unsigned unc;
                    c = nee_contrib(a, beta, N, unc);
                    R->px0 = N.pb.x0; R->py0 = N.pb.y0; R->pfx = N.pb.fx; R->pfy = N.pb.fy;
                    R->Ep[0] = N.ep.x; R->Ep[1] = N.ep.y; R->Ep[2] = N.ep.z;
                    R->G = N.G; R->sp = N.sp; R->dsp = N.dsp; R->unc = unc;
                }
                has_ext = false;
                if (b < a.bounces) {
                    Cont C;
                    if (continue_prepare(a, (uint32_t)pix, (uint32_t)s, b, S, C)) {
                        cnt.add(kCntCont);
                        beta = beta * C.w;
                        ed = C.wi;
                        has_ext = true;
                        R->si = C.si; R->dsi = C.dsi; R->cw = C.cw;
                    }
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
        nvs[k < kFusedSamples ? k : kFusedSamples - 1] = nv;
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
    // every lane of a pixel ends with the pixel's sum (the tree of render_lanes)
    for (int off = L >> 1; off > 0; off >>= 1) {
        sum.x += __shfl_xor_sync(0xffffffffu, sum.x, off);
        sum.y += __shfl_xor_sync(0xffffffffu, sum.y, off);
        sum.z += __shfl_xor_sync(0xffffffffu, sum.z, off);
    }
    const float inv = 1.0f / (float)a.spp;
    const float ec[3] = {sum.x * inv, sum.y * inv, sum.z * inv};
    float gb_in[3] = {0.f, 0.f, 0.f};
    float v[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // gamma_c(3), Gc, wb(3), loss
    if (valid) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float ic = crf(ec[j], a.gain_c, a.wb[j], a.gamma_c[j]);
            if (sl == 0) {
                if (a.Ec) a.Ec[3 * pix + j] = ec[j];
                a.Ic[3 * pix + j] = ic;
            }
            const float d = ic - l.target[3 * pix + j];
            const float g = l.kind == 0 ? l.scale * d : (d > 0.0f ? l.scale : (d < 0.0f ? -l.scale : 0.0f));
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
            if (sl == 0) v[7] += l.kind == 0 ? 0.5f * l.scale * d * d : l.scale * fabsf(d);
        }
    }
    block_reduce_add<8>(v, l.acc + 4);  // acc[4..10]: gamma_c, Gc, wb; acc[11]: the loss
    const bool any = gb_in[0] != 0.0f || gb_in[1] != 0.0f || gb_in[2] != 0.0f;
    for (int i = 0; any && i < k && i < kFusedSamples; ++i)
        replay_sweep<F64>(a, rec + i * a.bounces, nvs[i], gb_in, &s_row[threadIdx.x & ~31]);
}

// Forward render that keeps every path's vertex records in device memory
// (dpcs_render_keep): the loop is k_render_grad's, with the records of each
// sample copied out when its path ends and Ec / Ic written as k_render
// writes them, so a later k_sweep_kept can run the adjoint of any loss,
// including one that couples pixels (the Eq. 11 filter), without tracing
// the paths again.
__global__ void __launch_bounds__(kRenderBlock, DPCS_GRAD_MINB)
    k_render_keep(const RenderArgs a, uint4 *__restrict__ chunks, uint8_t *__restrict__ nvs) {
    const int L = 1 << a.log2L;
    const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t pix = gt >> a.log2L;
    const int sl = (int)(gt & (L - 1));
    const bool valid = pix < (int64_t)a.Hc * a.Wc;
    Cnt cnt;
    const int64_t nthr = ((int64_t)a.Hc * a.Wc) << a.log2L;
    int s = valid ? sl : a.spp;
    int b = 1, nv = 0, k = 0;
    bool shadow = false, has_ext = false, pending = false, nulls = false;
    f3 sum = mk3(0.f, 0.f, 0.f);
    f3 beta = sum, c = sum, ed = sum;
    Ray ray;
    ray.o = ray.d = ray.inv = beta;
    float tmax = INFINITY;
    Trav st;
    int stack[kStack];
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
        while (true) {  // the lane's current path; the warp starts its next samples together
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
            // the same call as in k_render and k_replay: passing a literal 0 for
            // min_active instead (the same value) made this kernel 3.2x slower
            const int alive = DPCS_YIELD_MIN > 0 ? __popc(__activemask()) : 0;
            if (!trav_resume(a.nodes, a.tris, nulls ? kEmptyRoot : a.root, a.T, ray, st, stack, a.status, cnt, min(DPCS_YIELD_MIN, alive),
                             a.visit_cap))
                continue;
            pending = false;
            const bool hit = st.h.pos >= 0;
            bool end = false;
            if (shadow) {
                if (hit) {
                    // occluded: no projector light at the last recorded vertex
                    if (valid) {
                        uint32_t *w = reinterpret_cast<uint32_t *>(chunks + kept_chunk(kKeptGChunk, k, nv - 1, spl,
                                                                                       a.bounces, nthr, gt));
                        __stcs(w + kKeptGWord, 0u);
                    }
                } else if (!nulls) {
                    sum = sum + c;
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
                const Surf S = surface_at(a, st.h, ray.d);
                const f3 beta_v = beta;
                Nee N;
                const bool cand = nee_prepare(a, S, N);
                unsigned unc = 0u;
                if (cand) c = nee_contrib(a, beta, N, unc);
                has_ext = false;
                Cont C;
                C.si = C.dsi = C.cw = 0.0f;
                if (b < a.bounces) {
                    if (continue_prepare(a, (uint32_t)pix, (uint32_t)s, b, S, C)) {
                        cnt.add(kCntCont);
                        beta = beta * C.w;
                        ed = C.wi;
                        has_ext = true;
                    } else {
                        C.si = C.dsi = C.cw = 0.0f;
                    }
                }
                // the vertex record (the fields of VRec, in order) straight to
                // the kept buffer: six 16-byte chunks, streaming stores
                if (valid) {
                    const uint32_t px0 = cand ? (uint32_t)N.pb.x0 : 0u, py0 = cand ? (uint32_t)N.pb.y0 : 0u;
                    const float pfx = cand ? N.pb.fx : 0.0f, pfy = cand ? N.pb.fy : 0.0f;
                    const float e0 = cand ? N.ep.x : 0.0f, e1 = cand ? N.ep.y : 0.0f, e2 = cand ? N.ep.z : 0.0f;
                    const float G = cand ? N.G : 0.0f, sp = cand ? N.sp : 0.0f, dsp = cand ? N.dsp : 0.0f;
                    const uint4 q[kKeptChunks] = {
                        make_uint4((uint32_t)S.tb.x0, (uint32_t)S.tb.y0, px0, py0),
                        make_uint4(__float_as_uint(S.tb.fx), __float_as_uint(S.tb.fy), __float_as_uint(pfx),
                                   __float_as_uint(pfy)),
                        make_uint4(__float_as_uint(beta_v.x), __float_as_uint(beta_v.y), __float_as_uint(beta_v.z),
                                   __float_as_uint(e0)),
                        make_uint4(__float_as_uint(e1), __float_as_uint(e2), __float_as_uint(G),
                                   __float_as_uint(S.rho.x)),
                        make_uint4(__float_as_uint(S.rho.y), __float_as_uint(S.rho.z), __float_as_uint(sp),
                                   __float_as_uint(dsp)),
                        make_uint4(__float_as_uint(C.si), __float_as_uint(C.dsi), __float_as_uint(C.cw), unc)};
#pragma unroll
                    for (int q4 = 0; q4 < kKeptChunks; ++q4)
                        __stcs(chunks + kept_chunk(q4, k, nv, spl, a.bounces, nthr, gt), q[q4]);
                }
                ++nv;
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
        if (valid) nvs[(int64_t)k * nthr + gt] = (uint8_t)nv;  // sample k's vertex count
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
        a.Ic[3 * pix] = crf(ex, a.gain_c, a.wb[0], a.gamma_c[0]);
        a.Ic[3 * pix + 1] = crf(ey, a.gain_c, a.wb[1], a.gamma_c[1]);
        a.Ic[3 * pix + 2] = crf(ez, a.gain_c, a.wb[2], a.gamma_c[2]);
    }
}

// The adjoint from the records k_render_keep wrote: the reverse sweep of
// every recorded path with its pixel's dLoss/dEc, without tracing again.
template <bool F64>
__global__ void __launch_bounds__(kRenderBlock) k_sweep_kept(const RenderArgs a, const uint4 *__restrict__ chunks,
                                                             const uint8_t *__restrict__ nvs) {
    const int L = 1 << a.log2L;
    const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t pix = gt >> a.log2L;
    const int64_t nthr = ((int64_t)a.Hc * a.Wc) << a.log2L;
    __shared__ float4 s_row[kRenderBlock];  // per-warp rows for scatter_add4
    if (pix >= (int64_t)a.Hc * a.Wc) return;
    const float inv = 1.0f / (float)a.spp;
    const float gb_in[3] = {a.gE[3 * pix] * inv, a.gE[3 * pix + 1] * inv, a.gE[3 * pix + 2] * inv};
    if (gb_in[0] == 0.0f && gb_in[1] == 0.0f && gb_in[2] == 0.0f) return;
    const int sl = (int)(gt & (L - 1));
    const int spl = (a.spp + L - 1) / L;
    VRec rec[DPCS_MAX_BOUNCES];
    for (int k = 0; k < spl && sl + k * L < a.spp; ++k) {
        const int nv = nvs[(int64_t)k * nthr + gt];
        for (int v = 0; v < nv; ++v) {
            uint4 *dst = reinterpret_cast<uint4 *>(&rec[v]);
#pragma unroll
            for (int q4 = 0; q4 < kKeptChunks; ++q4) dst[q4] = __ldcs(chunks + kept_chunk(q4, k, v, spl, a.bounces, nthr, gt));
        }
        replay_sweep<F64>(a, rec, nv, gb_in, &s_row[threadIdx.x & ~31]);
    }
}

// Eq. 1 adjoint: dIp += dEp Gp gamma Ip^(gamma-1); gamma_p and Gp reductions
__global__ void k_prf_backward(const float *__restrict__ Ip, const float4 *__restrict__ dEp, int64_t ntex,
                               float g0, float g1, float g2, float gain, float *__restrict__ dIp, double *acc) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float v[4] = {0, 0, 0, 0};
    if (t < ntex) {
        const float4 g4 = dEp[t];
        const float gs[3] = {g4.x, g4.y, g4.z}, gm[3] = {g0, g1, g2};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float ip = Ip[3 * t + j];
            if (ip > 0.0f && gs[j] != 0.0f) {
                const float pw = powf(ip, gm[j]);
                if (dIp) dIp[3 * t + j] += gs[j] * gain * gm[j] * powf(ip, gm[j] - 1.0f);
                v[j] += gs[j] * gain * pw * logf(ip);
                v[3] += gs[j] * pw;
            }
        }
    }
    block_reduce_add<4>(v, acc);
}

// the same from FP64 accumulators: the per-texel factors Ip^gamma, its
// derivative and ln Ip in FP32 (as k_prf_backward), the products and the
// reductions in FP64 before the result is rounded
__global__ void k_prf_backward64(const float *__restrict__ Ip, const double *__restrict__ dEp, int64_t ntex,
                                 float g0, float g1, float g2, float gain, float *__restrict__ dIp, double *acc) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double v[4] = {0, 0, 0, 0};
    if (t < ntex) {
        const float gm[3] = {g0, g1, g2};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float ip = Ip[3 * t + j];
            const double gs = dEp[3 * t + j];
            if (ip > 0.0f && gs != 0.0) {
                const double pw = (double)powf(ip, gm[j]);
                if (dIp) dIp[3 * t + j] += (float)(gs * (double)(gain * gm[j] * powf(ip, gm[j] - 1.0f)));
                v[j] += gs * (double)gain * pw * (double)logf(ip);
                v[3] += gs * pw;
            }
        }
    }
    __shared__ double red[4][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        for (int off = 16; off; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) red[k][w] = v[k];
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int j = 0; j < (int)(blockDim.x >> 5); ++j) s += red[threadIdx.x][j];
        if (s != 0.0) atomicAdd(acc + threadIdx.x, s);
    }
}

__global__ void k_tex_backward64(const double *__restrict__ dtex, int64_t ntex, float *__restrict__ dAlbedo,
                                 float *__restrict__ dRough) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= ntex) return;
    if (dAlbedo) {
        dAlbedo[3 * t] += (float)dtex[4 * t];
        dAlbedo[3 * t + 1] += (float)dtex[4 * t + 1];
        dAlbedo[3 * t + 2] += (float)dtex[4 * t + 2];
    }
    if (dRough) dRough[t] += (float)dtex[4 * t + 3];
}

__global__ void k_tex_backward(const float4 *__restrict__ dtex, int64_t ntex, float *__restrict__ dAlbedo,
                               float *__restrict__ dRough) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= ntex) return;
    const float4 g = dtex[t];
    if (dAlbedo) {
        dAlbedo[3 * t] += g.x;
        dAlbedo[3 * t + 1] += g.y;
        dAlbedo[3 * t + 2] += g.z;
    }
    if (dRough) dRough[t] += g.w;
}

// the per-pixel loss of LossArgs as its own pass (when k_render_grad would
// need more records than it keeps): dIc, and the loss into acc[11]
__global__ void k_pixel_loss(const float *__restrict__ Ic, int64_t n, const LossArgs l, float *__restrict__ dIc) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float v[1] = {0.0f};
    if (i < n) {
        const float d = Ic[i] - l.target[i];
        dIc[i] = l.kind == 0 ? l.scale * d : (d > 0.0f ? l.scale : (d < 0.0f ? -l.scale : 0.0f));
        v[0] = l.kind == 0 ? 0.5f * l.scale * d * d : l.scale * fabsf(d);
    }
    block_reduce_add<1>(v, l.acc + 11);
}

__global__ void k_loss_out(const double *__restrict__ acc, float *__restrict__ loss) { *loss = (float)acc[11]; }

__global__ void k_finalize(const double *__restrict__ acc, float *__restrict__ dParams) {
    const int i = threadIdx.x;
    if (i < 11) dParams[i] += (float)acc[i];
}

inline unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

}  // namespace

int launch_prf(const float *Ip, int64_t ntex, const float gamma_p[3], float gain_p, float4 *Ep, cudaStream_t st) {
    k_prf<<<grid_for(ntex, 256), 256, 0, st>>>(Ip, ntex, gamma_p[0], gamma_p[1], gamma_p[2], gain_p, Ep);
    return 1;
}

int launch_pack_tex(const float *albedo, const float *rough, int64_t ntex, float4 *tex, cudaStream_t st) {
    k_pack_tex<<<grid_for(ntex, 256), 256, 0, st>>>(albedo, rough, ntex, tex);
    return 1;
}

int launch_render(const RenderArgs &a, cudaStream_t st) {
    const int64_t threads = ((int64_t)a.Hc * a.Wc) << a.log2L;
    k_render<<<grid_for(threads, kRenderBlock), kRenderBlock, 0, st>>>(a);
    return 1;
}

int launch_render_batch(const RenderArgs *descs, const BatchSeg *segs, int nseg, int64_t total_vb,
                        unsigned long long *counter, int grid, cudaStream_t st) {
    k_render_batch<<<grid, kRenderBlock, 0, st>>>(descs, segs, nseg, total_vb, counter);
    return 1;
}

int render_batch_grid(int device) {
    int per_sm = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render_batch, kRenderBlock, 0);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    return per_sm > 0 && sms > 0 ? per_sm * sms : 1;
}

int64_t render_batch_vblocks(int64_t npix, int log2L) {
    return ((npix << log2L) + kRenderBlock - 1) / kRenderBlock;
}

int launch_trace(const Scene &sc, const float *o, const float *d, int64_t n, float *t, int32_t *tri,
                 unsigned *status, cudaStream_t st) {
    k_trace<<<grid_for(n, 128), 128, 0, st>>>(sc.nodes, sc.tris, sc.root, sc.T, o, d, n, t, tri, status);
    return 1;
}

int launch_crf_backward(const float *dIc, const float *Ec, const float *Ic, int64_t npix, const float gamma_c[3],
                        float gain_c, const float wb[3], float *gE, double *acc, cudaStream_t st) {
    k_crf_backward<<<grid_for(npix, 256), 256, 0, st>>>(dIc, Ec, Ic, npix, gamma_c[0], gamma_c[1], gamma_c[2],
                                                        gain_c, wb[0], wb[1], wb[2], gE, acc);
    return 1;
}

int launch_replay(const RenderArgs &a, cudaStream_t st) {
    const int64_t threads = ((int64_t)a.Hc * a.Wc) << a.log2L;
    if (a.dEp64)
        k_replay<true><<<grid_for(threads, kRenderBlock), kRenderBlock, 0, st>>>(a);
    else
        k_replay<false><<<grid_for(threads, kRenderBlock), kRenderBlock, 0, st>>>(a);
    return 1;
}

int launch_render_grad(const RenderArgs &a, const LossArgs &l, cudaStream_t st) {
    const int64_t threads = ((int64_t)a.Hc * a.Wc) << a.log2L;
    if (a.dEp64)
        k_render_grad<true><<<grid_for(threads, kRenderBlock), kRenderBlock, 0, st>>>(a, l);
    else
        k_render_grad<false><<<grid_for(threads, kRenderBlock), kRenderBlock, 0, st>>>(a, l);
    return 1;
}

int launch_render_keep(const RenderArgs &a, void *chunks, uint8_t *nvs, cudaStream_t st) {
    const int64_t threads = ((int64_t)a.Hc * a.Wc) << a.log2L;
    k_render_keep<<<grid_for(threads, kRenderBlock), kRenderBlock, 0, st>>>(a, (uint4 *)chunks, nvs);
    return 1;
}

int launch_sweep_kept(const RenderArgs &a, const void *chunks, const uint8_t *nvs, cudaStream_t st) {
    const int64_t threads = ((int64_t)a.Hc * a.Wc) << a.log2L;
    if (a.dEp64)
        k_sweep_kept<true><<<grid_for(threads, kRenderBlock), kRenderBlock, 0, st>>>(a, (const uint4 *)chunks, nvs);
    else
        k_sweep_kept<false><<<grid_for(threads, kRenderBlock), kRenderBlock, 0, st>>>(a, (const uint4 *)chunks, nvs);
    return 1;
}

int launch_pixel_loss(const float *Ic, int64_t n, const LossArgs &l, float *dIc, cudaStream_t st) {
    k_pixel_loss<<<grid_for(n, 256), 256, 0, st>>>(Ic, n, l, dIc);
    return 1;
}

int launch_loss_out(const double *acc, float *loss, cudaStream_t st) {
    k_loss_out<<<1, 1, 0, st>>>(acc, loss);
    return 1;
}

int launch_prf_backward(const float *Ip, const float4 *dEp, int64_t ntex, const float gamma_p[3], float gain_p,
                        float *dIp, double *acc, cudaStream_t st) {
    k_prf_backward<<<grid_for(ntex, 256), 256, 0, st>>>(Ip, dEp, ntex, gamma_p[0], gamma_p[1], gamma_p[2], gain_p,
                                                        dIp, acc);
    return 1;
}

int launch_tex_backward(const float4 *dtex, int64_t ntex, float *dAlbedo, float *dRough, cudaStream_t st) {
    k_tex_backward<<<grid_for(ntex, 256), 256, 0, st>>>(dtex, ntex, dAlbedo, dRough);
    return 1;
}

int launch_prf_backward64(const float *Ip, const double *dEp64, int64_t ntex, const float gamma_p[3], float gain_p,
                          float *dIp, double *acc, cudaStream_t st) {
    k_prf_backward64<<<grid_for(ntex, 256), 256, 0, st>>>(Ip, dEp64, ntex, gamma_p[0], gamma_p[1], gamma_p[2],
                                                          gain_p, dIp, acc);
    return 1;
}

int launch_tex_backward64(const double *dtex64, int64_t ntex, float *dAlbedo, float *dRough, cudaStream_t st) {
    k_tex_backward64<<<grid_for(ntex, 256), 256, 0, st>>>(dtex64, ntex, dAlbedo, dRough);
    return 1;
}

int launch_finalize_params(const double *acc, float *dParams, cudaStream_t st) {
    k_finalize<<<1, 32, 0, st>>>(acc, dParams);
    return 1;
}

int launch_zero(void *p, size_t bytes, cudaStream_t st) {
    cudaMemsetAsync(p, 0, bytes, st);
    return 0;
}

}  // namespace dpcs
