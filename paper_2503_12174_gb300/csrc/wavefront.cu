// wavefront.cu -- the forward render of Eq. 7 as a wavefront of short
// kernels over compacted path queues.
//
// The megakernel (k_render) runs each lane's path from camera to its last
// vertex; a warp's lanes then drift apart (different traversal lengths,
// shadow ray or not, paths ending early) and the warp executes the union of
// their work.  Here every pass does one kind of work for every live path:
//
//   k_wf_trace   closest hit of every extension ray of one bounce (camera
//                rays at bounce 1, generated in place from the Philox stream);
//   k_wf_shade   at each hit: surface, next-event estimation with its shadow
//                ray traced at once (shadow rays of neighbouring paths point
//                at the same projector centre), the lane's pixel sum, and the
//                BRDF continuation, whose paths are appended to the next
//                bounce's queue (warp-aggregated atomics).
//
// Path state between passes lives in device memory (hit, ray, throughput;
// 16-byte records).  Paths are processed in chunks small enough for that
// state to stay in L2.  A path is (pixel, lane, wave): lane sl of pixel pix
// traces sample sl + wave * L in wave `wave`, and adds its lit vertices to the
// lane's running sum in sample-then-vertex order, exactly as k_render's lane
// does; k_wf_finish combines the L lane sums with k_render's xor-shuffle tree.
// Every per-vertex function is the megakernel's (device.cuh), so the images
// are k_render's bit for bit.
#include <cuda_runtime.h>
#include <stdint.h>

#include "device.cuh"
#include "internal.h"

namespace dpcs {

static_assert(kStack >= kMaxTreeDepth, "a tree the builders accept must fit the traversal stack");


namespace {

constexpr int kWfBlock = 128;
#ifndef DPCS_WF_TRACE_MINB
#define DPCS_WF_TRACE_MINB 10  // resident blocks per SM asked of ptxas for the trace pass
#endif
#ifndef DPCS_WF_SHADE_MINB
#define DPCS_WF_SHADE_MINB 8   // and for the shading pass (shading plus a shadow-ray traversal)
#endif

__device__ __forceinline__ float crf_wf(float ec, float gain, float wb, float gamma) {
    const float a = gain * wb * ec;
    return a > 0.0f ? powf(a, gamma) : 0.0f;
}

// append this lane's path to a queue: one atomic per converged group of
// lanes (a warp, unless some of its lanes have left)
__device__ __forceinline__ void queue_push(int32_t *q, int32_t *n, int32_t v, bool take) {
    const unsigned act = __activemask();
    const unsigned m = __ballot_sync(act, take);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(n, __popc(m));
    base = __shfl_sync(act, base, leader);
    if (take) q[base + __popc(m & ((1u << lane) - 1u))] = v;
}

// closest or any hit of one ray with the context's visit cap (as k_render)
__device__ __forceinline__ bool trace_one(const RenderArgs &a, const Ray &ray, float tmax, bool any, Hit &h,
                                          Cnt &cnt) {
    Trav st;
    int stack[kStack];
    trav_begin(st, a.root, tmax, any);
    trav_resume(a.nodes, a.tris, a.root, a.T, ray, st, stack, a.status, cnt, 0, a.visit_cap);
    h = st.h;
    return h.pos >= 0;
}

// chunk-local path c -> pixel, lane-in-pixel, sample; false if the sample is
// past spp (the last wave of an spp that L does not divide) or the pixel is
// past the image
__device__ __forceinline__ bool path_of(const WfPass &w, int32_t c, int64_t &g, int64_t &pix, uint32_t &s) {
    g = w.path0 + c;
    pix = g >> w.r.log2L;
    const int sl = (int)(g & ((1 << w.r.log2L) - 1));
    s = (uint32_t)(sl + w.wave * (1 << w.r.log2L));
    return pix < (int64_t)w.r.Hc * w.r.Wc && (int)s < w.r.spp;
}

// Closest hit of the extension rays of one bounce.  At bounce 1 the rays are
// the camera rays of every path of the chunk; later, the paths of the input
// queue with the rays k_wf_shade stored.
__global__ void __launch_bounds__(kWfBlock, DPCS_WF_TRACE_MINB) k_wf_trace(const WfPass w) {
    const int32_t t = blockIdx.x * kWfBlock + threadIdx.x;
    const int32_t n = w.qin ? *w.nin : w.nchunk;
    Cnt cnt;
    const RenderArgs &a = w.r;
    if (t < n) {  // no early return: the counters build reduces over whole warps
        int32_t c;
        Ray ray;
        bool live = true;
        if (!w.qin) {
            c = t;
            int64_t g, pix;
            uint32_t s;
            live = path_of(w, c, g, pix, s) && a.bounces > 0;
            if (live) {
                f3 o, d;
                camera_ray(a, (uint32_t)pix, s, o, d);
                ray = make_ray(o, d);
                cnt.add(kCntPath);
            }
        } else {
            c = w.qin[t];
            const float4 o4 = w.ro[c], d4 = w.rd[c];
            ray = make_ray(xyz(o4), xyz(d4));
        }
        Hit h;
        h.pos = -1;
        h.u = h.v = 0.0f;
        if (live) {
            cnt.add(kCntRay);
            trace_one(a, ray, INFINITY, false, h, cnt);
        }
        w.hit[c] = make_float4(__int_as_float(h.pos), h.u, h.v, 0.f);
    }
    cnt.flush(a.counters);
}

#ifndef DPCS_WF_REFILL
// 0: one ray per thread; K > 0: persistent warps whose lanes take a new ray
// from the pass's queue as soon as fewer than K lanes are still traversing
#define DPCS_WF_REFILL 0
#endif

// Persistent closest-hit pass: each warp fetches rays for its idle lanes
// (one atomic per warp), traverses, and yields back to fetching once fewer
// than DPCS_WF_REFILL lanes are still traversing, so warps stay full until
// the queue runs dry.  Same rays and hits as k_wf_trace.
__global__ void __launch_bounds__(kWfBlock, DPCS_WF_TRACE_MINB) k_wf_trace_refill(const WfPass w) {
    const RenderArgs &a = w.r;
    const int32_t n = w.qin ? *w.nin : w.nchunk;
    const int lane = threadIdx.x & 31;
    Cnt cnt;
    bool has = false, done = false;
    int32_t c = 0;
    Ray ray;
    ray.o = ray.d = ray.inv = mk3(0.f, 0.f, 0.f);
    Trav st;
    int stack[kStack];
    trav_begin(st, a.root, INFINITY, false);
    while (true) {
        const unsigned need = __ballot_sync(0xffffffffu, !has && !done);
        if (need) {
            const int leader = __ffs(need) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(w.fetch, __popc(need));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (!has && !done) {
                const int32_t idx = base + __popc(need & ((1u << lane) - 1u));
                if (idx < n) {
                    bool live = true;
                    if (!w.qin) {
                        c = idx;
                        int64_t g, pix;
                        uint32_t s;
                        live = path_of(w, c, g, pix, s) && a.bounces > 0;
                        if (live) {
                            f3 o, d;
                            camera_ray(a, (uint32_t)pix, s, o, d);
                            ray = make_ray(o, d);
                            cnt.add(kCntPath);
                        }
                    } else {
                        c = w.qin[idx];
                        const float4 o4 = w.ro[c], d4 = w.rd[c];
                        ray = make_ray(xyz(o4), xyz(d4));
                    }
                    if (live) {
                        cnt.add(kCntRay);
                        trav_begin(st, a.root, INFINITY, false);
                        has = true;
                    } else {
                        w.hit[c] = make_float4(__int_as_float(-1), 0.f, 0.f, 0.f);
                    }
                } else {
                    done = true;
                }
            }
        }
        if (!__any_sync(0xffffffffu, has)) break;
        if (has) {
            const int alive = __popc(__activemask());
            if (trav_resume(a.nodes, a.tris, a.root, a.T, ray, st, stack, a.status, cnt, min(DPCS_WF_REFILL, alive),
                            a.visit_cap)) {
                w.hit[c] = make_float4(__int_as_float(st.h.pos), st.h.u, st.h.v, 0.f);
                has = false;
            }
        }
        __syncwarp();
    }
    cnt.flush(a.counters);
}

// Shading of one bounce's hits: next-event estimation (shadow ray traced
// here), the lane's pixel sum, and the continuation into the next queue.
__global__ void __launch_bounds__(kWfBlock, DPCS_WF_SHADE_MINB) k_wf_shade(const WfPass w) {
    const int32_t t = blockIdx.x * kWfBlock + threadIdx.x;
    const int32_t n = w.qin ? *w.nin : w.nchunk;
    Cnt cnt;
    const RenderArgs &a = w.r;
    bool cont = false;
    int32_t c = 0;
    if (t < n) {  // no early return: the queue append and the counters reduce over whole warps
        c = w.qin ? w.qin[t] : t;
        int64_t g, pix;
        uint32_t s;
        path_of(w, c, g, pix, s);
        const float4 h4 = w.hit[c];
        Hit h;
        h.pos = __float_as_int(h4.x);
        if (h.pos >= 0) {
            h.u = h4.y;
            h.v = h4.z;
            f3 d, beta;
            if (w.b == 1) {
                f3 o;
                camera_ray(a, (uint32_t)pix, s, o, d);
                beta = mk3(1.f, 1.f, 1.f);
            } else {
                d = xyz(w.rd[c]);
                beta = xyz(w.beta[c]);
            }
            cnt.add(kCntVert);
            const Surf S = surface_at(a, h, d);
            Nee N;
            const bool cand = nee_prepare(a, S, N);
            if (cand) {
                unsigned unc;
                const f3 cv = nee_contrib(a, beta, N, unc);
                cnt.add(kCntShadow);
                Hit sh;
                if (!trace_one(a, make_ray(N.so, N.sdir), N.smax, true, sh, cnt)) {
                    float4 sm = w.sum[g];
                    sm.x = sm.x + cv.x;
                    sm.y = sm.y + cv.y;
                    sm.z = sm.z + cv.z;
                    w.sum[g] = sm;
                    cnt.add(kCntLit);
                }
            }
            if (w.b < a.bounces) {
                Cont C;
                if (continue_prepare(a, (uint32_t)pix, s, w.b, S, C)) {
                    cnt.add(kCntCont);
                    beta = beta * C.w;
                    // the extension ray starts where the shadow ray did, as in
                    // k_render (the same value, computed in the same place)
                    const f3 o = cand ? N.so : S.x + S.n * kRayEps;
                    w.ro[c] = make_float4(o.x, o.y, o.z, 0.f);
                    w.rd[c] = make_float4(C.wi.x, C.wi.y, C.wi.z, 0.f);
                    w.beta[c] = make_float4(beta.x, beta.y, beta.z, 0.f);
                    cont = true;
                }
            }
        }
    }
    queue_push(w.qout, w.nout, c, cont);
    cnt.flush(a.counters);
}

// The L lane sums of each pixel through k_render's xor-shuffle tree; Ec and
// the camera response (Eqs. 4, 5) as k_render writes them.
__global__ void __launch_bounds__(kWfBlock) k_wf_finish(const RenderArgs a, const float4 *__restrict__ sum) {
    const int64_t gt = blockIdx.x * (int64_t)kWfBlock + threadIdx.x;
    const int64_t pix = gt >> a.log2L;
    const int L = 1 << a.log2L;
    const int64_t npix = (int64_t)a.Hc * a.Wc;
    const bool valid = pix < npix;
    f3 sm = mk3(0.f, 0.f, 0.f);
    if (valid) sm = xyz(sum[gt]);
    for (int off = L >> 1; off > 0; off >>= 1) {
        sm.x += __shfl_xor_sync(0xffffffffu, sm.x, off);
        sm.y += __shfl_xor_sync(0xffffffffu, sm.y, off);
        sm.z += __shfl_xor_sync(0xffffffffu, sm.z, off);
    }
    if (valid && (gt & (L - 1)) == 0) {
        const float inv = 1.0f / (float)a.spp;
        const float ex = sm.x * inv, ey = sm.y * inv, ez = sm.z * inv;
        if (a.Ec) {
            a.Ec[3 * pix] = ex;
            a.Ec[3 * pix + 1] = ey;
            a.Ec[3 * pix + 2] = ez;
        }
        a.Ic[3 * pix] = crf_wf(ex, a.gain_c, a.wb[0], a.gamma_c[0]);
        a.Ic[3 * pix + 1] = crf_wf(ey, a.gain_c, a.wb[1], a.gamma_c[1]);
        a.Ic[3 * pix + 2] = crf_wf(ez, a.gain_c, a.wb[2], a.gamma_c[2]);
    }
}

inline unsigned grid_of(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

}  // namespace

size_t wavefront_scratch_bytes(const RenderArgs &a, int64_t chunk) {
    const int64_t paths = ((int64_t)a.Hc * a.Wc) << a.log2L;
    const int L = 1 << a.log2L;
    const int waves = (a.spp + L - 1) / L;
    const int64_t nchunks = (paths + chunk - 1) / chunk;
    const int64_t npass = (int64_t)waves * nchunks * (a.bounces > 0 ? a.bounces : 1);
    // lane sums, per-chunk path state (hit, ray origin and direction,
    // throughput: four float4), two queues, a queue length and a fetch
    // counter per pass
    return (size_t)paths * 16 + (size_t)chunk * (4 * 16 + 2 * 4) + (size_t)npass * 8 + 256;
}

int launch_render_wavefront(const RenderArgs &a, int64_t chunk, void *scratch, cudaStream_t st) {
    const int64_t paths = ((int64_t)a.Hc * a.Wc) << a.log2L;
    const int L = 1 << a.log2L;
    const int waves = (a.spp + L - 1) / L;
    const int64_t nchunks = (paths + chunk - 1) / chunk;
    const int B = a.bounces > 0 ? a.bounces : 1;
    const int64_t npass = (int64_t)waves * nchunks * B;
    char *p = (char *)scratch;
    float4 *sum = (float4 *)p;
    p += (size_t)paths * 16;
    float4 *hit = (float4 *)p;
    p += (size_t)chunk * 16;
    float4 *ro = (float4 *)p;
    p += (size_t)chunk * 16;
    float4 *rd = (float4 *)p;
    p += (size_t)chunk * 16;
    float4 *beta = (float4 *)p;
    p += (size_t)chunk * 16;
    int32_t *q[2] = {(int32_t *)p, (int32_t *)p + chunk};
    p += (size_t)chunk * 8;
    int32_t *qlen = (int32_t *)p;
    int nl = 0;
    cudaMemsetAsync(sum, 0, (size_t)paths * 16, st);
    cudaMemsetAsync(qlen, 0, (size_t)npass * 8, st);  // queue lengths, then fetch counters
#if DPCS_WF_REFILL > 0
    int refill_grid = 0;
    {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wf_trace_refill, kWfBlock, 0);
        refill_grid = sms * (per_sm > 0 ? per_sm : 1);
    }
#endif
    int64_t pass = 0;
    for (int wv = 0; wv < waves; ++wv) {
        for (int64_t c0 = 0; c0 < paths; c0 += chunk) {
            WfPass w;
            w.r = a;
            w.path0 = c0;
            w.nchunk = (int32_t)(paths - c0 < chunk ? paths - c0 : chunk);
            w.wave = wv;
            w.hit = hit;
            w.ro = ro;
            w.rd = rd;
            w.beta = beta;
            w.sum = sum;
            w.qin = nullptr;
            w.nin = nullptr;
            for (int b = 1; b <= a.bounces; ++b, ++pass) {
                w.b = b;
                w.qout = q[b & 1];
                w.nout = qlen + pass;
#if DPCS_WF_REFILL > 0
                w.fetch = qlen + npass + pass;
                k_wf_trace_refill<<<refill_grid, kWfBlock, 0, st>>>(w);
#else
                k_wf_trace<<<grid_of(w.nchunk, kWfBlock), kWfBlock, 0, st>>>(w);
#endif
                k_wf_shade<<<grid_of(w.nchunk, kWfBlock), kWfBlock, 0, st>>>(w);
                nl += 2;
                w.qin = w.qout;
                w.nin = w.nout;
            }
            if (a.bounces <= 0) ++pass;
        }
    }
    k_wf_finish<<<grid_of(paths, kWfBlock), kWfBlock, 0, st>>>(a, sum);
    return nl + 1;
}

}  // namespace dpcs
