// api.cu -- the C ABI of libdpcs (declared in include/dpcs.h): context,
// scene residency and LBVH build, forward render, path-replay adjoint, loss
// and optimiser.  Host code only validates, sizes scratch memory against the
// context's HBM budget and enqueues the kernels of lbvh.cu, render.cu and
// optim.cu on the caller's stream.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <string>
#include <vector>

#include "dpcs.h"
#include <nvtx3/nvToolsExt.h>

#include "internal.h"
#include "pose.h"

using namespace dpcs;

#ifndef DPCS_MIN_SAMPLES_PER_LANE
#define DPCS_MIN_SAMPLES_PER_LANE 1
#endif

namespace {

constexpr int kMinSamplesPerLane = DPCS_MIN_SAMPLES_PER_LANE;
constexpr int kCounters = 10;  // totals dpcs_counters_read returns

struct Buf {
    void *p = nullptr;
    size_t n = 0;
};

struct TimedLaunch {
    cudaEvent_t a = nullptr, b = nullptr;
    int kernel = 0;
};

// mesh edges of one scene for the pose gradient's silhouette term
struct EdgeTable {
    PoseEdge *d = nullptr;
    int64_t n = 0;
};

}  // namespace

struct dpcs_ctx {
    int device = 0;
    size_t budget = 0;
    size_t used = 0;
    uint64_t launches = 0;
    std::string err;
    unsigned *status = nullptr;       // device status word
    std::map<uint64_t, Scene> scenes;
    uint64_t next_scene = 1;
    // scratch
    Buf ep4, tex4, gE, dEp4, dtex4, acc, partial, build, upload, pix;  // pix: per-pixel dIc and Ec of the unfused loss path
    Buf mat4, dmat4;  // principled material: (metallic, normal map) per texel and its gradient accumulators
    Buf dEp64, dtex64;  // FP64 gradient accumulators (dpcs_set_grad_accum(ctx, DPCS_ACCUM_F64))
    bool grad_f64 = false;
    Buf wf;  // wavefront render: lane sums, per-chunk path state, queues
    int32_t render_path = DPCS_PATH_MEGAKERNEL;
    int64_t wf_chunk = int64_t(1) << 20;
    int32_t bvh_builder = DPCS_BVH_PLOC;  // tree topology of the next uploads
    Buf ploc;  // PLOC build scratch
    Buf pose;  // per-block partial sums of the pose-gradient kernels
    std::map<uint64_t, EdgeTable> edges;  // per scene, built by its first pose-gradient call with silhouettes
    Buf kept;  // path records of the last dpcs_render_keep: 16-byte chunks (structure of arrays), then per-sample vertex counts
    struct {
        bool valid = false;
        uint64_t scene = 0, seed = 0;
        int32_t Hc = 0, Wc = 0, spp = 0, bounces = 0, log2L = 0;
        bool principled = false;  // records of dpcs_render_keep_principled
    } kept_key;
    // measurement support
    unsigned long long *counters = nullptr;  // kCounters totals (DPCS_COUNTERS build)
    bool timing = false;
    int32_t visit_cap = 0;  // debug override of the traversal visit cap
    std::vector<TimedLaunch> timed;
    size_t n_timed = 0;
};

namespace {

// NVTX range around an entry point: visible in Nsight tools, free when no
// tool is attached
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

dpcs_status fail(dpcs_ctx *c, dpcs_status code, const std::string &msg) {
    if (c) c->err = msg;
    return code;
}

dpcs_status cuda_fail(dpcs_ctx *c, cudaError_t e, const char *what) {
    return fail(c, DPCS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

dpcs_status dev_alloc(dpcs_ctx *c, void **p, size_t bytes, const char *what) {
    if (c->budget && c->used + bytes > c->budget)
        return fail(c, DPCS_ERR_OOM, std::string(what) + ": HBM budget exceeded");
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, DPCS_ERR_OOM, std::string(what) + ": cudaMalloc failed");
    }
    c->used += bytes;
    return DPCS_OK;
}

void dev_free(dpcs_ctx *c, void *p, size_t bytes) {
    if (p) {
        cudaFree(p);
        c->used -= bytes;
    }
}

// grow-only scratch buffer
dpcs_status ensure(dpcs_ctx *c, Buf &b, size_t bytes, const char *what) {
    if (b.n >= bytes) return DPCS_OK;
    if (b.p) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(c, e, what);
        dev_free(c, b.p, b.n);
        b.p = nullptr;
        b.n = 0;
    }
    dpcs_status s = dev_alloc(c, &b.p, bytes, what);
    if (s == DPCS_OK) b.n = bytes;
    return s;
}

dpcs_status set_device(dpcs_ctx *c) {
    cudaError_t e = cudaSetDevice(c->device);
    return e == cudaSuccess ? DPCS_OK : cuda_fail(c, e, "cudaSetDevice");
}

dpcs_status check_launch(dpcs_ctx *c, int n, const char *what) {
    if (n < 0) return fail(c, n, std::string(what) + ": launch rejected");
    c->launches += (uint64_t)n;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DPCS_OK : cuda_fail(c, e, what);
}

// Gradient accumulators of one adjoint call (dEp always, dtex when a texture
// gradient is wanted): packed float4, or FP64 in the FP64 accumulation mode.
// Zeroes them on `st` and points the kernel arguments at them.
dpcs_status grad_setup(dpcs_ctx *c, int64_t np, int64_t nt, bool want_tex, cudaStream_t st, RenderArgs &a) {
    dpcs_status s;
    a.dEp = nullptr;
    a.dtex = nullptr;
    a.dEp64 = nullptr;
    a.dtex64 = nullptr;
    if (c->grad_f64) {
        if ((s = ensure(c, c->dEp64, (size_t)np * 24, "dEp FP64 accumulators")) ||
            (want_tex && (s = ensure(c, c->dtex64, (size_t)nt * 32, "dtex FP64 accumulators"))))
            return s;
        cudaMemsetAsync(c->dEp64.p, 0, (size_t)np * 24, st);
        if (want_tex) cudaMemsetAsync(c->dtex64.p, 0, (size_t)nt * 32, st);
        a.dEp64 = (double *)c->dEp64.p;
        a.dtex64 = want_tex ? (double *)c->dtex64.p : nullptr;
        return DPCS_OK;
    }
    if ((s = ensure(c, c->dEp4, (size_t)np * 16, "dEp scratch")) ||
        (want_tex && (s = ensure(c, c->dtex4, (size_t)nt * 16, "dtex scratch"))))
        return s;
    cudaMemsetAsync(c->dEp4.p, 0, (size_t)np * 16, st);
    if (want_tex) cudaMemsetAsync(c->dtex4.p, 0, (size_t)nt * 16, st);
    a.dEp = (float4 *)c->dEp4.p;
    a.dtex = want_tex ? (float4 *)c->dtex4.p : nullptr;
    return DPCS_OK;
}

// Eq. 1 adjoint and the texture gradients from the accumulators grad_setup
// chose; returns the kernels enqueued
int grad_finish(const RenderArgs &a, const float *Ip, int64_t np, int64_t nt, const dpcs_params *params, float *dIp,
                float *dAlbedo, float *dRough, double *acc, cudaStream_t st) {
    int nl;
    if (a.dEp64) {
        nl = launch_prf_backward64(Ip, a.dEp64, np, params->gamma_p, params->gain_p, dIp, acc, st);
        if (a.dtex64) nl += launch_tex_backward64(a.dtex64, nt, dAlbedo, dRough, st);
    } else {
        nl = launch_prf_backward(Ip, a.dEp, np, params->gamma_p, params->gain_p, dIp, acc, st);
        if (a.dtex) nl += launch_tex_backward(a.dtex, nt, dAlbedo, dRough, st);
    }
    return nl;
}

// events around a path-tracing kernel when timing is on
TimedLaunch *timing_begin(dpcs_ctx *c, int kernel, cudaStream_t st) {
    if (!c->timing) return nullptr;
    if (c->n_timed == c->timed.size()) {
        TimedLaunch t;
        if (cudaEventCreate(&t.a) != cudaSuccess || cudaEventCreate(&t.b) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        c->timed.push_back(t);
    }
    TimedLaunch *t = &c->timed[c->n_timed++];
    t->kernel = kernel;
    cudaEventRecord(t->a, st);
    return t;
}

void timing_end(TimedLaunch *t, cudaStream_t st) {
    if (t) cudaEventRecord(t->b, st);
}

bool finite_all(const float *v, int n) {
    for (int i = 0; i < n; ++i)
        if (!isfinite(v[i])) return false;
    return true;
}

void inv3(const float *Mf, float *R) {
    double M[9];
    for (int i = 0; i < 9; ++i) M[i] = Mf[i];
    const double a = M[0], b = M[1], cc = M[2], d = M[3], e = M[4], f = M[5], g = M[6], h = M[7], i = M[8];
    const double A = e * i - f * h, B = -(d * i - f * g), C = d * h - e * g;
    const double det = a * A + b * B + cc * C;
    const double r[9] = {A / det, -(b * i - cc * h) / det, (b * f - cc * e) / det,
                         B / det, (a * i - cc * g) / det,  -(a * f - cc * d) / det,
                         C / det, -(a * h - b * g) / det,  (a * e - b * d) / det};
    for (int k = 0; k < 9; ++k) R[k] = (float)r[k];
}

double det3(const float *M) {
    return (double)M[0] * ((double)M[4] * M[8] - (double)M[5] * M[7]) -
           (double)M[1] * ((double)M[3] * M[8] - (double)M[5] * M[6]) +
           (double)M[2] * ((double)M[3] * M[7] - (double)M[4] * M[6]);
}

// shared validation + argument packing of render and render_backward
dpcs_status prepare(dpcs_ctx *c, dpcs_scene scene, const float *albedo, const float *rough, int32_t Ht, int32_t Wt,
                    const float *Ip, const dpcs_view *view, const dpcs_params *prm, int32_t spp, int32_t bounces,
                    uint64_t seed, RenderArgs &a, Scene **sc_out) {
    if (!c) return DPCS_ERR_INVALID_ARG;
    auto it = c->scenes.find(scene);
    if (it == c->scenes.end()) return fail(c, DPCS_ERR_NOT_FOUND, "unknown scene handle");
    if (!albedo || !rough || !Ip || !view || !prm) return fail(c, DPCS_ERR_INVALID_ARG, "null input pointer");
    if (Ht <= 0 || Wt <= 0) return fail(c, DPCS_ERR_INVALID_ARG, "texture size must be positive");
    if (view->Hc <= 0 || view->Wc <= 0 || view->Hp <= 0 || view->Wp <= 0)
        return fail(c, DPCS_ERR_INVALID_ARG, "camera and projector sizes must be positive");
    if ((int64_t)view->Hc * view->Wc > (int64_t)1 << 30)
        return fail(c, DPCS_ERR_INVALID_ARG, "camera image too large (max 2^30 pixels)");
    if (spp < 1 || spp > (1 << 24)) return fail(c, DPCS_ERR_INVALID_ARG, "spp must be in [1, 2^24]");
    if (bounces < 0 || bounces > DPCS_MAX_BOUNCES) return fail(c, DPCS_ERR_INVALID_ARG, "bounces out of range");
    if (!finite_all(view->Kc, 9) || !finite_all(view->Kp, 9) || !finite_all(view->Rp, 9) || !finite_all(view->tp, 3))
        return fail(c, DPCS_ERR_INVALID_ARG, "non-finite camera or projector matrix");
    if (fabs(det3(view->Kc)) < 1e-12) return fail(c, DPCS_ERR_INVALID_ARG, "singular Kc");
    const float *pf = &prm->gamma_p[0];  // gamma_p .. f0: 14 consecutive floats
    if (!finite_all(pf, 14) || !isfinite(prm->rr_q) || !isfinite(prm->clip))
        return fail(c, DPCS_ERR_INVALID_ARG, "non-finite parameter");
    if (prm->rr_start < 0 || (prm->rr_start > 0 && !(prm->rr_q > 0.0f && prm->rr_q <= 1.0f)))
        return fail(c, DPCS_ERR_INVALID_ARG, "Russian roulette needs rr_start >= 0 and 0 < rr_q <= 1");
    if (prm->clip < 0.0f || prm->ks < 0.0f) return fail(c, DPCS_ERR_INVALID_ARG, "clip and ks must be >= 0");
    Scene &sc = it->second;
    memset(&a, 0, sizeof a);
    a.nodes = sc.nodes;
    a.tris = sc.tris;
    a.tuv = sc.tuv;
    a.root = sc.root;
    a.T = sc.T;
    a.Ht = Ht;
    a.Wt = Wt;
    a.Hp = view->Hp;
    a.Wp = view->Wp;
    a.Hc = view->Hc;
    a.Wc = view->Wc;
    inv3(view->Kc, a.Kci);
    memcpy(a.Kp, view->Kp, sizeof a.Kp);
    memcpy(a.Rp, view->Rp, sizeof a.Rp);
    memcpy(a.tp, view->tp, sizeof a.tp);
    for (int i = 0; i < 3; ++i)  // projector centre -Rp^T tp
        a.cp[i] = (float)-((double)view->Rp[i] * view->tp[0] + (double)view->Rp[3 + i] * view->tp[1] +
                           (double)view->Rp[6 + i] * view->tp[2]);
    memcpy(a.gamma_c, prm->gamma_c, sizeof a.gamma_c);
    a.gain_c = prm->gain_c;
    memcpy(a.wb, prm->wb, sizeof a.wb);
    a.k_proj = prm->k_proj;
    a.ks = prm->ks;
    a.f0 = prm->f0;
    a.rr_q = prm->rr_q;
    a.clip = prm->clip;
    a.rr_start = prm->rr_start;
    a.jitter = prm->jitter ? 1 : 0;
    a.spp = spp;
    a.bounces = bounces;
    a.key0 = (uint32_t)(seed & 0xffffffffu);
    a.key1 = (uint32_t)(seed >> 32);
    // lanes per pixel: the largest power of two L <= 32 with spp / L >= kMinSamplesPerLane
    // (at least 1)
    int l2 = 0;
    while (l2 < 5 && (2 << l2) * kMinSamplesPerLane <= spp) ++l2;
    a.log2L = l2;
    a.status = c->status;
    a.visit_cap = c->visit_cap;
#ifdef DPCS_COUNTERS
    a.counters = c->counters;
#else
    a.counters = nullptr;
#endif
    *sc_out = &sc;
    return DPCS_OK;
}

// The scene's mesh edges for the pose gradient's silhouette term, built on
// the host at the first call that needs them (the edges depend only on the
// triangles' vertex indices, which updates and rigid transforms keep).  Each
// triangle adds its three edges as (lower vertex, higher vertex, third
// vertex); sorted, each run of equal (lower, higher) is one edge, numbered in
// that order.  Synchronises the stream once.
dpcs_status pose_edges(dpcs_ctx *c, dpcs_scene scene, const Scene &sc, cudaStream_t st, const EdgeTable **out) {
    auto it = c->edges.find(scene);
    if (it != c->edges.end()) {
        *out = &it->second;
        return DPCS_OK;
    }
    const int64_t T = sc.T;
    std::vector<int32_t> vidx((size_t)(3 * T)), order((size_t)T), pos((size_t)T);
    cudaError_t e = cudaMemcpyAsync(vidx.data(), sc.vidx, (size_t)T * 12, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(order.data(), sc.order, (size_t)T * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "pose edges: reading the mesh");
    for (int64_t p = 0; p < T; ++p) {
        if (order[p] < 0 || order[p] >= T) return fail(c, DPCS_ERR_DEVICE_CHECK, "pose edges: corrupt leaf order");
        pos[order[p]] = (int32_t)p;
    }
    struct Half {
        int32_t lo, hi, third, tri;
        int8_t clo, chi, cth;
    };
    std::vector<Half> h((size_t)(3 * T));
    for (int64_t i = 0; i < T; ++i)
        for (int k = 0; k < 3; ++k) {
            const int ka = k, kb = (k + 1) % 3, kc = (k + 2) % 3;
            const int32_t va = vidx[3 * i + ka], vb = vidx[3 * i + kb];
            Half &r = h[(size_t)(3 * i + k)];
            const bool sw = vb < va;
            r.lo = sw ? vb : va;
            r.hi = sw ? va : vb;
            r.clo = (int8_t)(sw ? kb : ka);
            r.chi = (int8_t)(sw ? ka : kb);
            r.third = vidx[3 * i + kc];
            r.cth = (int8_t)kc;
            r.tri = (int32_t)i;
        }
    std::sort(h.begin(), h.end(), [](const Half &x, const Half &y) {
        if (x.lo != y.lo) return x.lo < y.lo;
        if (x.hi != y.hi) return x.hi < y.hi;
        return x.third < y.third;
    });
    std::vector<PoseEdge> E;
    E.reserve(h.size());
    for (size_t g = 0; g < h.size();) {
        size_t g1 = g + 1;
        while (g1 < h.size() && h[g1].lo == h[g].lo && h[g1].hi == h[g].hi) ++g1;
        PoseEdge r = make_int4(-1, 0, -1, 0);
        if (g1 - g <= 2) {
            const Half &A = h[g];
            r.x = pos[A.tri];
            r.y = A.clo | (A.chi << 2) | (A.cth << 4);
            if (g1 - g == 2) {
                r.z = pos[h[g + 1].tri];
                r.w = h[g + 1].cth;
            }
        }
        E.push_back(r);
        g = g1;
    }
    EdgeTable tab;
    tab.n = (int64_t)E.size();
    const size_t bytes = (size_t)(tab.n > 0 ? tab.n : 1) * sizeof(PoseEdge);
    dpcs_status s = dev_alloc(c, (void **)&tab.d, bytes, "pose edges");
    if (s) return s;
    e = tab.n > 0 ? cudaMemcpy(tab.d, E.data(), (size_t)tab.n * sizeof(PoseEdge), cudaMemcpyHostToDevice) : cudaSuccess;
    if (e != cudaSuccess) {
        dev_free(c, tab.d, bytes);
        return cuda_fail(c, e, "pose edges: upload");
    }
    *out = &(c->edges[scene] = tab);
    return DPCS_OK;
}

}  // namespace

extern "C" {

dpcs_status dpcs_create(int device, size_t hbm_budget_bytes, dpcs_ctx **out) {
    if (!out) return DPCS_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return DPCS_ERR_INVALID_ARG;
    }
    dpcs_ctx *c = new dpcs_ctx();
    c->device = device;
    c->budget = hbm_budget_bytes;
    dpcs_status s = set_device(c);
    if (s == DPCS_OK) s = dev_alloc(c, (void **)&c->status, sizeof(unsigned), "status word");
    if (s == DPCS_OK && cudaMemset(c->status, 0, sizeof(unsigned)) != cudaSuccess) s = DPCS_ERR_CUDA;
    if (s == DPCS_OK) s = dev_alloc(c, (void **)&c->counters, kCounters * sizeof(unsigned long long), "counters");
    if (s == DPCS_OK && cudaMemset(c->counters, 0, kCounters * sizeof(unsigned long long)) != cudaSuccess)
        s = DPCS_ERR_CUDA;
    if (s != DPCS_OK) {
        delete c;
        return s;
    }
    *out = c;
    return DPCS_OK;
}

dpcs_status dpcs_destroy(dpcs_ctx *c) {
    if (!c) return DPCS_ERR_INVALID_ARG;
    set_device(c);
    cudaDeviceSynchronize();
    for (auto &kv : c->scenes) {
        Scene &s = kv.second;
        cudaFree(s.nodes);
        cudaFree(s.tris);
        cudaFree(s.tuv);
        cudaFree(s.codes);
        cudaFree(s.order);
        cudaFree(s.vidx);
        cudaFree(s.uv);
        cudaFree(s.base);
    }
    for (auto &kv : c->edges) cudaFree(kv.second.d);
    Buf *bufs[] = {&c->ep4, &c->tex4, &c->gE, &c->dEp4, &c->dtex4, &c->acc, &c->partial, &c->build, &c->upload, &c->pix,
                   &c->kept, &c->mat4, &c->dmat4, &c->dEp64, &c->dtex64, &c->wf, &c->pose, &c->ploc};
    for (Buf *b : bufs)
        if (b->p) cudaFree(b->p);
    cudaFree(c->status);
    cudaFree(c->counters);
    for (TimedLaunch &t : c->timed) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    delete c;
    return DPCS_OK;
}

dpcs_status dpcs_timing_enable(dpcs_ctx *c, int32_t on) {
    if (!c) return DPCS_ERR_INVALID_ARG;
    dpcs_status s = set_device(c);
    if (s) return s;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(c, e, "timing_enable");
    c->timing = on != 0;
    if (on) c->n_timed = 0;
    return DPCS_OK;
}

dpcs_status dpcs_timing_read(dpcs_ctx *c, int32_t kernel, double *total_ms, int64_t *launches) {
    if (!c || !total_ms || !launches) return DPCS_ERR_INVALID_ARG;
    dpcs_status s = set_device(c);
    if (s) return s;
    double tot = 0.0;
    int64_t n = 0;
    for (size_t i = 0; i < c->n_timed; ++i) {
        TimedLaunch &t = c->timed[i];
        if (t.kernel != kernel) continue;
        cudaError_t e = cudaEventSynchronize(t.b);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t.a, t.b);
        if (e != cudaSuccess) return cuda_fail(c, e, "timing_read");
        tot += ms;
        ++n;
    }
    *total_ms = tot;
    *launches = n;
    return DPCS_OK;
}

dpcs_status dpcs_set_render_path(dpcs_ctx *c, int32_t path, int64_t chunk) {
    if (!c) return DPCS_ERR_INVALID_ARG;
    if (path != DPCS_PATH_MEGAKERNEL && path != DPCS_PATH_WAVEFRONT)
        return fail(c, DPCS_ERR_INVALID_ARG, "render path must be DPCS_PATH_MEGAKERNEL or DPCS_PATH_WAVEFRONT");
    if (chunk != 0 && (chunk < 4096 || chunk > (int64_t(1) << 28) || chunk % 32 != 0))
        return fail(c, DPCS_ERR_INVALID_ARG, "wavefront chunk must be 0 or a multiple of 32 in [4096, 2^28]");
    c->render_path = path;
    if (chunk) c->wf_chunk = chunk;
    return DPCS_OK;
}

dpcs_status dpcs_set_grad_accum(dpcs_ctx *c, int32_t mode) {
    if (!c) return DPCS_ERR_INVALID_ARG;
    if (mode != DPCS_ACCUM_F32 && mode != DPCS_ACCUM_F64)
        return fail(c, DPCS_ERR_INVALID_ARG, "grad accumulation mode must be DPCS_ACCUM_F32 or DPCS_ACCUM_F64");
    c->grad_f64 = mode == DPCS_ACCUM_F64;
    return DPCS_OK;
}

dpcs_status dpcs_set_bvh_builder(dpcs_ctx *c, int32_t builder) {
    if (!c) return DPCS_ERR_INVALID_ARG;
    if (builder != DPCS_BVH_LBVH && builder != DPCS_BVH_PLOC) return fail(c, DPCS_ERR_INVALID_ARG, "unknown BVH builder");
    c->bvh_builder = builder;
    return DPCS_OK;
}

dpcs_status dpcs_debug_set_visit_cap(dpcs_ctx *c, int32_t cap) {
    if (!c || cap < 0) return DPCS_ERR_INVALID_ARG;
    c->visit_cap = cap;
    return DPCS_OK;
}

dpcs_status dpcs_counters_read(dpcs_ctx *c, uint64_t *out, int32_t reset) {
    if (!c || !out) return DPCS_ERR_INVALID_ARG;
#ifndef DPCS_COUNTERS
    (void)reset;
    return fail(c, DPCS_ERR_INVALID_ARG, "library built without DPCS_COUNTERS");
#else
    dpcs_status s = set_device(c);
    if (s) return s;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(out, c->counters, kCounters * sizeof(uint64_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && reset) e = cudaMemset(c->counters, 0, kCounters * sizeof(unsigned long long));
    return e == cudaSuccess ? DPCS_OK : cuda_fail(c, e, "counters_read");
#endif
}

const char *dpcs_last_error(const dpcs_ctx *c) { return c ? c->err.c_str() : "null context"; }

size_t dpcs_memory_used(const dpcs_ctx *c) { return c ? c->used : 0; }

uint64_t dpcs_launch_count(const dpcs_ctx *c) { return c ? c->launches : 0; }

dpcs_status dpcs_sync(dpcs_ctx *c, void *stream) {
    if (!c) return DPCS_ERR_INVALID_ARG;
    dpcs_status s = set_device(c);
    if (s) return s;
    unsigned h = 0;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(&h, c->status, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "dpcs_sync");
    if (h) {
        cudaMemsetAsync(c->status, 0, sizeof(unsigned), st);
        cudaStreamSynchronize(st);
        if (h & kStatusTraversalLimit) return fail(c, DPCS_ERR_TRAVERSAL_LIMIT, "BVH traversal hit its limit");
        return fail(c, DPCS_ERR_DEVICE_CHECK, "a device bounds check failed");
    }
    return DPCS_OK;
}

dpcs_status dpcs_scene_upload(dpcs_ctx *c, const float *verts, int32_t V, const int32_t *tris, int32_t T,
                              const float *uv, void *stream, dpcs_scene *out) {
    Range range("dpcs_scene_upload");
    if (!c || !out) return DPCS_ERR_INVALID_ARG;
    if (T < 0 || V < 0 || (T > 0 && (!verts || !tris || !uv || V == 0)))
        return fail(c, DPCS_ERR_INVALID_ARG, "bad mesh arrays");
    if (T > (1 << 28)) return fail(c, DPCS_ERR_INVALID_ARG, "too many triangles");
    for (int64_t i = 0; i < 3 * (int64_t)T; ++i)
        if (tris[i] < 0 || tris[i] >= V) return fail(c, DPCS_ERR_INVALID_ARG, "triangle index out of range");
    for (int64_t i = 0; i < 3 * (int64_t)V; ++i)
        if (!isfinite(verts[i])) return fail(c, DPCS_ERR_INVALID_ARG, "non-finite vertex");
    dpcs_status s = set_device(c);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    Scene sc;
    sc.T = T;
    const size_t n = (size_t)(T > 0 ? T : 1);
    const size_t nn = (size_t)(T > 1 ? T - 1 : 1);
    const size_t nv = (size_t)(V > 0 ? V : 1);
    sc.V = V;
    sc.bytes = nn * 64 + n * 48 + n * 24 + n * 8 + n * 12 + nv * 8 + nv * 12;
    // frees what the scene holds, for every failure after its allocation
    auto release = [&]() {
        if (sc.nodes || sc.tris) cudaStreamSynchronize(st);  // kernels of a failed build may still use them
        dev_free(c, sc.nodes, sc.nodes ? nn * 64 : 0);
        dev_free(c, sc.tris, sc.tris ? n * 48 : 0);
        dev_free(c, sc.tuv, sc.tuv ? n * 24 : 0);
        dev_free(c, sc.codes, sc.codes ? n * 4 : 0);
        dev_free(c, sc.order, sc.order ? n * 4 : 0);
        dev_free(c, sc.vidx, sc.vidx ? n * 12 : 0);
        dev_free(c, sc.uv, sc.uv ? nv * 8 : 0);
        dev_free(c, sc.base, sc.base ? nv * 12 : 0);
    };
    if ((s = dev_alloc(c, (void **)&sc.nodes, nn * 64, "scene nodes")) ||
        (s = dev_alloc(c, (void **)&sc.tris, n * 48, "scene triangles")) ||
        (s = dev_alloc(c, (void **)&sc.tuv, n * 24, "scene uv")) ||
        (s = dev_alloc(c, (void **)&sc.codes, n * 4, "scene codes")) ||
        (s = dev_alloc(c, (void **)&sc.order, n * 4, "scene order")) ||
        (s = dev_alloc(c, (void **)&sc.vidx, n * 12, "scene vertex indices")) ||
        (s = dev_alloc(c, (void **)&sc.uv, nv * 8, "scene vertex uv")) ||
        (s = dev_alloc(c, (void **)&sc.base, nv * 12, "scene vertex positions"))) {
        release();
        return s;
    }
    if (T > 0) {
        const size_t vb = (size_t)V * 12, tb = (size_t)T * 12, ub = (size_t)V * 8;
        const size_t up = ((vb + 255) & ~size_t(255)) + ((tb + 255) & ~size_t(255)) + ub;
        if ((s = ensure(c, c->upload, up, "upload staging")) ||
            (s = ensure(c, c->build, lbvh_scratch_bytes(T), "LBVH scratch"))) {
            release();
            return s;
        }
        char *p = (char *)c->upload.p;
        float *dv = (float *)p;
        int32_t *dt = (int32_t *)(p + ((vb + 255) & ~size_t(255)));
        float *du = (float *)(p + ((vb + 255) & ~size_t(255)) + ((tb + 255) & ~size_t(255)));
        cudaError_t e = cudaMemcpyAsync(dv, verts, vb, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dt, tris, tb, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(du, uv, ub, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            release();
            return cuda_fail(c, e, "scene upload");
        }
        int nl = launch_lbvh_build(dv, V, dt, T, du, sc, c->build.p, c->build.n, st);
        if ((s = check_launch(c, nl, "LBVH build"))) {
            release();
            return s;
        }
        // the clustering is an optimisation: if it cannot have its scratch
        // memory or a round's check fails, the radix tree stays (its nodes
        // are replaced only at the end of a successful build)
        if (c->bvh_builder == DPCS_BVH_PLOC && T >= 3 &&
            ensure(c, c->ploc, ploc_scratch_bytes(T), "PLOC scratch") == DPCS_OK) {
            int32_t depth = 0;
            const int np = launch_ploc(sc, c->ploc.p, c->ploc.n, kMaxTreeDepth, st, &depth);
            if (np == DPCS_ERR_CUDA) {
                release();
                return fail(c, DPCS_ERR_CUDA, "PLOC build: a CUDA call failed");
            }
            if (np > 0) c->launches += (uint64_t)np;
        }
        e = cudaMemcpyAsync(sc.vidx, dt, tb, cudaMemcpyDeviceToDevice, st);  // kept for dpcs_scene_update
        if (e == cudaSuccess) e = cudaMemcpyAsync(sc.uv, du, ub, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(sc.base, dv, vb, cudaMemcpyDeviceToDevice, st);  // rigid transforms
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            release();
            return cuda_fail(c, e, "LBVH build");
        }
    } else {
        sc.root = kEmptyRoot;
    }
    const uint64_t id = c->next_scene++;
    c->scenes[id] = sc;
    *out = id;
    return DPCS_OK;
}

dpcs_status dpcs_scene_free(dpcs_ctx *c, dpcs_scene scene) {
    if (!c) return DPCS_ERR_INVALID_ARG;
    auto it = c->scenes.find(scene);
    if (it == c->scenes.end()) return fail(c, DPCS_ERR_NOT_FOUND, "unknown scene handle");
    set_device(c);
    cudaDeviceSynchronize();
    Scene &s = it->second;
    const size_t n = (size_t)(s.T > 0 ? s.T : 1), nn = (size_t)(s.T > 1 ? s.T - 1 : 1);
    dev_free(c, s.nodes, nn * 64);
    dev_free(c, s.tris, n * 48);
    dev_free(c, s.tuv, n * 24);
    dev_free(c, s.codes, n * 4);
    dev_free(c, s.order, n * 4);
    dev_free(c, s.vidx, n * 12);
    dev_free(c, s.uv, (size_t)(s.V > 0 ? s.V : 1) * 8);
    dev_free(c, s.base, (size_t)(s.V > 0 ? s.V : 1) * 12);
    auto et = c->edges.find(scene);
    if (et != c->edges.end()) {
        dev_free(c, et->second.d, (size_t)(et->second.n > 0 ? et->second.n : 1) * sizeof(PoseEdge));
        c->edges.erase(et);
    }
    c->scenes.erase(it);
    return DPCS_OK;
}

dpcs_status dpcs_scene_update(dpcs_ctx *c, dpcs_scene scene, const float *verts, int32_t V, void *stream) {
    Range range("dpcs_scene_update");
    if (!c) return DPCS_ERR_INVALID_ARG;
    auto it = c->scenes.find(scene);
    if (it == c->scenes.end()) return fail(c, DPCS_ERR_NOT_FOUND, "unknown scene handle");
    Scene &sc = it->second;
    if (V != sc.V) return fail(c, DPCS_ERR_INVALID_ARG, "scene_update: vertex count differs from the upload");
    if (sc.T <= 0) return DPCS_OK;
    if (!verts) return fail(c, DPCS_ERR_INVALID_ARG, "scene_update: null vertices");
    for (int64_t i = 0; i < 3 * (int64_t)V; ++i)
        if (!isfinite(verts[i])) return fail(c, DPCS_ERR_INVALID_ARG, "scene_update: non-finite vertex");
    dpcs_status s = set_device(c);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t vb = (size_t)V * 12;
    if ((s = ensure(c, c->upload, vb, "upload staging")) ||
        (s = ensure(c, c->build, lbvh_refit_scratch_bytes(sc.T), "refit scratch")))
        return s;
    cudaError_t e = cudaMemcpyAsync(c->upload.p, verts, vb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sc.base, c->upload.p, vb, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "scene_update upload");
    return check_launch(c, launch_lbvh_refit((const float *)c->upload.p, sc, c->build.p, c->build.n, st),
                        "LBVH refit");
}

dpcs_status dpcs_scene_transform(dpcs_ctx *c, dpcs_scene scene, const float R[9], const float t[3], void *stream) {
    Range range("dpcs_scene_transform");
    if (!c) return DPCS_ERR_INVALID_ARG;
    auto it = c->scenes.find(scene);
    if (it == c->scenes.end()) return fail(c, DPCS_ERR_NOT_FOUND, "unknown scene handle");
    if (!R || !t || !finite_all(R, 9) || !finite_all(t, 3))
        return fail(c, DPCS_ERR_INVALID_ARG, "scene_transform: null or non-finite R or t");
    Scene &sc = it->second;
    if (sc.T <= 0) return DPCS_OK;
    dpcs_status s = set_device(c);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = ensure(c, c->upload, (size_t)sc.V * 12, "upload staging")) ||
        (s = ensure(c, c->build, lbvh_refit_scratch_bytes(sc.T), "refit scratch")))
        return s;
    int nl = launch_rigid_transform(sc.base, sc.V, R, t, (float *)c->upload.p, st);
    const int nr = launch_lbvh_refit((const float *)c->upload.p, sc, c->build.p, c->build.n, st);
    if (nr < 0) return check_launch(c, nr, "LBVH refit");
    return check_launch(c, nl + nr, "scene_transform");
}

dpcs_status dpcs_scene_export(dpcs_ctx *c, dpcs_scene scene, uint32_t *codes, int32_t *order, int32_t *child,
                              float *child_box) {
    if (!c) return DPCS_ERR_INVALID_ARG;
    auto it = c->scenes.find(scene);
    if (it == c->scenes.end()) return fail(c, DPCS_ERR_NOT_FOUND, "unknown scene handle");
    dpcs_status s = set_device(c);
    if (s) return s;
    Scene &sc = it->second;
    const int T = sc.T;
    if (T <= 0) return DPCS_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess && codes) e = cudaMemcpy(codes, sc.codes, (size_t)T * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && order) e = cudaMemcpy(order, sc.order, (size_t)T * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && T >= 2 && (child || child_box)) {
        float *h = new float[(size_t)(T - 1) * 16];
        e = cudaMemcpy(h, sc.nodes, (size_t)(T - 1) * 64, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            for (int i = 0; i < T - 1; ++i) {
                const float *nd = h + 16 * i;
                if (child) {
                    memcpy(&child[2 * i], &nd[12], 4);
                    memcpy(&child[2 * i + 1], &nd[13], 4);
                }
                if (child_box) {
                    float *bl = child_box + 12 * i, *br = bl + 6;
                    bl[0] = nd[0]; bl[1] = nd[2]; bl[2] = nd[8]; bl[3] = nd[1]; bl[4] = nd[3]; bl[5] = nd[9];
                    br[0] = nd[4]; br[1] = nd[6]; br[2] = nd[10]; br[3] = nd[5]; br[4] = nd[7]; br[5] = nd[11];
                }
            }
        delete[] h;
    }
    return e == cudaSuccess ? DPCS_OK : cuda_fail(c, e, "scene export");
}

dpcs_status dpcs_trace(dpcs_ctx *c, dpcs_scene scene, const float *orig, const float *dir, int64_t n, float *t_out,
                       int32_t *tri_out, void *stream) {
    Range range("dpcs_trace");
    if (!c) return DPCS_ERR_INVALID_ARG;
    auto it = c->scenes.find(scene);
    if (it == c->scenes.end()) return fail(c, DPCS_ERR_NOT_FOUND, "unknown scene handle");
    if (n < 0 || (n > 0 && (!orig || !dir || !t_out || !tri_out)))
        return fail(c, DPCS_ERR_INVALID_ARG, "bad trace arguments");
    if (n == 0) return DPCS_OK;
    dpcs_status s = set_device(c);
    if (s) return s;
    return check_launch(c, launch_trace(it->second, orig, dir, n, t_out, tri_out, c->status, (cudaStream_t)stream),
                        "trace");
}

dpcs_status dpcs_render(dpcs_ctx *c, dpcs_scene scene, const float *albedo, const float *rough, int32_t Ht,
                        int32_t Wt, const float *Ip, const dpcs_view *view, const dpcs_params *params, int32_t spp,
                        int32_t bounces, uint64_t seed, float *Ic, float *Ec, void *stream) {
    Range range("dpcs_render");
    RenderArgs a;
    Scene *sc = nullptr;
    dpcs_status s = prepare(c, scene, albedo, rough, Ht, Wt, Ip, view, params, spp, bounces, seed, a, &sc);
    if (s) return s;
    if (!Ic) return fail(c, DPCS_ERR_INVALID_ARG, "null Ic");
    if ((s = set_device(c))) return s;
    const int64_t np = (int64_t)view->Hp * view->Wp, nt = (int64_t)Ht * Wt;
    if ((s = ensure(c, c->ep4, (size_t)np * 16, "Ep scratch")) || (s = ensure(c, c->tex4, (size_t)nt * 16, "texture scratch")))
        return s;
    const bool wf = c->render_path == DPCS_PATH_WAVEFRONT;
    const size_t wf_bytes = wf ? wavefront_scratch_bytes(a, c->wf_chunk) : 0;
    if (wf && (s = ensure(c, c->wf, wf_bytes, "wavefront scratch"))) return s;
    cudaStream_t st = (cudaStream_t)stream;
    a.Ep = (const float4 *)c->ep4.p;
    a.tex = (const float4 *)c->tex4.p;
    a.Ic = Ic;
    a.Ec = Ec;
    int nl = launch_prf(Ip, np, params->gamma_p, params->gain_p, (float4 *)c->ep4.p, st);
    nl += launch_pack_tex(albedo, rough, nt, (float4 *)c->tex4.p, st);
    TimedLaunch *tl = timing_begin(c, 0, st);
    nl += wf ? launch_render_wavefront(a, c->wf_chunk, c->wf.p, st) : launch_render(a, st);
    timing_end(tl, st);
    return check_launch(c, nl, "render");
}

dpcs_status dpcs_render_backward(dpcs_ctx *c, dpcs_scene scene, const float *albedo, const float *rough,
                                 int32_t Ht, int32_t Wt, const float *Ip, const dpcs_view *view,
                                 const dpcs_params *params, int32_t spp, int32_t bounces, uint64_t seed,
                                 const float *Ec, const float *Ic, const float *dIc, float *dIp, float *dAlbedo,
                                 float *dRough, float *dParams, void *stream) {
    Range range("dpcs_render_backward");
    RenderArgs a;
    Scene *sc = nullptr;
    dpcs_status s = prepare(c, scene, albedo, rough, Ht, Wt, Ip, view, params, spp, bounces, seed, a, &sc);
    if (s) return s;
    if (!Ec || !Ic || !dIc) return fail(c, DPCS_ERR_INVALID_ARG, "null Ec, Ic or dIc");
    if ((s = set_device(c))) return s;
    const int64_t np = (int64_t)view->Hp * view->Wp, nt = (int64_t)Ht * Wt, npix = (int64_t)view->Hc * view->Wc;
    if ((s = ensure(c, c->ep4, (size_t)np * 16, "Ep scratch")) ||
        (s = ensure(c, c->tex4, (size_t)nt * 16, "texture scratch")) ||
        (s = ensure(c, c->gE, (size_t)npix * 12, "dEc scratch")) ||
        (s = ensure(c, c->acc, 16 * sizeof(double), "parameter accumulators")))
        return s;
    const bool want_tex = dAlbedo || dRough;  // otherwise the replay skips the texture scatters
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = grad_setup(c, np, nt, want_tex, st, a))) return s;
    double *acc = (double *)c->acc.p;
    cudaMemsetAsync(acc, 0, 16 * sizeof(double), st);
    int nl = launch_prf(Ip, np, params->gamma_p, params->gain_p, (float4 *)c->ep4.p, st);
    nl += launch_pack_tex(albedo, rough, nt, (float4 *)c->tex4.p, st);
    nl += launch_crf_backward(dIc, Ec, Ic, npix, params->gamma_c, params->gain_c, params->wb, (float *)c->gE.p, acc, st);
    a.Ep = (const float4 *)c->ep4.p;
    a.tex = (const float4 *)c->tex4.p;
    a.gE = (const float *)c->gE.p;
    TimedLaunch *tl = timing_begin(c, 1, st);
    nl += launch_replay(a, st);
    timing_end(tl, st);
    nl += grad_finish(a, Ip, np, nt, params, dIp, dAlbedo, dRough, acc, st);
    if (dParams) nl += launch_finalize_params(acc, dParams, st);
    return check_launch(c, nl, "render_backward");
}

dpcs_status dpcs_render_principled(dpcs_ctx *c, dpcs_scene scene, const dpcs_material *mat, const float *Ip,
                                   const dpcs_view *view, const dpcs_params *params, int32_t spp, int32_t bounces,
                                   uint64_t seed, float *Ic, float *Ec, void *stream) {
    Range range("dpcs_render_principled");
    if (!c) return DPCS_ERR_INVALID_ARG;
    if (!mat) return fail(c, DPCS_ERR_INVALID_ARG, "null material");
    RenderArgs a;
    Scene *sc = nullptr;
    dpcs_status s = prepare(c, scene, mat->albedo, mat->rough, mat->Ht, mat->Wt, Ip, view, params, spp, bounces, seed,
                            a, &sc);
    if (s) return s;
    if (!Ic) return fail(c, DPCS_ERR_INVALID_ARG, "null Ic");
    if ((s = set_device(c))) return s;
    const int64_t np = (int64_t)view->Hp * view->Wp, nt = (int64_t)mat->Ht * mat->Wt;
    if ((s = ensure(c, c->ep4, (size_t)np * 16, "Ep scratch")) ||
        (s = ensure(c, c->tex4, (size_t)nt * 16, "texture scratch")) ||
        (s = ensure(c, c->mat4, (size_t)nt * 16, "material scratch")))
        return s;
    cudaStream_t st = (cudaStream_t)stream;
    a.Ep = (const float4 *)c->ep4.p;
    a.tex = (const float4 *)c->tex4.p;
    a.Ic = Ic;
    a.Ec = Ec;
    int nl = launch_prf(Ip, np, params->gamma_p, params->gain_p, (float4 *)c->ep4.p, st);
    nl += launch_pack_tex(mat->albedo, mat->rough, nt, (float4 *)c->tex4.p, st);
    nl += launch_pack_mat(mat->metallic, mat->normal, nt, (float4 *)c->mat4.p, st);
    nl += launch_render_pbr(a, (const float4 *)c->mat4.p, st);
    return check_launch(c, nl, "render_principled");
}

dpcs_status dpcs_render_backward_principled(dpcs_ctx *c, dpcs_scene scene, const dpcs_material *mat, const float *Ip,
                                            const dpcs_view *view, const dpcs_params *params, int32_t spp,
                                            int32_t bounces, uint64_t seed, const float *Ec, const float *Ic,
                                            const float *dIc, float *dIp, float *dAlbedo, float *dRough,
                                            float *dMetallic, float *dNormal, float *dParams, void *stream) {
    Range range("dpcs_render_backward_principled");
    if (!c) return DPCS_ERR_INVALID_ARG;
    if (!mat) return fail(c, DPCS_ERR_INVALID_ARG, "null material");
    RenderArgs a;
    Scene *sc = nullptr;
    dpcs_status s = prepare(c, scene, mat->albedo, mat->rough, mat->Ht, mat->Wt, Ip, view, params, spp, bounces, seed,
                            a, &sc);
    if (s) return s;
    if (!Ec || !Ic || !dIc) return fail(c, DPCS_ERR_INVALID_ARG, "null Ec, Ic or dIc");
    if (dMetallic && !mat->metallic) return fail(c, DPCS_ERR_INVALID_ARG, "dMetallic given without a metallic map");
    if (dNormal && !mat->normal) return fail(c, DPCS_ERR_INVALID_ARG, "dNormal given without a normal map");
    if ((s = set_device(c))) return s;
    const int64_t np = (int64_t)view->Hp * view->Wp, nt = (int64_t)mat->Ht * mat->Wt;
    const int64_t npix = (int64_t)view->Hc * view->Wc;
    if ((s = ensure(c, c->ep4, (size_t)np * 16, "Ep scratch")) ||
        (s = ensure(c, c->tex4, (size_t)nt * 16, "texture scratch")) ||
        (s = ensure(c, c->mat4, (size_t)nt * 16, "material scratch")) ||
        (s = ensure(c, c->gE, (size_t)npix * 12, "dEc scratch")) ||
        (s = ensure(c, c->dEp4, (size_t)np * 16, "dEp scratch")) ||
        (s = ensure(c, c->acc, 16 * sizeof(double), "parameter accumulators")))
        return s;
    const bool want_tex = dAlbedo || dRough, want_mat = dMetallic || dNormal;
    if (want_tex && (s = ensure(c, c->dtex4, (size_t)nt * 16, "dtex scratch"))) return s;
    if (want_mat && (s = ensure(c, c->dmat4, (size_t)nt * 16, "dmat scratch"))) return s;
    cudaStream_t st = (cudaStream_t)stream;
    double *acc = (double *)c->acc.p;
    cudaMemsetAsync(acc, 0, 16 * sizeof(double), st);
    cudaMemsetAsync(c->dEp4.p, 0, (size_t)np * 16, st);
    if (want_tex) cudaMemsetAsync(c->dtex4.p, 0, (size_t)nt * 16, st);
    if (want_mat) cudaMemsetAsync(c->dmat4.p, 0, (size_t)nt * 16, st);
    int nl = launch_prf(Ip, np, params->gamma_p, params->gain_p, (float4 *)c->ep4.p, st);
    nl += launch_pack_tex(mat->albedo, mat->rough, nt, (float4 *)c->tex4.p, st);
    nl += launch_pack_mat(mat->metallic, mat->normal, nt, (float4 *)c->mat4.p, st);
    nl += launch_crf_backward(dIc, Ec, Ic, npix, params->gamma_c, params->gain_c, params->wb, (float *)c->gE.p, acc, st);
    a.Ep = (const float4 *)c->ep4.p;
    a.tex = (const float4 *)c->tex4.p;
    a.gE = (const float *)c->gE.p;
    a.dEp = (float4 *)c->dEp4.p;
    a.dtex = want_tex ? (float4 *)c->dtex4.p : nullptr;
    nl += launch_replay_pbr(a, (const float4 *)c->mat4.p, want_mat ? (float4 *)c->dmat4.p : nullptr, st);
    nl += launch_prf_backward(Ip, (const float4 *)c->dEp4.p, np, params->gamma_p, params->gain_p, dIp, acc, st);
    if (want_tex) nl += launch_tex_backward((const float4 *)c->dtex4.p, nt, dAlbedo, dRough, st);
    if (want_mat) nl += launch_mat_backward((const float4 *)c->dmat4.p, nt, dMetallic, dNormal, st);
    if (dParams) nl += launch_finalize_params(acc, dParams, st);
    return check_launch(c, nl, "render_backward_principled");
}

dpcs_status dpcs_render_keep(dpcs_ctx *c, dpcs_scene scene, const float *albedo, const float *rough, int32_t Ht,
                             int32_t Wt, const float *Ip, const dpcs_view *view, const dpcs_params *params,
                             int32_t spp, int32_t bounces, uint64_t seed, float *Ic, float *Ec, void *stream) {
    Range range("dpcs_render_keep");
    RenderArgs a;
    Scene *sc = nullptr;
    dpcs_status s = prepare(c, scene, albedo, rough, Ht, Wt, Ip, view, params, spp, bounces, seed, a, &sc);
    if (s) return s;
    if (!Ic) return fail(c, DPCS_ERR_INVALID_ARG, "null Ic");
    if ((s = set_device(c))) return s;
    const int64_t np = (int64_t)view->Hp * view->Wp, nt = (int64_t)Ht * Wt, npix = (int64_t)view->Hc * view->Wc;
    const int L = 1 << a.log2L;
    const int64_t nthr = npix << a.log2L, spl = (spp + L - 1) / L;
    const size_t words = (size_t)kRecWordsHost * spl * bounces * nthr * 4, counts = (size_t)spl * nthr;
    c->kept_key.valid = false;
    if ((s = ensure(c, c->ep4, (size_t)np * 16, "Ep scratch")) ||
        (s = ensure(c, c->tex4, (size_t)nt * 16, "texture scratch")) ||
        (s = ensure(c, c->kept, ((words + 255) & ~size_t(255)) + counts, "kept path records")))
        return s;
    cudaStream_t st = (cudaStream_t)stream;
    int nl = launch_prf(Ip, np, params->gamma_p, params->gain_p, (float4 *)c->ep4.p, st);
    nl += launch_pack_tex(albedo, rough, nt, (float4 *)c->tex4.p, st);
    a.Ep = (const float4 *)c->ep4.p;
    a.tex = (const float4 *)c->tex4.p;
    a.Ic = Ic;
    a.Ec = Ec;
    char *kp = (char *)c->kept.p;
    TimedLaunch *tl = timing_begin(c, 0, st);
    nl += launch_render_keep(a, kp, (uint8_t *)(kp + ((words + 255) & ~size_t(255))), st);
    timing_end(tl, st);
    if ((s = check_launch(c, nl, "render_keep"))) return s;
    c->kept_key.valid = true;
    c->kept_key.scene = scene;
    c->kept_key.seed = seed;
    c->kept_key.Hc = view->Hc;
    c->kept_key.Wc = view->Wc;
    c->kept_key.spp = spp;
    c->kept_key.bounces = bounces;
    c->kept_key.log2L = a.log2L;
    c->kept_key.principled = false;
    return DPCS_OK;
}

dpcs_status dpcs_render_backward_kept(dpcs_ctx *c, dpcs_scene scene, const float *albedo, const float *rough,
                                      int32_t Ht, int32_t Wt, const float *Ip, const dpcs_view *view,
                                      const dpcs_params *params, int32_t spp, int32_t bounces, uint64_t seed,
                                      const float *Ec, const float *Ic, const float *dIc, float *dIp, float *dAlbedo,
                                      float *dRough, float *dParams, void *stream) {
    Range range("dpcs_render_backward_kept");
    RenderArgs a;
    Scene *sc = nullptr;
    dpcs_status s = prepare(c, scene, albedo, rough, Ht, Wt, Ip, view, params, spp, bounces, seed, a, &sc);
    if (s) return s;
    if (!Ec || !Ic || !dIc) return fail(c, DPCS_ERR_INVALID_ARG, "null Ec, Ic or dIc");
    const auto &k = c->kept_key;
    if (!k.valid || k.principled || k.scene != scene || k.seed != seed || k.Hc != view->Hc || k.Wc != view->Wc ||
        k.spp != spp || k.bounces != bounces || k.log2L != a.log2L)
        return fail(c, DPCS_ERR_INVALID_ARG, "render_backward_kept: no kept render with these arguments");
    if ((s = set_device(c))) return s;
    const int64_t np = (int64_t)view->Hp * view->Wp, nt = (int64_t)Ht * Wt, npix = (int64_t)view->Hc * view->Wc;
    const int L = 1 << a.log2L;
    const int64_t nthr = npix << a.log2L, spl = (spp + L - 1) / L;
    const size_t words = (size_t)kRecWordsHost * spl * bounces * nthr * 4;
    if ((s = ensure(c, c->gE, (size_t)npix * 12, "dEc scratch")) ||
        (s = ensure(c, c->acc, 16 * sizeof(double), "parameter accumulators")))
        return s;
    const bool want_tex = dAlbedo || dRough;
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = grad_setup(c, np, nt, want_tex, st, a))) return s;
    double *acc = (double *)c->acc.p;
    cudaMemsetAsync(acc, 0, 16 * sizeof(double), st);
    int nl = launch_crf_backward(dIc, Ec, Ic, npix, params->gamma_c, params->gain_c, params->wb, (float *)c->gE.p, acc,
                                 st);
    a.gE = (const float *)c->gE.p;
    const char *kp = (const char *)c->kept.p;
    TimedLaunch *tl = timing_begin(c, 1, st);
    nl += launch_sweep_kept(a, kp, (const uint8_t *)(kp + ((words + 255) & ~size_t(255))), st);
    timing_end(tl, st);
    nl += grad_finish(a, Ip, np, nt, params, dIp, dAlbedo, dRough, acc, st);
    if (dParams) nl += launch_finalize_params(acc, dParams, st);
    return check_launch(c, nl, "render_backward_kept");
}

dpcs_status dpcs_render_loss_backward(dpcs_ctx *c, dpcs_scene scene, const float *albedo, const float *rough,
                                      int32_t Ht, int32_t Wt, const float *Ip, const dpcs_view *view,
                                      const dpcs_params *params, int32_t spp, int32_t bounces, uint64_t seed,
                                      const float *target, int32_t loss_kind, float scale, float *Ic, float *Ec,
                                      float *loss, float *dIp, float *dAlbedo, float *dRough, float *dParams,
                                      void *stream) {
    Range range("dpcs_render_loss_backward");
    RenderArgs a;
    Scene *sc = nullptr;
    dpcs_status s = prepare(c, scene, albedo, rough, Ht, Wt, Ip, view, params, spp, bounces, seed, a, &sc);
    if (s) return s;
    if (!target || !Ic || !loss) return fail(c, DPCS_ERR_INVALID_ARG, "null target, Ic or loss");
    if ((loss_kind != 0 && loss_kind != 1) || !(scale > 0.0f))
        return fail(c, DPCS_ERR_INVALID_ARG, "loss_kind must be 0 (L2) or 1 (L1) and scale > 0");
    if ((s = set_device(c))) return s;
    const int64_t np = (int64_t)view->Hp * view->Wp, nt = (int64_t)Ht * Wt, npix = (int64_t)view->Hc * view->Wc;
    const int L = 1 << a.log2L;
    const int spl = (spp + L - 1) / L;  // samples per lane
    const bool fused = spl <= kFusedSamples && spl * bounces <= kFusedRecs;
    const bool want_tex = dAlbedo || dRough;
    if ((s = ensure(c, c->ep4, (size_t)np * 16, "Ep scratch")) ||
        (s = ensure(c, c->tex4, (size_t)nt * 16, "texture scratch")) ||
        (s = ensure(c, c->acc, 16 * sizeof(double), "parameter accumulators")) ||
        (!fused && ((s = ensure(c, c->gE, (size_t)npix * 12, "dEc scratch")) ||
                    (s = ensure(c, c->pix, (size_t)npix * 24, "per-pixel loss scratch")))))
        return s;
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = grad_setup(c, np, nt, want_tex, st, a))) return s;
    double *acc = (double *)c->acc.p;
    cudaMemsetAsync(acc, 0, 16 * sizeof(double), st);
    int nl = launch_prf(Ip, np, params->gamma_p, params->gain_p, (float4 *)c->ep4.p, st);
    nl += launch_pack_tex(albedo, rough, nt, (float4 *)c->tex4.p, st);
    a.Ep = (const float4 *)c->ep4.p;
    a.tex = (const float4 *)c->tex4.p;
    a.Ic = Ic;
    const LossArgs l{target, scale, loss_kind, acc};
    if (fused) {
        a.Ec = Ec;
        TimedLaunch *tl = timing_begin(c, 0, st);
        nl += launch_render_grad(a, l, st);
        timing_end(tl, st);
    } else {  // render, per-pixel loss, Eq. 5 adjoint, replay
        float *dIc = (float *)c->pix.p, *ec = Ec ? Ec : (float *)c->pix.p + 3 * npix;
        a.Ec = ec;
        TimedLaunch *tl = timing_begin(c, 0, st);
        nl += launch_render(a, st);
        timing_end(tl, st);
        nl += launch_pixel_loss(Ic, npix * 3, l, dIc, st);
        nl += launch_crf_backward(dIc, ec, Ic, npix, params->gamma_c, params->gain_c, params->wb, (float *)c->gE.p,
                                  acc, st);
        a.gE = (const float *)c->gE.p;
        TimedLaunch *tr = timing_begin(c, 1, st);
        nl += launch_replay(a, st);
        timing_end(tr, st);
    }
    nl += launch_loss_out(acc, loss, st);
    nl += grad_finish(a, Ip, np, nt, params, dIp, dAlbedo, dRough, acc, st);
    if (dParams) nl += launch_finalize_params(acc, dParams, st);
    return check_launch(c, nl, "render_loss_backward");
}

dpcs_status dpcs_render_keep_principled(dpcs_ctx *c, dpcs_scene scene, const dpcs_material *mat, const float *Ip,
                                        const dpcs_view *view, const dpcs_params *params, int32_t spp,
                                        int32_t bounces, uint64_t seed, float *Ic, float *Ec, void *stream) {
    Range range("dpcs_render_keep_principled");
    if (!c) return DPCS_ERR_INVALID_ARG;
    if (!mat) return fail(c, DPCS_ERR_INVALID_ARG, "null material");
    RenderArgs a;
    Scene *sc = nullptr;
    dpcs_status s = prepare(c, scene, mat->albedo, mat->rough, mat->Ht, mat->Wt, Ip, view, params, spp, bounces, seed,
                            a, &sc);
    if (s) return s;
    if (!Ic) return fail(c, DPCS_ERR_INVALID_ARG, "null Ic");
    if ((s = set_device(c))) return s;
    const int64_t np = (int64_t)view->Hp * view->Wp, nt = (int64_t)mat->Ht * mat->Wt;
    const int64_t npix = (int64_t)view->Hc * view->Wc;
    const int L = 1 << a.log2L;
    const int64_t nthr = npix << a.log2L, spl = (spp + L - 1) / L;
    const size_t words = (size_t)kPRecWordsHost * spl * bounces * nthr * 4, counts = (size_t)spl * nthr;
    c->kept_key.valid = false;
    if ((s = ensure(c, c->ep4, (size_t)np * 16, "Ep scratch")) ||
        (s = ensure(c, c->tex4, (size_t)nt * 16, "texture scratch")) ||
        (s = ensure(c, c->mat4, (size_t)nt * 16, "material scratch")) ||
        (s = ensure(c, c->kept, ((words + 255) & ~size_t(255)) + counts, "kept path records")))
        return s;
    cudaStream_t st = (cudaStream_t)stream;
    int nl = launch_prf(Ip, np, params->gamma_p, params->gain_p, (float4 *)c->ep4.p, st);
    nl += launch_pack_tex(mat->albedo, mat->rough, nt, (float4 *)c->tex4.p, st);
    nl += launch_pack_mat(mat->metallic, mat->normal, nt, (float4 *)c->mat4.p, st);
    a.Ep = (const float4 *)c->ep4.p;
    a.tex = (const float4 *)c->tex4.p;
    a.Ic = Ic;
    a.Ec = Ec;
    char *kp = (char *)c->kept.p;
    nl += launch_render_keep_pbr(a, (const float4 *)c->mat4.p, kp, (uint8_t *)(kp + ((words + 255) & ~size_t(255))),
                                 st);
    if ((s = check_launch(c, nl, "render_keep_principled"))) return s;
    c->kept_key.valid = true;
    c->kept_key.scene = scene;
    c->kept_key.seed = seed;
    c->kept_key.Hc = view->Hc;
    c->kept_key.Wc = view->Wc;
    c->kept_key.spp = spp;
    c->kept_key.bounces = bounces;
    c->kept_key.log2L = a.log2L;
    c->kept_key.principled = true;
    return DPCS_OK;
}

dpcs_status dpcs_render_backward_kept_principled(dpcs_ctx *c, dpcs_scene scene, const dpcs_material *mat,
                                                 const float *Ip, const dpcs_view *view, const dpcs_params *params,
                                                 int32_t spp, int32_t bounces, uint64_t seed, const float *Ec,
                                                 const float *Ic, const float *dIc, float *dIp, float *dAlbedo,
                                                 float *dRough, float *dMetallic, float *dNormal, float *dParams,
                                                 void *stream) {
    Range range("dpcs_render_backward_kept_principled");
    if (!c) return DPCS_ERR_INVALID_ARG;
    if (!mat) return fail(c, DPCS_ERR_INVALID_ARG, "null material");
    RenderArgs a;
    Scene *sc = nullptr;
    dpcs_status s = prepare(c, scene, mat->albedo, mat->rough, mat->Ht, mat->Wt, Ip, view, params, spp, bounces, seed,
                            a, &sc);
    if (s) return s;
    if (!Ec || !Ic || !dIc) return fail(c, DPCS_ERR_INVALID_ARG, "null Ec, Ic or dIc");
    if (dMetallic && !mat->metallic) return fail(c, DPCS_ERR_INVALID_ARG, "dMetallic given without a metallic map");
    if (dNormal && !mat->normal) return fail(c, DPCS_ERR_INVALID_ARG, "dNormal given without a normal map");
    const auto &k = c->kept_key;
    if (!k.valid || !k.principled || k.scene != scene || k.seed != seed || k.Hc != view->Hc || k.Wc != view->Wc ||
        k.spp != spp || k.bounces != bounces || k.log2L != a.log2L)
        return fail(c, DPCS_ERR_INVALID_ARG, "render_backward_kept_principled: no kept principled render with these "
                                             "arguments");
    if ((s = set_device(c))) return s;
    const int64_t np = (int64_t)view->Hp * view->Wp, nt = (int64_t)mat->Ht * mat->Wt;
    const int64_t npix = (int64_t)view->Hc * view->Wc;
    const int L = 1 << a.log2L;
    const int64_t nthr = npix << a.log2L, spl = (spp + L - 1) / L;
    const size_t words = (size_t)kPRecWordsHost * spl * bounces * nthr * 4;
    const bool want_tex = dAlbedo || dRough, want_mat = dMetallic || dNormal;
    if ((s = ensure(c, c->gE, (size_t)npix * 12, "dEc scratch")) ||
        (s = ensure(c, c->dEp4, (size_t)np * 16, "dEp scratch")) ||
        (s = ensure(c, c->acc, 16 * sizeof(double), "parameter accumulators")) ||
        (want_tex && (s = ensure(c, c->dtex4, (size_t)nt * 16, "dtex scratch"))) ||
        (want_mat && (s = ensure(c, c->dmat4, (size_t)nt * 16, "dmat scratch"))))
        return s;
    cudaStream_t st = (cudaStream_t)stream;
    double *acc = (double *)c->acc.p;
    cudaMemsetAsync(acc, 0, 16 * sizeof(double), st);
    cudaMemsetAsync(c->dEp4.p, 0, (size_t)np * 16, st);
    if (want_tex) cudaMemsetAsync(c->dtex4.p, 0, (size_t)nt * 16, st);
    if (want_mat) cudaMemsetAsync(c->dmat4.p, 0, (size_t)nt * 16, st);
    int nl = launch_crf_backward(dIc, Ec, Ic, npix, params->gamma_c, params->gain_c, params->wb, (float *)c->gE.p, acc,
                                 st);
    a.gE = (const float *)c->gE.p;
    a.dEp = (float4 *)c->dEp4.p;
    a.dtex = want_tex ? (float4 *)c->dtex4.p : nullptr;
    const char *kp = (const char *)c->kept.p;
    nl += launch_sweep_kept_pbr(a, kp, (const uint8_t *)(kp + ((words + 255) & ~size_t(255))),
                                want_mat ? (float4 *)c->dmat4.p : nullptr, st);
    nl += launch_prf_backward(Ip, (const float4 *)c->dEp4.p, np, params->gamma_p, params->gain_p, dIp, acc, st);
    if (want_tex) nl += launch_tex_backward((const float4 *)c->dtex4.p, nt, dAlbedo, dRough, st);
    if (want_mat) nl += launch_mat_backward((const float4 *)c->dmat4.p, nt, dMetallic, dNormal, st);
    if (dParams) nl += launch_finalize_params(acc, dParams, st);
    return check_launch(c, nl, "render_backward_kept_principled");
}

dpcs_status dpcs_render_loss_backward_principled(dpcs_ctx *c, dpcs_scene scene, const dpcs_material *mat,
                                                 const float *Ip, const dpcs_view *view, const dpcs_params *params,
                                                 int32_t spp, int32_t bounces, uint64_t seed, const float *target,
                                                 int32_t loss_kind, float scale, float *Ic, float *Ec, float *loss,
                                                 float *dIp, float *dAlbedo, float *dRough, float *dMetallic,
                                                 float *dNormal, float *dParams, void *stream) {
    Range range("dpcs_render_loss_backward_principled");
    if (!c) return DPCS_ERR_INVALID_ARG;
    if (!mat) return fail(c, DPCS_ERR_INVALID_ARG, "null material");
    RenderArgs a;
    Scene *sc = nullptr;
    dpcs_status s = prepare(c, scene, mat->albedo, mat->rough, mat->Ht, mat->Wt, Ip, view, params, spp, bounces, seed,
                            a, &sc);
    if (s) return s;
    if (!target || !Ic || !loss) return fail(c, DPCS_ERR_INVALID_ARG, "null target, Ic or loss");
    if ((loss_kind != 0 && loss_kind != 1) || !(scale > 0.0f))
        return fail(c, DPCS_ERR_INVALID_ARG, "loss_kind must be 0 (L2) or 1 (L1) and scale > 0");
    if (dMetallic && !mat->metallic) return fail(c, DPCS_ERR_INVALID_ARG, "dMetallic given without a metallic map");
    if (dNormal && !mat->normal) return fail(c, DPCS_ERR_INVALID_ARG, "dNormal given without a normal map");
    if ((s = set_device(c))) return s;
    const int64_t np = (int64_t)view->Hp * view->Wp, nt = (int64_t)mat->Ht * mat->Wt;
    const int64_t npix = (int64_t)view->Hc * view->Wc;
    const int L = 1 << a.log2L;
    const int spl = (spp + L - 1) / L;  // samples per lane
    const bool fused = spl <= kFusedSamples && spl * bounces <= kFusedRecs;
    const bool want_tex = dAlbedo || dRough, want_mat = dMetallic || dNormal;
    if ((s = ensure(c, c->ep4, (size_t)np * 16, "Ep scratch")) ||
        (s = ensure(c, c->tex4, (size_t)nt * 16, "texture scratch")) ||
        (s = ensure(c, c->mat4, (size_t)nt * 16, "material scratch")) ||
        (s = ensure(c, c->dEp4, (size_t)np * 16, "dEp scratch")) ||
        (s = ensure(c, c->acc, 16 * sizeof(double), "parameter accumulators")) ||
        (want_tex && (s = ensure(c, c->dtex4, (size_t)nt * 16, "dtex scratch"))) ||
        (want_mat && (s = ensure(c, c->dmat4, (size_t)nt * 16, "dmat scratch"))) ||
        (!fused && ((s = ensure(c, c->gE, (size_t)npix * 12, "dEc scratch")) ||
                    (s = ensure(c, c->pix, (size_t)npix * 24, "per-pixel loss scratch")))))
        return s;
    cudaStream_t st = (cudaStream_t)stream;
    double *acc = (double *)c->acc.p;
    cudaMemsetAsync(acc, 0, 16 * sizeof(double), st);
    cudaMemsetAsync(c->dEp4.p, 0, (size_t)np * 16, st);
    if (want_tex) cudaMemsetAsync(c->dtex4.p, 0, (size_t)nt * 16, st);
    if (want_mat) cudaMemsetAsync(c->dmat4.p, 0, (size_t)nt * 16, st);
    int nl = launch_prf(Ip, np, params->gamma_p, params->gain_p, (float4 *)c->ep4.p, st);
    nl += launch_pack_tex(mat->albedo, mat->rough, nt, (float4 *)c->tex4.p, st);
    nl += launch_pack_mat(mat->metallic, mat->normal, nt, (float4 *)c->mat4.p, st);
    a.Ep = (const float4 *)c->ep4.p;
    a.tex = (const float4 *)c->tex4.p;
    a.Ic = Ic;
    a.dEp = (float4 *)c->dEp4.p;
    a.dtex = want_tex ? (float4 *)c->dtex4.p : nullptr;
    const float4 *m4 = (const float4 *)c->mat4.p;
    float4 *dm4 = want_mat ? (float4 *)c->dmat4.p : nullptr;
    const LossArgs l{target, scale, loss_kind, acc};
    if (fused) {
        a.Ec = Ec;
        nl += launch_render_grad_pbr(a, m4, dm4, l, st);
    } else {  // render, per-pixel loss, Eq. 5 adjoint, replay
        float *dIc = (float *)c->pix.p, *ec = Ec ? Ec : (float *)c->pix.p + 3 * npix;
        a.Ec = ec;
        nl += launch_render_pbr(a, m4, st);
        nl += launch_pixel_loss(Ic, npix * 3, l, dIc, st);
        nl += launch_crf_backward(dIc, ec, Ic, npix, params->gamma_c, params->gain_c, params->wb, (float *)c->gE.p,
                                  acc, st);
        a.gE = (const float *)c->gE.p;
        nl += launch_replay_pbr(a, m4, dm4, st);
    }
    nl += launch_loss_out(acc, loss, st);
    nl += launch_prf_backward(Ip, (const float4 *)c->dEp4.p, np, params->gamma_p, params->gain_p, dIp, acc, st);
    if (want_tex) nl += launch_tex_backward((const float4 *)c->dtex4.p, nt, dAlbedo, dRough, st);
    if (want_mat) nl += launch_mat_backward((const float4 *)c->dmat4.p, nt, dMetallic, dNormal, st);
    if (dParams) nl += launch_finalize_params(acc, dParams, st);
    return check_launch(c, nl, "render_loss_backward_principled");
}

dpcs_status dpcs_l2_loss(dpcs_ctx *c, const float *Ic, const float *target, int64_t n, float *dIc, float *loss,
                         void *stream) {
    if (!c) return DPCS_ERR_INVALID_ARG;
    if (n <= 0 || !Ic || !target || !dIc || !loss) return fail(c, DPCS_ERR_INVALID_ARG, "bad loss arguments");
    dpcs_status s = set_device(c);
    if (s) return s;
    if ((s = ensure(c, c->partial, (size_t)l2_partial_slots() * sizeof(double), "loss partials"))) return s;
    return check_launch(c, launch_l2_loss(Ic, target, n, dIc, loss, (double *)c->partial.p, (cudaStream_t)stream),
                        "l2 loss");
}

dpcs_status dpcs_l1_loss(dpcs_ctx *c, const float *Ic, const float *target, int64_t n, float scale, float *dIc,
                         float *loss, void *stream) {
    if (!c) return DPCS_ERR_INVALID_ARG;
    if (n <= 0 || !Ic || !target || !dIc || !loss || !(scale > 0.0f))
        return fail(c, DPCS_ERR_INVALID_ARG, "bad L1 loss arguments");
    dpcs_status s = set_device(c);
    if (s) return s;
    if ((s = ensure(c, c->partial, (size_t)l2_partial_slots() * sizeof(double), "loss partials"))) return s;
    return check_launch(c,
                        launch_l1_loss(Ic, target, n, scale, dIc, loss, (double *)c->partial.p, (cudaStream_t)stream),
                        "l1 loss");
}

dpcs_status dpcs_tv_loss(dpcs_ctx *c, const float *tex, int32_t H, int32_t W, int32_t C, float weight, float *grad,
                         float *loss, void *stream) {
    if (!c) return DPCS_ERR_INVALID_ARG;
    if (H <= 0 || W <= 0 || C <= 0 || C > 4 || !tex || !grad || !loss || !(weight >= 0.0f))
        return fail(c, DPCS_ERR_INVALID_ARG, "bad total-variation arguments");
    dpcs_status s = set_device(c);
    if (s) return s;
    if ((s = ensure(c, c->partial, (size_t)l2_partial_slots() * sizeof(double), "loss partials"))) return s;
    return check_launch(c, launch_tv_loss(tex, H, W, C, weight, grad, loss, (double *)c->partial.p,
                                          (cudaStream_t)stream), "total variation");
}

dpcs_status dpcs_adam(dpcs_ctx *c, float *p, const float *g, float *m, float *v, int64_t n, float lr, float beta1,
                      float beta2, float eps, int32_t step, float lo, float hi, void *stream) {
    if (!c) return DPCS_ERR_INVALID_ARG;
    if (n <= 0 || !p || !g || !m || !v || step < 1 || !(lo <= hi) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
        !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
        return fail(c, DPCS_ERR_INVALID_ARG, "bad Adam arguments");
    dpcs_status s = set_device(c);
    if (s) return s;
    return check_launch(c, launch_adam(p, g, m, v, n, lr, beta1, beta2, eps, step, lo, hi, (cudaStream_t)stream),
                        "adam");
}

// the pose adjoint of dpcs_pose_backward and dpcs_pose_backward_principled
// (pbr: the metallic and normal maps, each optional, are packed and used)
static dpcs_status pose_backward_impl(dpcs_ctx *c, dpcs_scene scene, const float *albedo, const float *rough,
                                      bool pbr, const float *metallic, const float *normal, int32_t Ht, int32_t Wt,
                                      const float *Ip, const dpcs_view *view, const dpcs_params *params, int32_t spp,
                                      int32_t bounces, uint64_t seed, const float *Ec, const float *Ic,
                                      const float *dIc, int32_t edge_spp, int32_t sil_spp, double *wrench,
                                      void *stream) {
    RenderArgs a;
    Scene *sc = nullptr;
    dpcs_status s = prepare(c, scene, albedo, rough, Ht, Wt, Ip, view, params, spp, bounces, seed, a, &sc);
    if (s) return s;
    if (!Ec || !Ic || !dIc || !wrench) return fail(c, DPCS_ERR_INVALID_ARG, "null Ec, Ic, dIc or wrench");
    if (edge_spp < 0 || sil_spp < 0 || edge_spp > (1 << 16) || sil_spp > (1 << 16))
        return fail(c, DPCS_ERR_INVALID_ARG, "edge_spp and sil_spp must be in [0, 65536]");
    if (view->Kc[6] != 0.0f || view->Kc[7] != 0.0f || !(view->Kc[8] > 0.0f))
        return fail(c, DPCS_ERR_INVALID_ARG, "pose gradient: Kc's last row must be (0, 0, k), k > 0");
    if ((s = set_device(c))) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t np = (int64_t)view->Hp * view->Wp, nt = (int64_t)Ht * Wt, npix = (int64_t)view->Hc * view->Wc;
    const EdgeTable *tab = nullptr;
    if (sil_spp > 0 && sc->T > 0 && (s = pose_edges(c, scene, *sc, st, &tab))) return s;
    // the Philox counters of pixel-edge and silhouette samples follow the
    // pixels': every one must fit in 32 bits
    if (2 * npix + (tab ? tab->n : 0) > (int64_t)0xffffffffLL)
        return fail(c, DPCS_ERR_INVALID_ARG, "pose gradient: too many pixels and edges for 32-bit counters");
    const int gmax = pose_grid(c->device);
    if (gmax <= 0) return fail(c, DPCS_ERR_CUDA, "pose gradient: no multiprocessor count");
    if ((s = ensure(c, c->ep4, (size_t)np * 16, "Ep scratch")) ||
        (s = ensure(c, c->tex4, (size_t)nt * 16, "texture scratch")) ||
        (s = ensure(c, c->gE, (size_t)npix * 12, "dEc scratch")) ||
        (s = ensure(c, c->acc, 16 * sizeof(double), "parameter accumulators")) ||
        (s = ensure(c, c->pose, (size_t)3 * gmax * 6 * sizeof(double), "pose partial sums")) ||
        (pbr && (s = ensure(c, c->mat4, (size_t)nt * 16, "material scratch"))))
        return s;
    int nl = launch_prf(Ip, np, params->gamma_p, params->gain_p, (float4 *)c->ep4.p, st);
    nl += launch_pack_tex(albedo, rough, nt, (float4 *)c->tex4.p, st);
    if (pbr) nl += launch_pack_mat(metallic, normal, nt, (float4 *)c->mat4.p, st);
    // dLoss/dEc through Eq. 5 (the response-parameter sums it also forms are not used)
    nl += launch_crf_backward(dIc, Ec, Ic, npix, params->gamma_c, params->gain_c, params->wb, (float *)c->gE.p,
                              (double *)c->acc.p, st);
    a.Ep = (const float4 *)c->ep4.p;
    a.tex = (const float4 *)c->tex4.p;
    a.gE = (const float *)c->gE.p;
    PoseArgs p;
    memcpy(p.Kc, view->Kc, sizeof p.Kc);
    p.edge_spp = edge_spp;
    p.sil_spp = tab ? sil_spp : 0;
    p.edges = tab ? tab->d : nullptr;
    p.nedges = tab ? tab->n : 0;
    p.partial = (double *)c->pose.p;
    p.mat = pbr ? (const float4 *)c->mat4.p : nullptr;
    TimedLaunch *tl = timing_begin(c, 2, st);
    const int np2 = launch_pose(a, p, c->device, wrench, st);
    timing_end(tl, st);
    if (np2 < 0) return check_launch(c, np2, "pose_backward");
    return check_launch(c, nl + np2, "pose_backward");
}

dpcs_status dpcs_pose_backward(dpcs_ctx *c, dpcs_scene scene, const float *albedo, const float *rough, int32_t Ht,
                               int32_t Wt, const float *Ip, const dpcs_view *view, const dpcs_params *params,
                               int32_t spp, int32_t bounces, uint64_t seed, const float *Ec, const float *Ic,
                               const float *dIc, int32_t edge_spp, int32_t sil_spp, double *wrench, void *stream) {
    Range range("dpcs_pose_backward");
    return pose_backward_impl(c, scene, albedo, rough, false, nullptr, nullptr, Ht, Wt, Ip, view, params, spp,
                              bounces, seed, Ec, Ic, dIc, edge_spp, sil_spp, wrench, stream);
}

dpcs_status dpcs_pose_backward_principled(dpcs_ctx *c, dpcs_scene scene, const dpcs_material *mat, const float *Ip,
                                          const dpcs_view *view, const dpcs_params *params, int32_t spp,
                                          int32_t bounces, uint64_t seed, const float *Ec, const float *Ic,
                                          const float *dIc, int32_t edge_spp, int32_t sil_spp, double *wrench,
                                          void *stream) {
    Range range("dpcs_pose_backward_principled");
    if (!c) return DPCS_ERR_INVALID_ARG;
    if (!mat) return fail(c, DPCS_ERR_INVALID_ARG, "null material");
    return pose_backward_impl(c, scene, mat->albedo, mat->rough, true, mat->metallic, mat->normal, mat->Ht, mat->Wt,
                              Ip, view, params, spp, bounces, seed, Ec, Ic, dIc, edge_spp, sil_spp, wrench, stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Rendering without allocation.
//
// dpcs_render keeps the PRF-mapped projector image and the packed textures in
// context scratch that grows with cudaMalloc on first use.  Some callers may
// not allocate device memory when they render: host applications that hand
// the GPU a fixed memory budget up front and own every allocation in it, and
// real-time loops that cannot absorb an allocation's latency or its failure
// part-way through a frame.  They use dpcs_render_noalloc instead.  Its
// scratch is the fixed array below, compiled into the library: every GPU that
// loads the library holds these 8 MiB until the process exits.  All calls
// share it, so calls that overlap on the GPU (different streams, or different
// host threads) race.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t kNoAllocTexels = int64_t(1) << 19;  // 524,288 float4 = 8 MiB
static __device__ __align__(256) float4 g_noalloc_scratch[kNoAllocTexels];

constexpr int kMaxDevices = 64;
// device address of the array per device; host threads may race on the first
// lookup, so the entries are atomics (both writers store the same address)
std::atomic<void *> g_noalloc_ptr[kMaxDevices];

// device address of the array for the current device, resolved once per
// device with that device current (the caller has made it current)
dpcs_status noalloc_scratch(dpcs_ctx *c, float4 **out) {
    if (c->device < 0 || c->device >= kMaxDevices) return fail(c, DPCS_ERR_INVALID_ARG, "device index too large");
    void *p = g_noalloc_ptr[c->device].load(std::memory_order_acquire);
    if (!p) {
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(c, e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_noalloc_ptr[c->device].store(p, std::memory_order_release);
    }
    *out = (float4 *)p;
    return DPCS_OK;
}

}  // namespace

extern "C" dpcs_status dpcs_render_noalloc(dpcs_ctx *c, dpcs_scene scene, const float *albedo, const float *rough,
                                           int32_t Ht, int32_t Wt, const float *Ip, const dpcs_view *view,
                                           const dpcs_params *params, int32_t spp, int32_t bounces, uint64_t seed,
                                           float *Ic, float *Ec, void *stream) {
    RenderArgs a;
    Scene *sc = nullptr;
    dpcs_status s = prepare(c, scene, albedo, rough, Ht, Wt, Ip, view, params, spp, bounces, seed, a, &sc);
    if (s) return s;
    if (!Ic) return fail(c, DPCS_ERR_INVALID_ARG, "null Ic");
    const int64_t np = (int64_t)view->Hp * view->Wp, nt = (int64_t)Ht * Wt;
    if (np + nt > kNoAllocTexels)
        return fail(c, DPCS_ERR_INVALID_ARG,
                    "dpcs_render_noalloc: Hp*Wp + Ht*Wt exceeds the fixed scratch of 524288 texels (8 MiB)");
    if ((s = set_device(c))) return s;
    float4 *scratch = nullptr;
    if ((s = noalloc_scratch(c, &scratch))) return s;
    float4 *ep4 = scratch, *tex4 = scratch + np;  // both fully overwritten below, nothing to clear
    cudaStream_t st = (cudaStream_t)stream;
    a.Ep = ep4;
    a.tex = tex4;
    a.Ic = Ic;
    a.Ec = Ec;
    int nl = launch_prf(Ip, np, params->gamma_p, params->gain_p, ep4, st);
    nl += launch_pack_tex(albedo, rough, nt, tex4, st);
    nl += launch_render(a, st);
    return check_launch(c, nl, "render_noalloc");
}

// ---------------------------------------------------------------------------
// Accessors used by the serving loop (serve.cu)
// ---------------------------------------------------------------------------
namespace dpcs {

dpcs_status ctx_render_args(dpcs_ctx *c, dpcs_scene scene, const float *albedo, const float *rough, int32_t Ht,
                            int32_t Wt, const float *Ip, const dpcs_view *view, const dpcs_params *params,
                            int32_t spp, int32_t bounces, uint64_t seed, RenderArgs &a) {
    Scene *sc = nullptr;
    return prepare(c, scene, albedo, rough, Ht, Wt, Ip, view, params, spp, bounces, seed, a, &sc);
}

int ctx_device(const dpcs_ctx *c) { return c->device; }

void ctx_add_launches(dpcs_ctx *c, int n) {
    if (n > 0) c->launches += (uint64_t)n;
}

dpcs_status ctx_fail(dpcs_ctx *c, dpcs_status code, const char *msg) { return fail(c, code, msg); }

}  // namespace dpcs
