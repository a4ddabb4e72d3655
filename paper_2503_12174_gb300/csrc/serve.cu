// serve.cu -- continuous-batching request loop for relighting (Eq. 7) and
// projector compensation (Eq. 13) on resident scenes.
//
// Host side only.  Each dpcs_serve_step is one iteration of the scheduler:
//   1. retire iterations whose completion event has fired, crediting the
//      pixels and steps they carried; finish requests whose results have
//      reached host memory and release their device memory;
//   2. admit waiting requests in arrival order while their device memory
//      fits the HBM budget and fewer than max_active are admitted;
//   3. plan about samples_per_iteration samples of work: every relighting
//      request first gets quantum_samples; then (fixed-share policy) one
//      compensation step per request (a full image) within
//      compensation_share of the iteration; the rest goes to relighting
//      requests in arrival order, and what relighting leaves unused runs
//      further consecutive compensation steps, still within that share; or
//      (deadline policy) everything goes to requests in order of deadline,
//      with no quanta; or (quanta-deadline policy) the quanta first, then
//      the rest in order of deadline;
//   4. enqueue on the server stream: the batch descriptors, one persistent
//      k_render_batch launch over the relighting pixels, each compensation
//      request's step: render, loss and path adjoint in one trace
//      (k_render_grad, or render + loss + replay when its records would not
//      fit), then Adam and PRF; the host copies of requests that finish in
//      this batch, and the iteration's completion event.
// Everything runs on one stream, so a compensation step always sees the
// previous step's Adam update; the host prepares the next iteration while
// the GPU runs the previous ones (up to max_inflight).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dpcs.h"
#include "internal.h"

using namespace dpcs;

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t al256(size_t n) { return (n + 255) & ~size_t(255); }

struct ServeScene {
    dpcs_scene handle;
    const float *albedo, *rough;
    int32_t Ht, Wt;
    float4 *tex4 = nullptr;  // packed albedo + roughness, server-owned
    dpcs_view view;
    dpcs_params params;
    int32_t bounces;
};

struct Req {
    uint64_t id = 0;
    dpcs_request r{};
    int state = DPCS_REQ_WAITING;
    double t_submit = 0, t_done = 0;
    size_t bytes = 0;
    char *mem = nullptr;
    // device buffers (sub-allocations of mem)
    float *Ip = nullptr, *Ic = nullptr, *Ec = nullptr, *target = nullptr, *dIc = nullptr, *gE = nullptr;
    float *M = nullptr, *V = nullptr, *G = nullptr, *loss = nullptr;
    float4 *Ep4 = nullptr, *dEp4 = nullptr;
    double *acc = nullptr, *partial = nullptr;
    RenderArgs args{};
    int64_t npix = 0, next_pix = 0, pix_done = 0;
    int steps_issued = 0, steps_done = 0;
    bool copy_queued = false;
    cudaEvent_t done_ev = nullptr;
    int64_t remaining_samples() const {
        return r.kind == DPCS_REQ_RELIGHT ? (npix - next_pix) * (int64_t)r.spp
                                          : (int64_t)(r.steps - steps_issued) * npix * r.spp;
    }
};

struct Batch {
    bool busy = false;
    int64_t seq = 0;  // iteration number, to find the oldest queued batch
    cudaEvent_t ev = nullptr;
    RenderArgs *descs_host = nullptr, *descs_dev = nullptr;
    BatchSeg *segs_host = nullptr, *segs_dev = nullptr;
    unsigned long long *counter = nullptr;
    std::vector<std::pair<Req *, int64_t>> pixels;  // relighting pixels carried
    std::vector<Req *> steps;                        // compensation steps carried
};

}  // namespace

struct dpcs_server {
    dpcs_ctx *ctx = nullptr;
    int device = 0;
    dpcs_serve_config cfg{};
    cudaStream_t stream = nullptr;
    cudaMemPool_t pool = nullptr;  // request memory; keeps what requests free for the next admissions
    std::vector<ServeScene> scenes;
    std::deque<Req *> waiting;
    std::vector<Req *> active;
    std::unordered_map<uint64_t, Req *> all;
    std::vector<Batch> batches;
    uint64_t next_id = 1;
    size_t used = 0, high_water = 0;
    int64_t submitted = 0, completed = 0, failed = 0, iterations = 0, launches = 0;
    int grid = 1;
};

namespace {

dpcs_status sfail(dpcs_server *s, dpcs_status code, const char *msg) { return ctx_fail(s->ctx, code, msg); }

dpcs_status scuda(dpcs_server *s, cudaError_t e, const char *what) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return ctx_fail(s->ctx, DPCS_ERR_CUDA, buf);
}

// device bytes a request holds while admitted
size_t request_bytes(const dpcs_server *s, const dpcs_request &r) {
    const ServeScene &sc = s->scenes[r.scene];
    const size_t np = (size_t)sc.view.Hp * sc.view.Wp, npix = (size_t)r.Hc * r.Wc;
    size_t b = al256(np * 12) + al256(np * 16) + al256(npix * 12);  // Ip, Ep4, Ic
    if (r.kind == DPCS_REQ_COMPENSATE)  // compensation moves Ip only: no texture gradient is kept
        b += 4 * al256(npix * 12) + 3 * al256(np * 12) + al256(np * 16) + al256(16 * 8) + al256(4) +
             al256((size_t)l2_partial_slots() * 8);  // Ec target dIc gE; M V G; dEp4; acc; loss
    return b;
}

dpcs_view request_view(const ServeScene &sc, const dpcs_request &r) {
    dpcs_view v = sc.view;
    const float sx = (float)r.Wc / (float)sc.view.Wc, sy = (float)r.Hc / (float)sc.view.Hc;
    v.Kc[0] *= sx; v.Kc[1] *= sx; v.Kc[2] *= sx;  // keep the field of view at the new resolution
    v.Kc[3] *= sy; v.Kc[4] *= sy; v.Kc[5] *= sy;
    v.Hc = r.Hc;
    v.Wc = r.Wc;
    return v;
}

dpcs_status admit(dpcs_server *s, Req *q) {
    const ServeScene &sc = s->scenes[q->r.scene];
    const dpcs_request &r = q->r;
    const size_t np = (size_t)sc.view.Hp * sc.view.Wp, npix = (size_t)r.Hc * r.Wc;
    cudaError_t e = cudaMallocFromPoolAsync((void **)&q->mem, q->bytes, s->pool, s->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return sfail(s, DPCS_ERR_OOM, "serve: stream-ordered allocation failed");
    }
    s->used += q->bytes;  // released with the memory in release()
    s->high_water = std::max(s->high_water, s->used);
    char *p = q->mem;
    auto take = [&](size_t n) {
        char *r0 = p;
        p += al256(n);
        return r0;
    };
    q->Ip = (float *)take(np * 12);
    q->Ep4 = (float4 *)take(np * 16);
    q->Ic = (float *)take(npix * 12);
    if (r.kind == DPCS_REQ_COMPENSATE) {
        q->Ec = (float *)take(npix * 12);
        q->target = (float *)take(npix * 12);
        q->dIc = (float *)take(npix * 12);
        q->gE = (float *)take(npix * 12);
        q->M = (float *)take(np * 12);
        q->V = (float *)take(np * 12);
        q->G = (float *)take(np * 12);
        q->dEp4 = (float4 *)take(np * 16);
        q->acc = (double *)take(16 * 8);
        q->loss = (float *)take(4);
        q->partial = (double *)take((size_t)l2_partial_slots() * 8);
    }
    e = cudaMemcpyAsync(q->Ip, r.Ip, np * 12, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess && q->target) e = cudaMemcpyAsync(q->target, r.target, npix * 12, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess && q->M) e = cudaMemsetAsync(q->M, 0, np * 12, s->stream);
    if (e == cudaSuccess && q->V) e = cudaMemsetAsync(q->V, 0, np * 12, s->stream);
    if (e != cudaSuccess) return scuda(s, e, "serve: request upload");
    const dpcs_view v = request_view(sc, r);
    dpcs_status st = ctx_render_args(s->ctx, sc.handle, sc.albedo, sc.rough, sc.Ht, sc.Wt, q->Ip, &v, &sc.params,
                                     r.spp, sc.bounces, r.seed, q->args);
    if (st) return st;
    q->args.Ep = q->Ep4;
    q->args.tex = sc.tex4;
    q->args.Ic = q->Ic;
    q->args.Ec = q->Ec;
    q->args.counters = nullptr;
    q->npix = (int64_t)npix;
    s->launches += launch_prf(q->Ip, (int64_t)np, sc.params.gamma_p, sc.params.gain_p, q->Ep4, s->stream);
    q->state = DPCS_REQ_ACTIVE;
    return DPCS_OK;
}

// one compensation step after its render: L2 loss, path replay, PRF
// adjoint, Adam on Ip with the clamp to [0, 1], then Ep for the next render
int enqueue_comp_backward(dpcs_server *s, Req *q) {
    const ServeScene &sc = s->scenes[q->r.scene];
    const int64_t np = (int64_t)sc.view.Hp * sc.view.Wp;
    cudaStream_t st = s->stream;
    int n = launch_l2_loss(q->Ic, q->target, q->npix * 3, q->dIc, q->loss, q->partial, st);
    cudaMemsetAsync(q->acc, 0, 16 * 8, st);
    cudaMemsetAsync(q->dEp4, 0, (size_t)np * 16, st);
    cudaMemsetAsync(q->G, 0, (size_t)np * 12, st);
    n += launch_crf_backward(q->dIc, q->Ec, q->Ic, q->npix, sc.params.gamma_c, sc.params.gain_c, sc.params.wb, q->gE,
                             q->acc, st);
    RenderArgs a = q->args;
    a.gE = q->gE;
    a.dEp = q->dEp4;
    a.dtex = nullptr;  // only Ip is optimised
    n += launch_replay(a, st);
    n += launch_prf_backward(q->Ip, q->dEp4, np, sc.params.gamma_p, sc.params.gain_p, q->G, q->acc, st);
    n += launch_adam(q->Ip, q->G, q->M, q->V, np * 3, q->r.lr, 0.9f, 0.999f, 1e-8f, q->steps_issued, 0.0f, 1.0f, st);
    n += launch_prf(q->Ip, np, sc.params.gamma_p, sc.params.gain_p, q->Ep4, st);
    return n;
}

// one compensation step in a single trace of its paths (k_render_grad):
// render, L2 loss, adjoint, then PRF adjoint, Adam and Ep for the next step
bool comp_step_fuses(const Req *q) {
    const int L = 1 << q->args.log2L;
    const int spl = (q->args.spp + L - 1) / L;
    return spl <= kFusedSamples && spl * q->args.bounces <= kFusedRecs;
}

int enqueue_comp_step_fused(dpcs_server *s, Req *q) {
    const ServeScene &sc = s->scenes[q->r.scene];
    const int64_t np = (int64_t)sc.view.Hp * sc.view.Wp;
    cudaStream_t st = s->stream;
    cudaMemsetAsync(q->acc, 0, 16 * 8, st);
    cudaMemsetAsync(q->dEp4, 0, (size_t)np * 16, st);
    cudaMemsetAsync(q->G, 0, (size_t)np * 12, st);
    RenderArgs a = q->args;
    a.dEp = q->dEp4;
    a.dtex = nullptr;  // only Ip is optimised
    const LossArgs l{q->target, 1.0f, 0, q->acc};
    int n = launch_render_grad(a, l, st);
    n += launch_loss_out(q->acc, q->loss, st);
    n += launch_prf_backward(q->Ip, q->dEp4, np, sc.params.gamma_p, sc.params.gain_p, q->G, q->acc, st);
    n += launch_adam(q->Ip, q->G, q->M, q->V, np * 3, q->r.lr, 0.9f, 0.999f, 1e-8f, q->steps_issued, 0.0f, 1.0f, st);
    n += launch_prf(q->Ip, np, sc.params.gamma_p, sc.params.gain_p, q->Ep4, st);
    return n;
}

void release(dpcs_server *s, Req *q) {
    if (q->mem) {
        cudaFreeAsync(q->mem, s->stream);
        q->mem = nullptr;
        s->used -= q->bytes;
    }
    if (q->done_ev) {
        cudaEventDestroy(q->done_ev);
        q->done_ev = nullptr;
    }
}

int retire(dpcs_server *s) {
    for (Batch &b : s->batches) {
        if (!b.busy || cudaEventQuery(b.ev) != cudaSuccess) continue;
        for (auto &pr : b.pixels) pr.first->pix_done += pr.second;
        for (Req *q : b.steps) q->steps_done++;
        b.pixels.clear();
        b.steps.clear();
        b.busy = false;
    }
    cudaGetLastError();  // cudaErrorNotReady from the queries above is not an error
    int done = 0;
    for (size_t i = 0; i < s->active.size();) {
        Req *q = s->active[i];
        if (q->copy_queued && cudaEventQuery(q->done_ev) == cudaSuccess) {
            q->t_done = now_s();
            q->state = DPCS_REQ_DONE;
            release(s, q);
            s->active.erase(s->active.begin() + i);
            ++s->completed;
            ++done;
            continue;
        }
        ++i;
    }
    cudaGetLastError();
    return done;
}

Batch *free_batch(dpcs_server *s) {
    for (Batch &b : s->batches)
        if (!b.busy) return &b;
    return nullptr;
}

// queue the host copy of a request's results after the work that completes it
dpcs_status queue_result_copy(dpcs_server *s, Req *q) {
    const ServeScene &sc = s->scenes[q->r.scene];
    cudaError_t e = cudaEventCreateWithFlags(&q->done_ev, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(q->r.Ic_out, q->Ic, (size_t)q->npix * 12, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess && q->r.kind == DPCS_REQ_COMPENSATE && q->r.Ip_out)
        e = cudaMemcpyAsync(q->r.Ip_out, q->Ip, (size_t)sc.view.Hp * sc.view.Wp * 12, cudaMemcpyDeviceToHost,
                            s->stream);
    if (e == cudaSuccess) e = cudaEventRecord(q->done_ev, s->stream);
    if (e != cudaSuccess) return scuda(s, e, "serve: result copy");
    q->copy_queued = true;
    return DPCS_OK;
}

void plan_fixed_share(dpcs_server *s, const std::vector<Req *> &relight, const std::vector<Req *> &comp,
                      std::vector<int64_t> &give, int64_t &budget, int64_t total_budget, Batch &b);
void plan_by_deadline(dpcs_server *s, const std::vector<Req *> &relight, const std::vector<Req *> &comp,
                      std::vector<int64_t> &give, int64_t &budget, Batch &b);
dpcs_status enqueue_iteration(dpcs_server *s, Batch &b, int nseg, int64_t vb);

dpcs_status launch_iteration(dpcs_server *s, Batch &b) {
    std::vector<Req *> comp, relight;
    for (Req *q : s->active) {
        if (q->copy_queued) continue;
        if (q->r.kind == DPCS_REQ_COMPENSATE) {
            if (q->steps_issued < q->r.steps) comp.push_back(q);
        } else if (q->next_pix < q->npix) {
            relight.push_back(q);
        }
    }
    if (comp.empty() && relight.empty()) return DPCS_OK;
    int nseg = 0;
    int64_t vb = 0;
    const int64_t total_budget = s->cfg.samples_per_iteration;
    int64_t budget = total_budget;
    auto add_seg = [&](Req *q, int64_t pix0, int64_t npx) {
        b.descs_host[nseg] = q->args;
        BatchSeg &g = b.segs_host[nseg];
        g.vb_begin = vb;
        g.pix_begin = pix0;
        g.npix = npx;
        g.slot = nseg;
        g.pad = 0;
        vb += render_batch_vblocks(npx, q->args.log2L);
        ++nseg;
    };
    // `active` is in arrival order.  1) (fixed share, quanta-deadline) every
    // relighting request gets a small quantum, so short requests finish
    // within an iteration or two; under the deadline policy the deadlines
    // order them
    std::vector<int64_t> give(relight.size(), 0);
    for (size_t i = 0; s->cfg.policy != DPCS_SERVE_DEADLINE && i < relight.size() && budget > 0; ++i) {
        Req *q = relight[i];
        give[i] = std::min(q->npix - q->next_pix, std::max<int64_t>(1, s->cfg.quantum_samples / q->r.spp));
        budget -= give[i] * q->r.spp;
    }
    if (s->cfg.policy == DPCS_SERVE_DEADLINE || s->cfg.policy == DPCS_SERVE_QUANTA_DEADLINE) {
        plan_by_deadline(s, relight, comp, give, budget, b);
    } else {
        plan_fixed_share(s, relight, comp, give, budget, total_budget, b);
    }
    for (size_t i = 0; i < relight.size(); ++i) {
        if (give[i] <= 0) continue;
        Req *q = relight[i];
        add_seg(q, q->next_pix, give[i]);
        b.pixels.push_back({q, give[i]});
        q->next_pix += give[i];
    }
    return enqueue_iteration(s, b, nseg, vb);
}

// The fixed-share plan: 2) one compensation step per request in arrival
// order (a full image) within compensation_share of the iteration; 3) the rest
// to relighting requests in arrival order; 4) what relighting leaves unused
// runs further consecutive steps of the same compensation requests.
void plan_fixed_share(dpcs_server *s, const std::vector<Req *> &relight, const std::vector<Req *> &comp,
                      std::vector<int64_t> &give, int64_t &budget, int64_t total_budget, Batch &b) {
    const int64_t comp_cap = (int64_t)(s->cfg.compensation_share * (double)total_budget);
    int64_t comp_used = 0;
    for (Req *q : comp) {
        const int64_t need = q->npix * q->r.spp;
        if (!b.steps.empty() && comp_used + need > comp_cap) break;
        comp_used += need;
        b.steps.push_back(q);
    }
    budget -= comp_used;
    // 3) the rest goes to relighting requests in arrival order, so long
    //    requests advance first-come first-served and none is starved;
    for (size_t i = 0; i < relight.size() && budget > 0; ++i) {
        Req *q = relight[i];
        const int64_t extra = std::min(q->npix - q->next_pix - give[i], budget / q->r.spp);
        if (extra > 0) {
            give[i] += extra;
            budget -= extra * q->r.spp;
        }
    }
    // 4) budget that relighting left unused runs further consecutive steps of
    //    the same compensation requests, in rounds, still within that share of the
    //    iteration (rounds keep each request's steps in order on the stream).
    const size_t n_first = b.steps.size();
    std::vector<int> planned(n_first, 1);
    for (bool more = true; more;) {
        more = false;
        for (size_t i = 0; i < n_first; ++i) {
            Req *q = b.steps[i];
            const int64_t need = q->npix * q->r.spp;
            if (q->steps_issued + planned[i] >= q->r.steps || comp_used + need > comp_cap || need > budget) continue;
            comp_used += need;
            budget -= need;
            b.steps.push_back(q);
            ++planned[i];
            more = true;
        }
    }
}

// The deadline plan: every request (after the relighting quanta) has a
// deadline, its arrival plus its slack times the time its remaining work
// would take alone at est_samples_per_s; the iteration's remaining budget
// goes to requests in deadline order -- relighting pixels, or consecutive
// compensation steps (a step counts its samples x kStepCost).  Small
// requests therefore pass large ones, and a large request's deadline comes
// up as it waits.
void plan_by_deadline(dpcs_server *s, const std::vector<Req *> &relight, const std::vector<Req *> &comp,
                      std::vector<int64_t> &give, int64_t &budget, Batch &b) {
    constexpr double kStepCost = 1.4;  // a fused render + adjoint step, in forward samples
    struct Claim {
        double deadline;
        int relight;  // index into relight, or -1
        Req *q;
    };
    std::vector<Claim> claims;
    const double R = s->cfg.est_samples_per_s;
    for (size_t i = 0; i < relight.size(); ++i) {
        Req *q = relight[i];
        const double work = (double)q->npix * q->r.spp;
        claims.push_back({q->t_submit + s->cfg.relight_slack * work / R, (int)i, q});
    }
    for (Req *q : comp) {
        const double work = kStepCost * (double)q->r.steps * q->npix * q->r.spp;
        claims.push_back({q->t_submit + s->cfg.compensation_slack * work / R, -1, q});
    }
    std::stable_sort(claims.begin(), claims.end(), [](const Claim &x, const Claim &y) { return x.deadline < y.deadline; });
    for (const Claim &c : claims) {
        if (budget <= 0) break;
        Req *q = c.q;
        if (c.relight >= 0) {
            const int64_t extra = std::min(q->npix - q->next_pix - give[c.relight], budget / q->r.spp);
            if (extra > 0) {
                give[c.relight] += extra;
                budget -= extra * q->r.spp;
            }
        } else {
            const int64_t need = (int64_t)(kStepCost * (double)q->npix * q->r.spp);
            for (int k = q->steps_issued; k < q->r.steps && (need <= budget || b.steps.empty()); ++k) {
                b.steps.push_back(q);
                budget -= need;
            }
        }
    }
}

dpcs_status enqueue_iteration(dpcs_server *s, Batch &b, int nseg, int64_t vb) {
    cudaStream_t st = s->stream;
    cudaError_t e = cudaSuccess;
    int n = 0;
    if (nseg > 0) {
        e = cudaMemcpyAsync(b.descs_dev, b.descs_host, sizeof(RenderArgs) * nseg, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b.segs_dev, b.segs_host, sizeof(BatchSeg) * nseg, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(b.counter, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return scuda(s, e, "serve: batch upload");
        n += launch_render_batch(b.descs_dev, b.segs_dev, nseg, vb, b.counter, s->grid, st);
    }
    for (Req *q : b.steps) {
        // a fresh Philox key per step (step k uses seed + k); a whole image is
        // one k_render launch, whose arguments sit in constant space
        q->args.key0 = (uint32_t)((q->r.seed + (uint64_t)q->steps_issued) & 0xffffffffu);
        q->args.key1 = (uint32_t)((q->r.seed + (uint64_t)q->steps_issued) >> 32);
        if (comp_step_fuses(q)) {
            q->steps_issued++;
            n += enqueue_comp_step_fused(s, q);
        } else {
            n += launch_render(q->args, st);
            q->steps_issued++;
            n += enqueue_comp_backward(s, q);
        }
        if (q->steps_issued == q->r.steps) {
            dpcs_status rs = queue_result_copy(s, q);
            if (rs) return rs;
        }
    }
    for (auto &pr : b.pixels) {
        Req *q = pr.first;
        if (q->next_pix == q->npix) {
            dpcs_status rs = queue_result_copy(s, q);
            if (rs) return rs;
        }
    }
    s->launches += n;
    ctx_add_launches(s->ctx, n);
    e = cudaEventRecord(b.ev, st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return scuda(s, e, "serve: iteration launch");
    b.busy = true;
    b.seq = ++s->iterations;
    return DPCS_OK;
}

void free_batch_bufs(Batch &b) {
    if (b.ev) cudaEventDestroy(b.ev);
    if (b.descs_host) cudaFreeHost(b.descs_host);
    if (b.segs_host) cudaFreeHost(b.segs_host);
    if (b.descs_dev) cudaFree(b.descs_dev);
    if (b.segs_dev) cudaFree(b.segs_dev);
    if (b.counter) cudaFree(b.counter);
}

}  // namespace

extern "C" {

dpcs_status dpcs_serve_create(dpcs_ctx *ctx, const dpcs_serve_config *cfg, dpcs_server **out) {
    if (!ctx || !cfg || !out) return DPCS_ERR_INVALID_ARG;
    *out = nullptr;
    if (cfg->max_active < 1 || cfg->max_active > 1024 || cfg->max_inflight < 1 || cfg->max_inflight > 4 ||
        cfg->samples_per_iteration < 1 || cfg->quantum_samples < 1 ||
        (cfg->policy != DPCS_SERVE_DEADLINE && cfg->policy != DPCS_SERVE_FIXED_SHARE &&
         cfg->policy != DPCS_SERVE_QUANTA_DEADLINE) ||
        (cfg->policy != DPCS_SERVE_FIXED_SHARE &&
         !(cfg->relight_slack > 0.0 && cfg->compensation_slack > 0.0 && cfg->est_samples_per_s > 0.0)) ||
        (cfg->policy == DPCS_SERVE_FIXED_SHARE && !(cfg->compensation_share > 0.0 && cfg->compensation_share <= 1.0)))
        return ctx_fail(ctx, DPCS_ERR_INVALID_ARG, "serve: bad config");
    dpcs_server *s = new dpcs_server();
    s->ctx = ctx;
    s->cfg = *cfg;
    s->device = ctx_device(ctx);
    cudaError_t e = cudaSetDevice(s->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        // a pool of its own whose freed memory is never trimmed back to the
        // driver, so admissions after the first reuse mapped memory
        cudaMemPoolProps pp{};
        pp.allocType = cudaMemAllocationTypePinned;
        pp.location.type = cudaMemLocationTypeDevice;
        pp.location.id = s->device;
        e = cudaMemPoolCreate(&s->pool, &pp);
        uint64_t keep = ~0ull;
        if (e == cudaSuccess) e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    s->batches.resize(cfg->max_inflight);
    for (Batch &b : s->batches) {
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&b.descs_host, sizeof(RenderArgs) * cfg->max_active);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&b.segs_host, sizeof(BatchSeg) * cfg->max_active);
        if (e == cudaSuccess) e = cudaMalloc((void **)&b.descs_dev, sizeof(RenderArgs) * cfg->max_active);
        if (e == cudaSuccess) e = cudaMalloc((void **)&b.segs_dev, sizeof(BatchSeg) * cfg->max_active);
        if (e == cudaSuccess) e = cudaMalloc((void **)&b.counter, sizeof(unsigned long long));
    }
    if (e != cudaSuccess) {
        dpcs_status st = ctx_fail(ctx, DPCS_ERR_CUDA, "serve: create failed");
        for (Batch &b : s->batches) free_batch_bufs(b);
        if (s->stream) cudaStreamDestroy(s->stream);
        if (s->pool) cudaMemPoolDestroy(s->pool);
        delete s;
        return st;
    }
    s->grid = render_batch_grid(s->device);
    *out = s;
    return DPCS_OK;
}

dpcs_status dpcs_serve_destroy(dpcs_server *s) {
    if (!s) return DPCS_ERR_INVALID_ARG;
    cudaSetDevice(s->device);
    cudaStreamSynchronize(s->stream);
    for (auto &kv : s->all) {
        release(s, kv.second);
        delete kv.second;
    }
    for (ServeScene &sc : s->scenes)
        if (sc.tex4) cudaFree(sc.tex4);
    for (Batch &b : s->batches) free_batch_bufs(b);
    cudaStreamSynchronize(s->stream);
    cudaStreamDestroy(s->stream);
    cudaMemPoolDestroy(s->pool);
    delete s;
    return DPCS_OK;
}

dpcs_status dpcs_serve_add_scene(dpcs_server *s, dpcs_scene scene, const float *albedo, const float *rough,
                                 int32_t Ht, int32_t Wt, const dpcs_view *view, const dpcs_params *params,
                                 int32_t bounces, int32_t *slot) {
    if (!s || !view || !params || !slot) return DPCS_ERR_INVALID_ARG;
    RenderArgs probe;
    // validates the scene handle, textures, view and parameters once
    dpcs_status st = ctx_render_args(s->ctx, scene, albedo, rough, Ht, Wt, albedo, view, params, 1, bounces, 0, probe);
    if (st) return st;
    ServeScene sc;
    sc.handle = scene;
    sc.albedo = albedo;
    sc.rough = rough;
    sc.Ht = Ht;
    sc.Wt = Wt;
    sc.view = *view;
    sc.params = *params;
    sc.bounces = bounces;
    cudaSetDevice(s->device);
    cudaError_t e = cudaMalloc((void **)&sc.tex4, (size_t)Ht * Wt * 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return sfail(s, DPCS_ERR_OOM, "serve: scene texture allocation failed");
    }
    s->launches += launch_pack_tex(albedo, rough, (int64_t)Ht * Wt, sc.tex4, s->stream);
    e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return scuda(s, e, "serve: add_scene");
    *slot = (int32_t)s->scenes.size();
    s->scenes.push_back(sc);
    return DPCS_OK;
}

dpcs_status dpcs_serve_submit(dpcs_server *s, const dpcs_request *req, uint64_t *id) {
    if (!s || !req || !id) return DPCS_ERR_INVALID_ARG;
    const dpcs_request &r = *req;
    if (r.scene < 0 || r.scene >= (int32_t)s->scenes.size()) return sfail(s, DPCS_ERR_NOT_FOUND, "serve: unknown scene");
    if (r.kind != DPCS_REQ_RELIGHT && r.kind != DPCS_REQ_COMPENSATE) return sfail(s, DPCS_ERR_INVALID_ARG, "serve: bad kind");
    if (r.Hc <= 0 || r.Wc <= 0 || (int64_t)r.Hc * r.Wc > (int64_t)1 << 26 || r.spp < 1 || r.spp > 4096 || !r.Ip ||
        !r.Ic_out)
        return sfail(s, DPCS_ERR_INVALID_ARG, "serve: bad request size or buffer");
    if (r.kind == DPCS_REQ_COMPENSATE && (!r.target || r.steps < 1 || !(r.lr > 0.0f)))
        return sfail(s, DPCS_ERR_INVALID_ARG, "serve: compensation needs target, steps >= 1, lr > 0");
    Req *q = new Req();
    q->id = s->next_id++;
    q->r = r;
    q->bytes = request_bytes(s, r);
    if (s->cfg.hbm_budget_bytes && q->bytes > s->cfg.hbm_budget_bytes) {
        delete q;
        return sfail(s, DPCS_ERR_OOM, "serve: request larger than the HBM budget");
    }
    q->t_submit = now_s();
    s->all[q->id] = q;
    s->waiting.push_back(q);
    ++s->submitted;
    *id = q->id;
    return DPCS_OK;
}

dpcs_status dpcs_serve_step(dpcs_server *s, int32_t *completed) {
    if (!s) return DPCS_ERR_INVALID_ARG;
    cudaSetDevice(s->device);
    int done = retire(s);
    // admission by HBM budget and slot count, in arrival order
    while (!s->waiting.empty() && (int)s->active.size() < s->cfg.max_active) {
        Req *q = s->waiting.front();
        if (s->cfg.hbm_budget_bytes && s->used + q->bytes > s->cfg.hbm_budget_bytes) break;
        s->waiting.pop_front();
        dpcs_status st = admit(s, q);
        if (st) {
            q->state = DPCS_REQ_FAILED;
            release(s, q);
            ++s->failed;
            return st;
        }
        s->active.push_back(q);
    }
    Batch *b = free_batch(s);
    if (!b) {
        // every slot is queued: wait (bounded by the queued GPU work) for the oldest
        Batch *oldest = &s->batches[0];
        for (Batch &x : s->batches)
            if (x.seq < oldest->seq) oldest = &x;
        cudaEventSynchronize(oldest->ev);
        done += retire(s);
        b = free_batch(s);
    }
    dpcs_status st = b ? launch_iteration(s, *b) : DPCS_OK;
    if (completed) *completed = done;
    return st;
}

dpcs_status dpcs_serve_query(dpcs_server *s, uint64_t id, int32_t *state, double *latency_ms) {
    if (!s || !state) return DPCS_ERR_INVALID_ARG;
    auto it = s->all.find(id);
    if (it == s->all.end()) return sfail(s, DPCS_ERR_NOT_FOUND, "serve: unknown request");
    *state = it->second->state;
    if (latency_ms) *latency_ms = it->second->state == DPCS_REQ_DONE ? (it->second->t_done - it->second->t_submit) * 1e3 : -1.0;
    return DPCS_OK;
}

dpcs_status dpcs_serve_drain(dpcs_server *s, double timeout_s) {
    if (!s) return DPCS_ERR_INVALID_ARG;
    const double t0 = now_s();
    while (!s->waiting.empty() || !s->active.empty()) {
        if (now_s() - t0 > timeout_s) return sfail(s, DPCS_ERR_TIMEOUT, "serve: drain timed out");
        int32_t done = 0;
        dpcs_status st = dpcs_serve_step(s, &done);
        if (st) return st;
        if (!done) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    return DPCS_OK;
}

dpcs_status dpcs_serve_stats_get(dpcs_server *s, dpcs_serve_stats *o) {
    if (!s || !o) return DPCS_ERR_INVALID_ARG;
    o->submitted = s->submitted;
    o->completed = s->completed;
    o->failed = s->failed;
    o->waiting = (int64_t)s->waiting.size();
    o->active = (int64_t)s->active.size();
    o->iterations = s->iterations;
    o->launches = s->launches;
    o->memory_used = s->used;
    o->memory_high_water = s->high_water;
    return DPCS_OK;
}

}  // extern "C"
