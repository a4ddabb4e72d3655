// internal.h -- host-side structures shared by the translation units of libdpcs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "dpcs.h"

namespace dpcs {

// Device status bits, OR-ed into the context's status word by kernels.
enum : unsigned {
    kStatusTraversalLimit = 1u << 0,  // stack overflow or node-visit cap
    kStatusBoundsCheck = 1u << 1,     // an index failed a bounds check
};

// Resident scene: LBVH nodes (64 B: two child boxes and two child references),
// triangles in leaf order (48 B: v0 with the original index in .w, v1, v2)
// and their per-corner texture coordinates.
struct Scene {
    int32_t T = 0;
    int32_t root = 0;          // 0 = internal node 0; ~0 = single leaf; kEmptyRoot = no geometry
    float4 *nodes = nullptr;   // 4 x (T-1)
    float4 *tris = nullptr;    // 3 x T
    float2 *tuv = nullptr;     // 3 x T
    uint32_t *codes = nullptr; // sorted Morton codes, T
    int32_t *order = nullptr;  // original triangle of each sorted position, T
    int32_t V = 0;             // vertex count the mesh was uploaded with
    int32_t *vidx = nullptr;   // triangle vertex indices, 3 x T (kept for refits)
    float *uv = nullptr;       // per-vertex texture coordinates, 2 x V (kept for refits)
    float *base = nullptr;     // vertex positions of the last upload or update, 3 x V (rigid transforms start here)
    size_t bytes = 0;
};
constexpr int32_t kEmptyRoot = (int32_t)0x80000000;

// Kernel arguments of one render / replay launch (passed by value).
struct RenderArgs {
    const float4 *nodes;   // LBVH nodes
    const float4 *tris;
    const float2 *tuv;
    int32_t root;          // root reference
    int32_t T;
    const float4 *tex;   // Ht x Wt: albedo rgb, roughness
    int32_t Ht, Wt;
    const float4 *Ep;    // Hp x Wp: PRF-mapped projector image rgb, 0
    int32_t Hp, Wp;
    float Kci[9];        // inverse camera intrinsics
    float Kp[9], Rp[9], tp[3], cp[3];
    int32_t Hc, Wc;
    float gamma_c[3], gain_c, wb[3];
    float k_proj, ks, f0, rr_q, clip;
    int32_t rr_start, jitter;
    int32_t spp, bounces;
    uint32_t key0, key1;
    int32_t log2L;       // log2 of lanes per pixel
    float *Ic;
    float *Ec;
    // backward only
    const float *gE;     // dLoss/dEc per pixel (Hc x Wc x 3)
    float4 *dEp;         // dLoss/dEp accumulators (Hp x Wp)
    float4 *dtex;        // dLoss/d(albedo, rough) accumulators (Ht x Wt); null = not wanted
    unsigned *status;
    unsigned long long *counters;  // DPCS_COUNTERS build only (8 totals)
    int32_t visit_cap;             // traversal steps per ray before giving up (0 = 2T + 16)
    // backward only, FP64 accumulation mode: when dEp64 is set the adjoint
    // adds into these instead of dEp / dtex
    double *dEp64;                 // Hp x Wp x 3
    double *dtex64;                // Ht x Wt x 4 (albedo rgb, roughness); null = not wanted
};

// Per-pixel loss of the fused forward + adjoint kernel (k_render_grad).
struct LossArgs {
    const float *target;  // Hc x Wc x 3
    float scale;          // kind 0: loss 1/2 scale |Ic - t|^2, gradient scale (Ic - t); kind 1: scale |Ic - t|, scale sign
    int32_t kind;
    double *acc;          // parameter accumulators; acc[11] receives the loss
};
// Vertex records the fused kernel keeps per lane: up to kFusedSamples
// samples (ceil(spp / L)) and kFusedRecs vertices in all.
constexpr int kFusedSamples = 4;
constexpr int kFusedRecs = 12;

// One pass of the wavefront render (wavefront.cu): bounce b of the paths
// [path0, path0 + nchunk) of wave `wave`.  Path state arrays are indexed by
// the chunk-local path, the lane sums by the global path.
struct WfPass {
    RenderArgs r;
    int64_t path0;
    int32_t nchunk, wave, b;
    const int32_t *qin;   // paths of this bounce (null: every path of the chunk, bounce 1)
    const int32_t *nin;   // length of qin
    int32_t *qout;        // paths that continue to bounce b + 1
    int32_t *nout;        // length of qout (zeroed before the pass)
    float4 *hit;          // (leaf position as int bits, u, v, -) of the last traced ray
    float4 *ro, *rd;      // origin and direction of the next extension ray
    float4 *beta;         // throughput entering the next vertex
    float4 *sum;          // lane sums (xyz) per global path
    int32_t *fetch;       // rays taken from the pass's queue (persistent trace)
};

// One pixel range of one request in a batched render launch.
struct BatchSeg {
    int64_t vb_begin;   // first virtual block of the segment
    int64_t pix_begin;  // first pixel (y * Wc + x) of the range
    int64_t npix;       // pixels in the range
    int32_t slot;       // index of the request's RenderArgs
    int32_t pad;
};

// Launchers (render.cu, lbvh.cu, optim.cu).  Each returns the number of
// kernels it enqueued, or a negative dpcs_status.
int launch_lbvh_build(const float *d_verts, int32_t V, const int32_t *d_tris, int32_t T, const float *d_uv,
                      Scene &sc, void *scratch, size_t scratch_bytes, cudaStream_t st);
size_t lbvh_scratch_bytes(int32_t T);
// Refit after the vertices moved: new triangle records and node boxes over
// the existing tree (topology and leaf order kept).  d_verts holds sc.V
// vertices.  Returns the kernels enqueued or a negative dpcs_status.
int launch_lbvh_refit(const float *d_verts, Scene &sc, void *scratch, size_t scratch_bytes, cudaStream_t st);
// out[v] = R in[v] + t for V points (R row-major)
int launch_rigid_transform(const float *in, int32_t V, const float R[9], const float t[3], float *out, cudaStream_t st);
size_t lbvh_refit_scratch_bytes(int32_t T);
// Rebuild of the tree's topology by agglomerative clustering (PLOC) over the
// leaf order of the radix tree, for a lower surface-area cost: the nodes are
// replaced only if the new tree is at most max_depth deep (depth_out gets
// its depth).  Synchronises the stream once per clustering round.
size_t ploc_scratch_bytes(int32_t T);
int launch_ploc(Scene &sc, void *scratch, size_t scratch_bytes, int max_depth, cudaStream_t st, int32_t *depth_out);
constexpr int kMaxTreeDepth = 64;  // internal nodes on a root-to-leaf path: the traversal stack's depth

int launch_prf(const float *Ip, int64_t ntex, const float gamma_p[3], float gain_p, float4 *Ep, cudaStream_t st);
int launch_pack_tex(const float *albedo, const float *rough, int64_t ntex, float4 *tex, cudaStream_t st);
int launch_render(const RenderArgs &a, cudaStream_t st);
// the same render as a wavefront of trace and shade passes over path queues
// in chunks of `chunk` paths; scratch of wavefront_scratch_bytes(a, chunk)
size_t wavefront_scratch_bytes(const RenderArgs &a, int64_t chunk);
int launch_render_wavefront(const RenderArgs &a, int64_t chunk, void *scratch, cudaStream_t st);
int launch_render_batch(const RenderArgs *descs, const BatchSeg *segs, int nseg, int64_t total_vb,
                        unsigned long long *counter, int grid, cudaStream_t st);
int render_batch_grid(int device);
int64_t render_batch_vblocks(int64_t npix, int log2L);
int launch_trace(const Scene &sc, const float *o, const float *d, int64_t n, float *t, int32_t *tri,
                 unsigned *status, cudaStream_t st);
int launch_crf_backward(const float *dIc, const float *Ec, const float *Ic, int64_t npix, const float gamma_c[3],
                        float gain_c, const float wb[3], float *gE, double *acc, cudaStream_t st);
int launch_replay(const RenderArgs &a, cudaStream_t st);
int launch_render_grad(const RenderArgs &a, const LossArgs &l, cudaStream_t st);
int launch_pixel_loss(const float *Ic, int64_t n, const LossArgs &l, float *dIc, cudaStream_t st);
// principled material (principled.cu)
int launch_pack_mat(const float *metallic, const float *normal, int64_t ntex, float4 *mat, cudaStream_t st);
int launch_render_pbr(const RenderArgs &a, const float4 *mat, cudaStream_t st);
int launch_replay_pbr(const RenderArgs &a, const float4 *mat, float4 *dmat, cudaStream_t st);
int launch_mat_backward(const float4 *dmat, int64_t ntex, float *dMetallic, float *dNormal, cudaStream_t st);
int launch_render_grad_pbr(const RenderArgs &a, const float4 *mat, float4 *dmat, const LossArgs &l, cudaStream_t st);
// kept principled records: kPRecWordsHost 32-bit words per vertex
constexpr int kPRecWordsHost = 52;
int launch_render_keep_pbr(const RenderArgs &a, const float4 *mat, void *chunks, uint8_t *nvs, cudaStream_t st);
int launch_sweep_kept_pbr(const RenderArgs &a, const void *chunks, const uint8_t *nvs, float4 *dmat, cudaStream_t st);
int launch_render_keep(const RenderArgs &a, void *chunks, uint8_t *nvs, cudaStream_t st);
int launch_sweep_kept(const RenderArgs &a, const void *chunks, const uint8_t *nvs, cudaStream_t st);
constexpr int kRecWordsHost = 24;  // 32-bit words of one kept vertex record (VRec)
int launch_loss_out(const double *acc, float *loss, cudaStream_t st);
int launch_prf_backward(const float *Ip, const float4 *dEp, int64_t ntex, const float gamma_p[3], float gain_p,
                        float *dIp, double *acc, cudaStream_t st);
int launch_tex_backward(const float4 *dtex, int64_t ntex, float *dAlbedo, float *dRough, cudaStream_t st);
// the same from the FP64 accumulators (dEp64: 3 per texel, dtex64: 4 per texel)
int launch_prf_backward64(const float *Ip, const double *dEp64, int64_t ntex, const float gamma_p[3], float gain_p,
                          float *dIp, double *acc, cudaStream_t st);
int launch_tex_backward64(const double *dtex64, int64_t ntex, float *dAlbedo, float *dRough, cudaStream_t st);
int launch_finalize_params(const double *acc, float *dParams, cudaStream_t st);
int launch_zero(void *p, size_t bytes, cudaStream_t st);
int launch_l2_loss(const float *Ic, const float *target, int64_t n, float *dIc, float *loss, double *partial,
                   cudaStream_t st);
int launch_l1_loss(const float *Ic, const float *target, int64_t n, float scale, float *dIc, float *loss,
                   double *partial, cudaStream_t st);
int launch_tv_loss(const float *m, int H, int W, int C, float weight, float *grad, float *loss, double *partial,
                   cudaStream_t st);
int l2_partial_slots();
int launch_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2, float eps,
                int32_t step, float lo, float hi, cudaStream_t st);

// context accessors (api.cu) for the serving loop
dpcs_status ctx_render_args(dpcs_ctx *c, dpcs_scene scene, const float *albedo, const float *rough, int32_t Ht,
                            int32_t Wt, const float *Ip, const dpcs_view *view, const dpcs_params *params,
                            int32_t spp, int32_t bounces, uint64_t seed, RenderArgs &a);
int ctx_device(const dpcs_ctx *c);
void ctx_add_launches(dpcs_ctx *c, int n);
dpcs_status ctx_fail(dpcs_ctx *c, dpcs_status code, const char *msg);

}  // namespace dpcs
