/*
 * dpcs.h -- C ABI of libdpcs, a GB300 (sm_103a) path tracer for
 * differentiable projector-camera simulation (DPCS, arxiv 2503.12174).
 *
 * The library renders the camera image Ic of a triangle scene lit only by a
 * pinhole projector showing the image Ip (forward rendering, Sec. 3.2 Eq. 7),
 * and back-propagates dLoss/dIc to Ip, to the BRDF textures and to the
 * projector/camera response parameters (the gradient used by inverse
 * rendering, Eq. 8, projector compensation, Eq. 13, and scene fitting,
 * Eq. 9).  Every step runs in the library's own CUDA kernels.
 *
 * Conventions for every entry point:
 *  - Images and textures are float32, contiguous, row-major HWC with y down.
 *    Matrices are float32 row-major (OpenCV style).
 *  - "dev" pointers are CUDA device pointers on the context's device, owned
 *    by the caller; "host" pointers are ordinary host memory, owned by the
 *    caller.  The library owns scene data and its own scratch memory.
 *  - Calls that take a stream enqueue work on it (cudaStream_t passed as
 *    void*, NULL = legacy default stream) and return before the GPU is done.
 *    Argument errors are reported synchronously.  Device-side check failures
 *    (traversal limits, bounds checks) are recorded in a device status word
 *    and reported by dpcs_sync.  No kernel traps.
 *  - One context per host thread; a context is not thread safe.
 *  - Scratch memory is allocated on first use for a given problem size and
 *    counted against the context's HBM budget; call an entry point once with
 *    the largest sizes before capturing it in a CUDA graph.
 */
#ifndef DPCS_H
#define DPCS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t dpcs_status;
#define DPCS_OK 0
#define DPCS_ERR_INVALID_ARG (-1)     /* bad pointer, size or parameter */
#define DPCS_ERR_OOM (-2)             /* allocation failed or HBM budget exceeded */
#define DPCS_ERR_CUDA (-3)            /* a CUDA runtime call failed */
#define DPCS_ERR_DEVICE_CHECK (-4)    /* a kernel's bounds check failed */
#define DPCS_ERR_TRAVERSAL_LIMIT (-5) /* BVH traversal hit its stack or visit cap */
#define DPCS_ERR_TIMEOUT (-6)         /* a bounded wait ran out */
#define DPCS_ERR_BUSY (-7)            /* no free slot / budget right now */
#define DPCS_ERR_NOT_FOUND (-8)       /* unknown scene or request handle */

#define DPCS_MAX_BOUNCES 8            /* most path vertices per camera sample */

typedef struct dpcs_ctx dpcs_ctx;
typedef uint64_t dpcs_scene;

/*
 * Response, BRDF and sampling parameters.
 *  gamma_p, gain_p : projector response Ep = gain_p * Ip^gamma_p (Eq. 1)
 *  gamma_c, gain_c, wb : camera response Ic = (gain_c * wb * Ec)^gamma_c (Eq. 5)
 *  k_proj  : projector intensity scale k; stands for 1/phi of Eq. 2 and is the
 *            k of the radiance clip of Eq. 12
 *  ks, f0  : weight of the GGX specular lobe and its Schlick F0; the diffuse
 *            lobe is albedo/pi (the paper's principled BRDF reduced to
 *            Lambert + GGX, Sec. 3.2)
 *  rr_start, rr_q : Russian roulette on continuations from vertex rr_start on
 *            (0 = off) with survival probability rr_q
 *  clip    : per-vertex radiance clamp of Eq. 12 (0 = off)
 *  jitter  : 1 = uniform jitter inside each camera pixel (box filter of Eq. 4),
 *            0 = rays through pixel centres
 */
typedef struct dpcs_params {
    float gamma_p[3];
    float gain_p;
    float gamma_c[3];
    float gain_c;
    float wb[3];
    float k_proj;
    float ks;
    float f0;
    int32_t rr_start;
    float rr_q;
    float clip;
    int32_t jitter;
} dpcs_params;

/*
 * Camera and projector (Eq. 6).  The world origin is the camera's optical
 * centre (Sec. 3.1); x_c = Kc x_s.  The projector maps a world point to its
 * pixel by x_p = Kp (Rp x_s + tp).  Hc x Wc is the camera image, Hp x Wp the
 * projector image.
 */
typedef struct dpcs_view {
    float Kc[9];
    int32_t Hc, Wc;
    float Kp[9];
    float Rp[9];
    float tp[3];
    int32_t Hp, Wp;
} dpcs_view;

/* Create a context on CUDA device `device`; scratch and scenes may use at
 * most `hbm_budget_bytes` (0 = no limit).  *out receives the context. */
dpcs_status dpcs_create(int device, size_t hbm_budget_bytes, dpcs_ctx **out);

/* Free every scene, scratch buffer and the context itself (synchronises). */
dpcs_status dpcs_destroy(dpcs_ctx *ctx);

/* Text of the last error recorded by this context ("" if none). */
const char *dpcs_last_error(const dpcs_ctx *ctx);

/* Wait for `stream`, then read and clear the device status word.  Returns
 * DPCS_ERR_TRAVERSAL_LIMIT or DPCS_ERR_DEVICE_CHECK if a kernel recorded one. */
dpcs_status dpcs_sync(dpcs_ctx *ctx, void *stream);

/* Bytes of device memory the context holds now (scenes + scratch). */
size_t dpcs_memory_used(const dpcs_ctx *ctx);

/* Number of kernels the context has launched since it was created. */
uint64_t dpcs_launch_count(const dpcs_ctx *ctx);

/*
 * Kernel timing with CUDA events recorded on the launching stream around the
 * path-tracing kernels: kernel 0 = forward render (k_render), 1 = path replay
 * (k_replay), 2 = the pose-gradient kernels (dpcs_pose_backward).
 * dpcs_timing_enable(ctx, 1) clears and starts recording, (ctx, 0) stops it.
 * dpcs_timing_read waits for the recorded events and returns the summed
 * duration in milliseconds and the number of launches.
 * Measurement support, not part of the paper's method.
 */
dpcs_status dpcs_timing_enable(dpcs_ctx *ctx, int32_t on);
dpcs_status dpcs_timing_read(dpcs_ctx *ctx, int32_t kernel, double *total_ms, int64_t *launches);

/*
 * Work counters of a library built with DPCS_COUNTERS: out[0..9] = BVH node
 * visits, triangle tests, closest-hit rays, shadow rays, path vertices,
 * vertices lit by the projector, BRDF continuations, camera paths, warp
 * iterations of the traversal loop and warp iterations of the path loop
 * (one ray per lane and iteration), summed over every render / replay launch
 * since the last reset (reset != 0 clears them after reading).  The last two
 * give SIMT efficiencies: (node visits + triangle tests) / (32 x traversal
 * warp iterations) and rays / (32 x path warp iterations).  `out` holds 10
 * values.  Synchronous.  Returns DPCS_ERR_INVALID_ARG in a library built
 * without counters.  Measurement support for the roofline.
 */
dpcs_status dpcs_counters_read(dpcs_ctx *ctx, uint64_t *out, int32_t reset);

/*
 * Failure-path testing: cap every ray's BVH traversal at `cap` steps in the
 * render and replay calls that follow (0 restores the default, 2T + 16, which
 * a correct tree never reaches).  A ray that reaches the cap ends as a miss
 * and sets the status bit that dpcs_sync reports as
 * DPCS_ERR_TRAVERSAL_LIMIT; nothing traps and the context stays usable.
 * Not part of the paper's method.
 */
dpcs_status dpcs_debug_set_visit_cap(dpcs_ctx *ctx, int32_t cap);

/*
 * How dpcs_render traces its paths (the same estimator, Eqs. 3, 10; the same
 * images bit for bit):
 *  DPCS_PATH_MEGAKERNEL (default): one kernel; each lane runs its paths from
 *    the camera to their last vertex.
 *  DPCS_PATH_WAVEFRONT: per bounce, a closest-hit pass over the extension
 *    rays of every live path and a shading pass (next-event estimation with
 *    its shadow ray, BRDF continuation) that appends the paths that go on to
 *    the next bounce's queue.  Paths run in chunks of `chunk` paths (0 keeps
 *    the current value, 2^20 at creation; else a multiple of 32 in
 *    [4096, 2^28]), whose state (64 B per path) is context scratch, plus 16 B
 *    of running sum per (pixel, lane).
 * DPCS_ERR_INVALID_ARG for another path or chunk.
 */
#define DPCS_PATH_MEGAKERNEL 0
#define DPCS_PATH_WAVEFRONT 1
dpcs_status dpcs_set_render_path(dpcs_ctx *ctx, int32_t path, int64_t chunk);

/*
 * Accumulation precision of the adjoint's gradient scatters (the path-replay
 * adjoint of Eq. 8's inverse rendering; Sec. 3.2, Eq. 13):
 *  DPCS_ACCUM_F32 (default): packed float4 atomics into FP32 accumulators.
 *    Fast; each projector texel or texture texel sums its contributions in
 *    whatever order the atomics arrive, so the last bits vary run to run.
 *  DPCS_ACCUM_F64: one FP64 atomic per component (FP64 accumulators,
 *    24 B per projector texel and 32 B per texture texel of context
 *    scratch), and the Eq. 1 adjoint and its reductions in FP64 before the
 *    result is rounded to FP32.  The order of the adds then changes the sums
 *    only at FP64 rounding, about 1e-16 of their magnitude.
 * Applies to dpcs_render_backward, dpcs_render_backward_kept and
 * dpcs_render_loss_backward on this context; the principled-material calls
 * always accumulate in FP32.  DPCS_ERR_INVALID_ARG for another mode.
 */
#define DPCS_ACCUM_F32 0
#define DPCS_ACCUM_F64 1
dpcs_status dpcs_set_grad_accum(dpcs_ctx *ctx, int32_t mode);

/*
 * Upload a triangle mesh and build its LBVH on the device (Morton codes of
 * triangle centroids, radix sort, Karras radix tree, bottom-up AABB refit).
 *  verts : host, V x 3 float32 positions (world = camera frame)
 *  tris  : host, T x 3 int32 vertex indices, each in [0, V)
 *  uv    : host, V x 2 float32 texture coordinates in [0,1]^2
 * T may be 0 (every ray misses).  The host arrays may be reused once the call
 * returns (it synchronises on `stream`).  *out receives the scene handle.
 * The paper renders Poisson-reconstructed triangle meshes (Sec. 4, Sec. 4.4).
 */
dpcs_status dpcs_scene_upload(dpcs_ctx *ctx, const float *verts, int32_t V, const int32_t *tris, int32_t T,
                              const float *uv, void *stream, dpcs_scene *out);

/*
 * Move the vertices of an uploaded scene (novel scene simulation and
 * deforming surfaces, Sec. 4.4: a morphing mesh re-lit frame by frame).
 * verts (host, V x 3) are the new positions of the same V vertices; the
 * triangles and texture coordinates stay as uploaded.  The library rewrites
 * its triangle records and refits every box of the existing tree bottom-up
 * (topology and leaf order kept, so the tree stays valid; it loses quality
 * as the motion grows, and a re-upload rebuilds it).  Enqueued on `stream`
 * after the host copy; renders that use the scene must be ordered after it
 * on the same stream.  DPCS_ERR_INVALID_ARG if V differs from the upload or
 * a coordinate is not finite; DPCS_ERR_NOT_FOUND for an unknown scene.
 */
dpcs_status dpcs_scene_update(dpcs_ctx *ctx, dpcs_scene scene, const float *verts, int32_t V, void *stream);

/*
 * Tree topology of the scenes uploaded from now on (closest hits, and so
 * every image and gradient, do not depend on it):
 *  DPCS_BVH_PLOC (default): the radix tree over the Morton order is rebuilt
 *    by agglomerative clustering (PLOC, Meister & Bittner 2018: mutual
 *    nearest neighbours by union surface area within 16 clusters on either
 *    side in Morton order), a tree of lower surface-area cost that rays
 *    traverse with fewer node visits.  The upload then synchronises the
 *    stream once per clustering round.  A tree deeper than the traversal
 *    stack (64) is not taken, nor one whose build could not have its
 *    scratch memory or failed a check: the radix tree stays.
 *  DPCS_BVH_LBVH: the Karras radix tree itself.
 * Codes, leaf order and the triangle records are the same for both; refits
 * (dpcs_scene_update, dpcs_scene_transform) keep whichever topology the
 * upload built.  Measurement and quality setting, not part of the paper.
 */
#define DPCS_BVH_LBVH 0
#define DPCS_BVH_PLOC 1
dpcs_status dpcs_set_bvh_builder(dpcs_ctx *ctx, int32_t builder);

/*
 * Rigid transform of an uploaded scene, for the camera pose (Rc, tc) of
 * Sec. 3.2's scene parameters: renders take the camera at the origin
 * (Eq. 6), and a camera at pose (Rc, tc) sees each world point x at
 * Rc x + tc, so a pose refinement moves the mesh by (R, t) = (Rc, tc) and
 * the projector extrinsics by Rp' = Rp R^T, tp' = tp - Rp' t (the caller
 * passes those in the view).  Every vertex of the scene's last upload or
 * update goes to R v + t (R host, row-major 3 x 3; t host, 3 floats) and the
 * tree is refitted as by dpcs_scene_update.  The stored positions are not
 * changed, so transforms do not compound: each call maps the same positions.
 * DPCS_ERR_INVALID_ARG for a null or non-finite R or t; DPCS_ERR_NOT_FOUND
 * for an unknown scene.
 */
dpcs_status dpcs_scene_transform(dpcs_ctx *ctx, dpcs_scene scene, const float R[9], const float t[3], void *stream);

/* Release a scene's device memory. */
dpcs_status dpcs_scene_free(dpcs_ctx *ctx, dpcs_scene scene);

/*
 * Copy a scene's LBVH to host memory (for inspection and tests):
 *  codes    : T uint32 Morton codes in sorted order
 *  order    : T int32 original triangle index of each sorted position
 *  child    : (T-1) x 2 int32 child references of the internal nodes;
 *             >= 0 internal node, < 0 leaf ~sorted_position
 *  child_box: (T-1) x 2 x 6 float32 child boxes (lo.xyz, hi.xyz)
 * Any output pointer may be NULL.  Synchronous.
 */
dpcs_status dpcs_scene_export(dpcs_ctx *ctx, dpcs_scene scene, uint32_t *codes, int32_t *order, int32_t *child,
                              float *child_box);

/*
 * Closest hit of n rays through the scene's BVH.
 *  orig, dir : dev, n x 3 float32 (dir need not be normalised; t is in units of dir)
 *  t_out     : dev, n float32 hit distance (+inf on a miss)
 *  tri_out   : dev, n int32 original triangle index (-1 on a miss)
 * Ties in t go to the lowest triangle index.
 */
dpcs_status dpcs_trace(dpcs_ctx *ctx, dpcs_scene scene, const float *orig, const float *dir, int64_t n,
                       float *t_out, int32_t *tri_out, void *stream);

/*
 * Forward rendering Ic = R(Ip, theta) (Eq. 7).  For every camera pixel, spp
 * paths of at most `bounces` vertices are traced; each vertex does next-event
 * estimation towards the projector (Eqs. 1, 2, 3, 6) and continues by
 * sampling the BRDF (Eq. 10).  Ec is the mean path radiance of the pixel
 * (Eq. 4) and Ic its camera response (Eq. 5).
 *  albedo : dev, Ht x Wt x 3;  rough : dev, Ht x Wt (GGX alpha = rough^2)
 *  Ip     : dev, Hp x Wp x 3 projector input image
 *  Ic     : dev out, Hc x Wc x 3
 *  Ec     : dev out, Hc x Wc x 3, or NULL (keep it for render_backward)
 *  seed   : key of the Philox4x32-10 stream; counters are
 *           (pixel index y*Wc+x, sample, vertex, 0), so a pixel's result does
 *           not depend on how the image is partitioned.
 * 1 <= spp, 0 <= bounces <= DPCS_MAX_BOUNCES.  Deterministic: the same
 * inputs give bitwise the same Ic.
 */
dpcs_status dpcs_render(dpcs_ctx *ctx, dpcs_scene scene, const float *albedo, const float *rough, int32_t Ht,
                        int32_t Wt, const float *Ip, const dpcs_view *view, const dpcs_params *params, int32_t spp,
                        int32_t bounces, uint64_t seed, float *Ic, float *Ec, void *stream);

/*
 * dpcs_render without any device allocation.  It is for callers that cannot
 * call cudaMalloc when they render: host applications that give the GPU a
 * fixed memory budget up front and own every allocation in it, and real-time
 * loops that cannot absorb an allocation's latency, or its failure, part-way
 * through a frame.  Arguments, results and error codes are those of
 * dpcs_render: the same kernels run, and Ic and Ec are bit-identical to
 * dpcs_render's.  The PRF-mapped projector image and the packed textures
 * live in one fixed array compiled into the library instead of context
 * scratch:
 *  - limit: Hp*Wp + Ht*Wt <= 524288 texels (8 MiB); larger sizes return
 *    DPCS_ERR_INVALID_ARG without launching anything;
 *  - every GPU that loads the library holds the 8 MiB until the process exits;
 *  - the first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture begins;
 *  - all calls share the array and every call overwrites the part it uses:
 *    calls that overlap on the GPU (other streams, other host threads) race
 *    and must be serialised by the caller.
 * The paper has no counterpart.
 */
dpcs_status dpcs_render_noalloc(dpcs_ctx *ctx, dpcs_scene scene, const float *albedo, const float *rough,
                                int32_t Ht, int32_t Wt, const float *Ip, const dpcs_view *view,
                                const dpcs_params *params, int32_t spp, int32_t bounces, uint64_t seed, float *Ic,
                                float *Ec, void *stream);

/*
 * Adjoint of dpcs_render (path replay): every path is re-traced from its
 * Philox counters, and dLoss/dIc is carried back with the sampled directions
 * held fixed.  Inputs are those of the forward call plus
 *  Ec, Ic : dev, the forward call's outputs;  dIc : dev, Hc x Wc x 3
 * Outputs are ACCUMULATED (+=):
 *  dIp     : dev, Hp x Wp x 3   (may be NULL)
 *  dAlbedo : dev, Ht x Wt x 3   (may be NULL)
 *  dRough  : dev, Ht x Wt       (may be NULL)
 *  dParams : dev, 11 float32 [gamma_p(3), gain_p, gamma_c(3), gain_c, wb(3)]
 *            (may be NULL)
 * These are the gradients of the scene parameters theta of Eq. 9 that do not
 * move geometry, and of the projector input of Eq. 13.  With dAlbedo and
 * dRough both NULL the replay skips the texture scatters (compensation
 * needs only dIp); the other outputs are unchanged.
 */
dpcs_status dpcs_render_backward(dpcs_ctx *ctx, dpcs_scene scene, const float *albedo, const float *rough,
                                 int32_t Ht, int32_t Wt, const float *Ip, const dpcs_view *view,
                                 const dpcs_params *params, int32_t spp, int32_t bounces, uint64_t seed,
                                 const float *Ec, const float *Ic, const float *dIc, float *dIp, float *dAlbedo,
                                 float *dRough, float *dParams, void *stream);

/*
 * Gradient with respect to the camera pose (Rc, tc), which Sec. 3.2 counts
 * among the scene parameters theta of Eq. 9.  Renders keep the camera at the
 * origin (Eq. 6), so a pose parameter moves the whole scene (mesh and
 * projector) rigidly in the camera frame: a point y moves with velocity
 * a x y + b, the twist (a, b) of that parameter.  The call returns, for a
 * loss with dLoss/dIc = dIc, the six numbers W = dLoss/d(a, b); the
 * derivative for a parameter with twist (a, b) is a . W[0..2] + b . W[3..5].
 * It differentiates the box-filtered pixel means of Eq. 4 with their
 * visibility changes, as three Monte Carlo terms:
 *   interior     every camera sample of the render (same Philox counters):
 *                its first vertex's BRDF as the direction to the camera
 *                turns, and the path contribution times the change of the
 *                pixel footprint's area on the surface;
 *   pixel edges  per pixel, edge_spp points on each of its four edges,
 *                the paths through them weighted by the pixel's dLoss/dEc
 *                and the image velocity out of the pixel (the four paths of
 *                a sample share their random numbers, so that opposite
 *                edges give a low-variance difference across the pixel);
 *   silhouettes  sil_spp points on each mesh edge that is a silhouette from
 *                the camera, in view and inside the image, weighted by the
 *                radiance of the surface behind it and the relative image
 *                velocity of the two surfaces across the edge.
 * Inputs are those of dpcs_render_backward (the scene at the pose where the
 * gradient is wanted, i.e. after dpcs_scene_transform, with the matching
 * view) plus
 *  edge_spp : samples per pixel edge, 0..65536 (0 drops the term)
 *  sil_spp  : samples per mesh edge, 0..65536 (0 drops the term)
 * Output, ACCUMULATED (+=):
 *  wrench   : dev, 18 float64: interior, pixel-edge and silhouette terms,
 *             each (W_a[3], W_b[3]); their sum is W.
 * The plain material (dpcs_pose_backward_principled below takes the
 * metallic and normal maps).  Kc's last row must
 * be (0, 0, k) with k > 0.  The first call with sil_spp > 0 on a scene builds
 * its edge table on the host (one stream synchronisation); later calls,
 * updates and transforms reuse it.  Results repeat bit for bit for the same
 * inputs on the same device.
 */
dpcs_status dpcs_pose_backward(dpcs_ctx *ctx, dpcs_scene scene, const float *albedo, const float *rough, int32_t Ht,
                               int32_t Wt, const float *Ip, const dpcs_view *view, const dpcs_params *params,
                               int32_t spp, int32_t bounces, uint64_t seed, const float *Ec, const float *Ic,
                               const float *dIc, int32_t edge_spp, int32_t sil_spp, double *wrench, void *stream);

/* ------------------------------------------------------------------------ */
/* Denoiser of Eq. 11: Ic' = D(Ic), a differentiable cross-bilateral filter  */
/* ------------------------------------------------------------------------ */
/*
 * The paper applies a differentiable cross-bilateral filter D to the
 * rendered camera image before the loss (Sec. 3.3, Eq. 11), without naming
 * its guide or widths.  Here the guide is the renderer's own noise-free
 * first hit through each pixel centre, and
 *   D(I)(p) = sum_q w(p,q) I(q) / W(p),   W(p) = sum_q w(p,q),
 *   w(p,q)  = exp(-|p-q|^2/(2 s^2) - |a_p-a_q|^2/(2 sa^2) - |n_p-n_q|^2/(2 sn^2)
 *                 - (t_p-t_q)^2/(2 sd^2))
 * over the (2r+1)^2 window around p that lies inside the image (a albedo,
 * n normal, t hit distance; a width <= 0 drops its term).  The weights depend
 * on the guide only: D is linear in I and the gradient does not flow into
 * the guide.
 */
/*
 * Principled material (Sec. 3.2: the BRDF maps m -- here base colour,
 * roughness and metallic -- and the normal map Vn; Sec. 4.3 gives metallic
 * in [0, 1] and the normal map in [0, 1]^3).  All maps are device arrays
 * of one size Ht x Wt, HWC float32, sampled bilinearly with the albedo's
 * texture coordinates.
 *
 *   f_j = (1 - m) rho_j / pi + ks D G F_j / (4 cos_i cos_o),
 *   F_j = F0_j + (1 - F0_j) (1 - wo.h)^5,  F0_j = (1 - m) f0 + m rho_j
 *
 * The normal map decodes to v = 2 Vn - 1 in the triangle's tangent frame
 * (T = dp/du orthogonal to the geometric normal N turned towards the ray,
 * B = N x T); the shading normal v / |v| replaces N in the BRDF, its
 * sampling and both cosines, while N keeps the ray offsets and light or
 * continuations below the geometric surface are dropped.  metallic == NULL
 * means 0 everywhere; normal == NULL means (0.5, 0.5, 1), no perturbation.
 * The caller owns every map.
 */
typedef struct dpcs_material {
    const float *albedo;    /* Ht x Wt x 3 */
    const float *rough;     /* Ht x Wt */
    const float *metallic;  /* Ht x Wt or NULL */
    const float *normal;    /* Ht x Wt x 3 or NULL */
    int32_t Ht, Wt;
} dpcs_material;

/*
 * dpcs_render_principled: dpcs_render with the principled material (same
 * view, parameters, sampling, determinism and errors; the one-trace loss
 * step and the kept records have principled variants below, the batched
 * serving render has none).
 *
 * dpcs_render_backward_principled: its path-replay adjoint, as
 * dpcs_render_backward, adding (+=) also dLoss/dmetallic (Ht x Wt) and
 * dLoss/dnormal (Ht x Wt x 3); each output may be NULL, and asking for the
 * gradient of a map the material does not have is DPCS_ERR_INVALID_ARG.
 * Sampled directions and pdfs are held fixed (detached sampling), so the
 * normal-map gradient, like roughness, is exact per seed only for one
 * bounce and unbiased beyond.
 */
dpcs_status dpcs_render_principled(dpcs_ctx *ctx, dpcs_scene scene, const dpcs_material *mat, const float *Ip,
                                   const dpcs_view *view, const dpcs_params *params, int32_t spp, int32_t bounces,
                                   uint64_t seed, float *Ic, float *Ec, void *stream);
dpcs_status dpcs_render_backward_principled(dpcs_ctx *ctx, dpcs_scene scene, const dpcs_material *mat,
                                            const float *Ip, const dpcs_view *view, const dpcs_params *params,
                                            int32_t spp, int32_t bounces, uint64_t seed, const float *Ec,
                                            const float *Ic, const float *dIc, float *dIp, float *dAlbedo,
                                            float *dRough, float *dMetallic, float *dNormal, float *dParams,
                                            void *stream);

/*
 * dpcs_render_keep_principled / dpcs_render_backward_kept_principled:
 * dpcs_render_keep and dpcs_render_backward_kept (same arguments, checks,
 * memory and errors) with the principled material; the records are 208 B
 * per recorded vertex.  A kept plain render does not serve the principled
 * adjoint, nor the other way round (DPCS_ERR_INVALID_ARG).
 */
dpcs_status dpcs_render_keep_principled(dpcs_ctx *ctx, dpcs_scene scene, const dpcs_material *mat, const float *Ip,
                                        const dpcs_view *view, const dpcs_params *params, int32_t spp,
                                        int32_t bounces, uint64_t seed, float *Ic, float *Ec, void *stream);
dpcs_status dpcs_render_backward_kept_principled(dpcs_ctx *ctx, dpcs_scene scene, const dpcs_material *mat,
                                                 const float *Ip, const dpcs_view *view, const dpcs_params *params,
                                                 int32_t spp, int32_t bounces, uint64_t seed, const float *Ec,
                                                 const float *Ic, const float *dIc, float *dIp, float *dAlbedo,
                                                 float *dRough, float *dMetallic, float *dNormal, float *dParams,
                                                 void *stream);

/*
 * dpcs_render_loss_backward_principled: dpcs_render_loss_backward (render,
 * per-pixel L2 / L1 loss and adjoint; same arguments, loss kinds, scale,
 * outputs and record limits, one trace of each path when
 * ceil(spp / L) <= 4 and ceil(spp / L) * bounces <= 12, otherwise render,
 * loss, Eq. 5 adjoint and replay) with the principled material, adding (+=)
 * also dLoss/dmetallic and dLoss/dnormal when given (each needs its map:
 * DPCS_ERR_INVALID_ARG otherwise).
 */
dpcs_status dpcs_render_loss_backward_principled(dpcs_ctx *ctx, dpcs_scene scene, const dpcs_material *mat,
                                                 const float *Ip, const dpcs_view *view, const dpcs_params *params,
                                                 int32_t spp, int32_t bounces, uint64_t seed, const float *target,
                                                 int32_t loss_kind, float scale, float *Ic, float *Ec, float *loss,
                                                 float *dIp, float *dAlbedo, float *dRough, float *dMetallic,
                                                 float *dNormal, float *dParams, void *stream);

/*
 * dpcs_pose_backward with the principled material (Sec. 3.2: metallic m
 * and normal map Vn among theta, with the pose): the first vertex's BRDF
 * and its turn with the camera are the principled lobe's at the shading
 * normal, which moves with the surface.  mat as for dpcs_render_principled
 * (metallic and normal may be NULL); the other arguments and the output as
 * for dpcs_pose_backward.
 */
dpcs_status dpcs_pose_backward_principled(dpcs_ctx *ctx, dpcs_scene scene, const dpcs_material *mat, const float *Ip,
                                          const dpcs_view *view, const dpcs_params *params, int32_t spp,
                                          int32_t bounces, uint64_t seed, const float *Ec, const float *Ic,
                                          const float *dIc, int32_t edge_spp, int32_t sil_spp, double *wrench,
                                          void *stream);

typedef struct dpcs_denoise_params {
    int32_t radius;      /* window half-width r, 0..8 (0 = identity) */
    float sigma_s;       /* spatial width in pixels, > 0 */
    float sigma_albedo;  /* albedo width (<= 0: term off) */
    float sigma_normal;  /* normal width (<= 0: term off) */
    float sigma_depth;   /* hit-distance width, scene units (<= 0: term off) */
} dpcs_denoise_params;

/* Guide features of scene `scene` seen through each camera pixel centre of
 * `view` (jitter and the projector fields of the view are not used):
 * guide (dev, 16-byte aligned, Hc x Wc x 8 float32) = albedo rgb (bilinear,
 * as the renderer samples it), geometric normal turned towards the camera,
 * hit distance along the unit ray, 1; all 8 are 0 where the ray misses.
 * albedo/rough: dev textures as in dpcs_render.  Allocates a temporary
 * 16 * Ht * Wt byte texture, stream-ordered, for the call. */
dpcs_status dpcs_gbuffer(dpcs_ctx *ctx, dpcs_scene scene, const float *albedo, const float *rough, int32_t Ht,
                         int32_t Wt, const dpcs_view *view, float *guide, void *stream);

/* out = D(Ic) (dev, Hc x Wc x 3, must not alias Ic); wsum (dev, Hc x Wc, may
 * be NULL) receives W, which dpcs_denoise_backward needs.  guide from
 * dpcs_gbuffer.  DPCS_ERR_INVALID_ARG for radius outside 0..8, sigma_s <= 0,
 * a misaligned guide or null pointers. */
dpcs_status dpcs_denoise(dpcs_ctx *ctx, const float *Ic, const float *guide, int32_t Hc, int32_t Wc,
                         const dpcs_denoise_params *params, float *out, float *wsum, void *stream);

/* Adjoint of dpcs_denoise: dIc (dev, Hc x Wc x 3) += D^T(dOut), i.e.
 * dIc(q) += sum_p w(p,q) dOut(p) / W(p), with wsum = W from the forward call
 * (same guide and params).  dIc must not alias dOut. */
dpcs_status dpcs_denoise_backward(dpcs_ctx *ctx, const float *dOut, const float *guide, const float *wsum,
                                  int32_t Hc, int32_t Wc, const dpcs_denoise_params *params, float *dIc,
                                  void *stream);

/*
 * dpcs_render that also keeps every path's vertex records on the device, so
 * that the adjoint of a loss that is not per-pixel (e.g. after the Eq. 11
 * filter) can run without tracing the paths again.  Arguments and results
 * are those of dpcs_render (Ic and Ec equal bit for bit).  The records
 * (96 B per recorded vertex: ceil(spp / L) samples x `bounces` vertices per
 * lane, L lanes per pixel, L = min(32, the largest power of two <= spp))
 * live in context scratch, counted against the HBM budget, until the next
 * dpcs_render_keep; DPCS_ERR_OOM if they do not fit.
 *
 * dpcs_render_backward_kept: the adjoint of the last dpcs_render_keep call,
 * with the arguments and outputs of dpcs_render_backward.  The call must
 * repeat that render's arguments (scene, textures, Ip, view, params, spp,
 * bounces, seed); the scene, image size, spp, bounces and seed are checked
 * (DPCS_ERR_INVALID_ARG when they differ).  It runs the reverse sweeps over
 * the kept records instead of re-tracing.
 */
dpcs_status dpcs_render_keep(dpcs_ctx *ctx, dpcs_scene scene, const float *albedo, const float *rough, int32_t Ht,
                             int32_t Wt, const float *Ip, const dpcs_view *view, const dpcs_params *params,
                             int32_t spp, int32_t bounces, uint64_t seed, float *Ic, float *Ec, void *stream);
dpcs_status dpcs_render_backward_kept(dpcs_ctx *ctx, dpcs_scene scene, const float *albedo, const float *rough,
                                      int32_t Ht, int32_t Wt, const float *Ip, const dpcs_view *view,
                                      const dpcs_params *params, int32_t spp, int32_t bounces, uint64_t seed,
                                      const float *Ec, const float *Ic, const float *dIc, float *dIp, float *dAlbedo,
                                      float *dRough, float *dParams, void *stream);

/*
 * Forward render, per-pixel loss and adjoint in one call, for the losses of
 * Eqs. 13 and 9 that compare each pixel with a target on its own:
 *   loss_kind 0 (L2): *loss = 1/2 scale sum |Ic - target|^2, dLoss/dIc = scale (Ic - target)
 *   loss_kind 1 (L1): *loss = scale sum |Ic - target|,       dLoss/dIc = scale sign(Ic - target)
 * Inputs are those of dpcs_render plus target (dev, Hc x Wc x 3); Ic (dev,
 * required) and Ec (dev, may be NULL) receive the forward results, equal bit
 * for bit to dpcs_render's; *loss (dev float) the loss; dIp, dAlbedo,
 * dRough, dParams are ACCUMULATED as in dpcs_render_backward.
 * When every lane's paths fit its vertex records (ceil(spp / L) samples of
 * `bounces` vertices, at most 4 samples and 12 vertices; L is the lanes per
 * pixel, min(32, the largest power of two <= spp)), each path is traced
 * once: the warp renders its pixels, derives dLoss/dEc from them and sweeps
 * the recorded vertices backwards.  Otherwise the call renders, takes the
 * loss and replays the paths, as the separate calls would.
 */
dpcs_status dpcs_render_loss_backward(dpcs_ctx *ctx, dpcs_scene scene, const float *albedo, const float *rough,
                                      int32_t Ht, int32_t Wt, const float *Ip, const dpcs_view *view,
                                      const dpcs_params *params, int32_t spp, int32_t bounces, uint64_t seed,
                                      const float *target, int32_t loss_kind, float scale, float *Ic, float *Ec,
                                      float *loss, float *dIp, float *dAlbedo, float *dRough, float *dParams,
                                      void *stream);

/*
 * L2 image loss of projector compensation (Eq. 13 with a squared norm):
 * loss = 1/2 sum (Ic - target)^2 written to *loss (dev, 1 float32, overwritten),
 * dIc = Ic - target (dev, n floats, overwritten).  n = number of floats.
 */
dpcs_status dpcs_l2_loss(dpcs_ctx *ctx, const float *Ic, const float *target, int64_t n, float *dIc, float *loss,
                         void *stream);

/*
 * One Adam step (Kingma & Ba 2015, bias-corrected; `step` counts from 1) on
 * n float32 parameters p with gradient g and moments m, v (all dev, updated
 * in place), followed by a clamp to [lo, hi] -- the projection that keeps Ip
 * in [0, 1] and the PRF/CRF/white-balance parameters inside the ranges of
 * Sec. 3.2.
 */
dpcs_status dpcs_adam(dpcs_ctx *ctx, float *p, const float *g, float *m, float *v, int64_t n, float lr, float beta1,
                      float beta2, float eps, int32_t step, float lo, float hi, void *stream);

/*
 * Scene-parameter fitting (Eq. 9):
 *   theta* = argmin (1/K) sum_i |R(Ip_i, theta) - Ic_i| + lambda L(m),
 * with |.| read as an L1 norm and L(m) as the total variation of the BRDF
 * maps m (albedo, roughness).  The render_backward outputs of the K pairs
 * accumulate; dpcs_adam with the ranges of Sec. 3.2 as bounds updates the
 * textures and the response parameters.
 *
 * dpcs_l1_loss: dIc (dev, n floats) = scale * sign(Ic - target) (sign(0) =
 * 0), *loss (dev float) = scale * sum |Ic - target| (reduced in FP64).
 * scale > 0 (e.g. 1 / (K n) for the mean over K pairs).
 *
 * dpcs_tv_loss: tex (dev, H x W x C, C <= 4): *loss (dev float) = weight *
 * sum over texels and channels of |m(x+1,y) - m(x,y)| + |m(x,y+1) - m(x,y)|,
 * and grad (dev, same shape) += its derivative (sign terms; 0 at ties).
 */
dpcs_status dpcs_l1_loss(dpcs_ctx *ctx, const float *Ic, const float *target, int64_t n, float scale, float *dIc,
                         float *loss, void *stream);
dpcs_status dpcs_tv_loss(dpcs_ctx *ctx, const float *tex, int32_t H, int32_t W, int32_t C, float weight, float *grad,
                         float *loss, void *stream);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of relighting and compensation requests      */
/* ------------------------------------------------------------------------ */
/*
 * The paper's two downstream tasks -- ProCams relighting, Ic' = R(Ip', theta)
 * (Sec. 3.2, Eq. 7) and projector compensation, Ip* = argmin |R(Ip) - Ic|
 * (Eq. 13) -- served as requests on resident scenes.  The paper runs them
 * one at a time; batching them is this library's addition.
 *
 * A server owns a CUDA stream and device memory for admitted requests.  Each
 * dpcs_serve_step is one scheduler iteration: it retires finished work,
 * admits waiting requests (FIFO) while their device memory fits the HBM
 * budget and fewer than max_active are admitted, and plans about
 * samples_per_iteration camera samples of work: every active relighting
 * request first gets quantum_samples (so short requests finish within an
 * iteration or two); then one compensation step per request (a full-image
 * render, loss, path-replay adjoint and Adam step) within half of the
 * iteration's samples; the rest goes to relighting
 * requests in arrival order, and budget that relighting leaves unused runs
 * further consecutive compensation steps, still within that half.  The relighting pixels run as one batched
 * render; the compensation steps follow on the same stream.  Requests that
 * arrive while others run join at the next iteration.  A pixel's result is computed exactly as dpcs_render computes
 * it, whatever else is in the batch.  Waits are bounded; nothing spins on
 * the GPU.  A server is not thread safe; use it from one host thread.
 */
typedef struct dpcs_server dpcs_server;

typedef struct dpcs_serve_config {
    size_t hbm_budget_bytes;        /* device memory for admitted requests (0 = no limit) */
    int32_t max_active;             /* most requests admitted at once (1..1024) */
    int32_t max_inflight;           /* batched iterations queued on the GPU at once (1..4) */
    int64_t samples_per_iteration;  /* camera samples one batched iteration aims at */
    int64_t quantum_samples;        /* samples every active relighting request gets first */
    /* How an iteration is shared.  DPCS_SERVE_FIXED_SHARE: every relighting
     * request first gets quantum_samples, then one compensation step per
     * request within compensation_share of the iteration, the rest to
     * relighting in arrival order, and what relighting leaves to further
     * compensation steps.  DPCS_SERVE_DEADLINE: by earliest deadline, a
     * request's deadline being its arrival plus slack x its work /
     * est_samples_per_s (a compensation step counts its samples x 1.4 for
     * the adjoint); no quanta.  DPCS_SERVE_QUANTA_DEADLINE: the relighting
     * quanta first, then the rest by earliest deadline (deadline fields as
     * for DPCS_SERVE_DEADLINE; no cap on compensation). */
    int32_t policy;
    int32_t pad;
    double relight_slack;           /* deadline policies, > 0 */
    double compensation_slack;      /* deadline policies, > 0 */
    double est_samples_per_s;       /* deadline policies, > 0: the throughput the deadlines assume */
    double compensation_share;      /* fixed-share policy, in (0, 1] */
} dpcs_serve_config;
#define DPCS_SERVE_DEADLINE 0
#define DPCS_SERVE_FIXED_SHARE 1
#define DPCS_SERVE_QUANTA_DEADLINE 2

#define DPCS_REQ_RELIGHT 0
#define DPCS_REQ_COMPENSATE 1

#define DPCS_REQ_WAITING 0
#define DPCS_REQ_ACTIVE 1
#define DPCS_REQ_DONE 2
#define DPCS_REQ_FAILED (-1)

typedef struct dpcs_request {
    int32_t kind;          /* DPCS_REQ_RELIGHT or DPCS_REQ_COMPENSATE */
    int32_t scene;         /* slot returned by dpcs_serve_add_scene */
    int32_t Hc, Wc;        /* camera image; the scene camera's field of view is kept */
    int32_t spp;           /* samples per pixel */
    uint64_t seed;         /* Philox key; compensation step k uses seed + k */
    int32_t steps;         /* compensation: Adam steps (Eq. 13) */
    float lr;              /* compensation: Adam learning rate */
    const float *Ip;       /* host, Hp x Wp x 3: the image to relight / the compensation start */
    const float *target;   /* host, Hc x Wc x 3: compensation target Ic (NULL for relighting) */
    float *Ic_out;         /* host, Hc x Wc x 3: rendered image (compensation: of the last step) */
    float *Ip_out;         /* host, Hp x Wp x 3: compensated projector image, or NULL */
} dpcs_request;

typedef struct dpcs_serve_stats {
    int64_t submitted, completed, failed, waiting, active;
    int64_t iterations, launches;
    size_t memory_used, memory_high_water;
} dpcs_serve_stats;

/* Create a server on ctx's device.  The host buffers of a request must stay
 * valid until it is done. */
dpcs_status dpcs_serve_create(dpcs_ctx *ctx, const dpcs_serve_config *cfg, dpcs_server **out);
/* Wait (bounded by the GPU work queued) and free everything. */
dpcs_status dpcs_serve_destroy(dpcs_server *srv);
/* Register a resident scene with its textures (dev, caller-owned, kept
 * unchanged while the server lives), the scene's camera/projector and
 * parameters; *slot receives its index. */
dpcs_status dpcs_serve_add_scene(dpcs_server *srv, dpcs_scene scene, const float *albedo, const float *rough,
                                 int32_t Ht, int32_t Wt, const dpcs_view *view, const dpcs_params *params,
                                 int32_t bounces, int32_t *slot);
/* Queue a request; *id receives its handle.  Sizes are validated here. */
dpcs_status dpcs_serve_submit(dpcs_server *srv, const dpcs_request *req, uint64_t *id);
/* One scheduler iteration (see above); *completed (may be NULL) receives the
 * number of requests that finished during it.  Returns without waiting
 * unless max_inflight iterations are already queued on the GPU. */
dpcs_status dpcs_serve_step(dpcs_server *srv, int32_t *completed);
/* State of request id (DPCS_REQ_*) and, once done, its latency in ms from
 * submission to the moment the server saw its result in host memory. */
dpcs_status dpcs_serve_query(dpcs_server *srv, uint64_t id, int32_t *state, double *latency_ms);
/* Step until no request is waiting or active, for at most timeout_s seconds
 * (DPCS_ERR_TIMEOUT after that). */
dpcs_status dpcs_serve_drain(dpcs_server *srv, double timeout_s);
dpcs_status dpcs_serve_stats_get(dpcs_server *srv, dpcs_serve_stats *out);

#ifdef __cplusplus
}
#endif

#endif /* DPCS_H */
