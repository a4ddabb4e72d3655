/*
 * dpcs_oracle.c -- FP64 CPU oracle for the DPCS projector-camera path tracer.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file: only the tests, the smoke check and the benchmark's CPU-baseline
 * leg use it.  It shares no code, header, table or constant generator with the
 * CUDA library.
 *
 * What it computes (arxiv 2503.12174, "DPCS: Path Tracing-Based Differentiable
 * Projector-Camera Systems", Sec. 3):
 *   - Eq. 1   PRF:  Ep = Gp * Ip^gamma_p                      (prf_texel)
 *   - Eq. 2   projector radiance Lp = Ep / phi, folded into k (nee)
 *   - Eq. 3   rendering equation, estimated by Eq. 10          (trace_sample)
 *   - Eq. 4   camera irradiance = mean over pixel samples      (or_render)
 *   - Eq. 5   CRF + white balance: Ic = (Gc w Ec)^gamma_c      (crf)
 *   - Eq. 6   projection xc = Kc xs, xp = Kp [Rp|tp] xs        (camera ray, nee)
 *   - Eq. 12  radiance clipping (optional, off when clip == 0)
 *   - Eq. 11  the guide features of the cross-bilateral denoiser (or_gbuffer;
 *             the filter itself is in oracle.py)
 *   - Sec. 3.2's scene parameters m and Vn: the principled BRDF's metallic
 *     map and the normal map (or_render_m / or_render_backward_m; NULL maps
 *     give metallic 0 and the unperturbed normal, i.e. or_render)
 *   - the analytic adjoint of the same estimator with the sampled directions
 *     held fixed (detached sampling), used by projector compensation (Eq. 13)
 *     and scene-parameter fitting (Eq. 9).
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   - the projector is a pinhole point emitter at cp = -Rp^T tp with radiant
 *     intensity k * Ep(xp) * cos(theta_p); irradiance at xs is that times
 *     cos(theta_s) / r^2.  NEE is the only projector estimator.
 *   - PRF is applied per projector texel, then Ep is bilinearly interpolated
 *     with texel centres at (i + 1/2) and clamp-to-edge; outside [0,Wp)x[0,Hp)
 *     or behind the projector there is no light.
 *   - camera: pinhole at the world origin, OpenCV axes, pixel (i,j) spans
 *     [i,i+1)x[j,j+1), box filter by uniform jitter (or pixel centre).
 *   - BRDF: Lambert rho/pi + ks * D G F / (4 cos_i cos_o), GGX D with
 *     alpha = r^2 (r clamped to [0.01, 1]), separable Smith G, Schlick F.
 *     Sampling: probability 1/2 cosine lobe, 1/2 GGX visible normals (Heitz
 *     2018); when ks == 0 only the cosine lobe is sampled.
 *   - Russian roulette from vertex rr_start on with a fixed survival q.
 *   - random numbers: Philox4x32-10 (Salmon et al., SC'11), key = seed,
 *     counter = (pixel, sample, vertex, 0); u = (x >> 8) * 2^-24.
 *   - local shading frame: Duff et al. (JCGT 2017) with its seam at n.z = -1/pi.
 *   - metallic m (Burley 2012's metallic workflow): diffuse weight (1 - m),
 *     Schlick F0 per channel (1 - m) f0 + m rho.
 *   - normal map: Vn in [0,1]^3 decodes to v = 2 Vn - 1 in the tangent frame
 *     (T = dp/du made orthogonal to the geometric normal N turned towards
 *     the incoming ray, B = N x T); the shading normal is v / |v| in that
 *     frame and replaces N in the BRDF, its sampling and both cosines.  N
 *     stays the ray-offset direction, and light or continuations below the
 *     geometric surface are dropped.
 *   - Morton codes in FP32 without contraction (this file is compiled with
 *     -ffp-contract=off), 10 bits per axis, x in the highest bit of each triple.
 *
 * Everything else is FP64.  Ray-triangle tests are brute force over all
 * triangles in their original order (Moller-Trumbore 1997); ties in t go to the
 * lowest triangle index.  A timing mode (or_set_accel(1)) tests only the
 * triangles whose padded boxes a median-split BVH cannot cull; it returns the
 * same hits, so its images equal the brute-force ones bit for bit.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846
#define OR_MAX_VERTS 16
#define OR_RAY_EPS 1e-4

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, from its published definition (Salmon, Moraes, Dror, Shaw,  */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11): each round takes    */
/* the two 32x32->64 products M0*c0 and M1*c2 and permutes/xors the halves    */
/* with the counter and the round key; the key is bumped by the Weyl          */
/* constants between rounds.                                                  */
/* ------------------------------------------------------------------------- */
static void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}

void or_philox(const uint32_t *ctr, int64_t n, uint64_t seed, uint32_t *out)
{
    for (int64_t i = 0; i < n; ++i) {
        uint32_t c[4] = {ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
        philox4x32_10(c, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
        memcpy(out + 4 * i, c, sizeof c);
    }
}

/* the four uniforms of one (pixel, sample, vertex) counter, 24-bit exact */
static void rand4(uint64_t seed, uint32_t pix, uint32_t s, uint32_t b, double u[4])
{
    uint32_t c[4] = {pix, s, b, 0u};
    philox4x32_10(c, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
    for (int i = 0; i < 4; ++i) u[i] = (double)(c[i] >> 8) * (1.0 / 16777216.0);
}

/* ------------------------------------------------------------------------- */
/* small vector algebra                                                       */
/* ------------------------------------------------------------------------- */
typedef struct { double x, y, z; } d3;
static d3 mk(double x, double y, double z) { d3 r = {x, y, z}; return r; }
static d3 add(d3 a, d3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static d3 sub(d3 a, d3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static d3 scl(d3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static d3 cross(d3 a, d3 b)
{
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static double len(d3 a) { return sqrt(dot(a, a)); }
static d3 nrm(d3 a) { return scl(a, 1.0 / len(a)); }
static d3 mat3v(const double *M, d3 v)
{
    return mk(M[0] * v.x + M[1] * v.y + M[2] * v.z, M[3] * v.x + M[4] * v.y + M[5] * v.z,
              M[6] * v.x + M[7] * v.y + M[8] * v.z);
}
static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

static void inv3(const double *M, double *R)
{
    double a = M[0], b = M[1], c = M[2], d = M[3], e = M[4], f = M[5], g = M[6], h = M[7], i = M[8];
    double A = e * i - f * h, B = -(d * i - f * g), C = d * h - e * g;
    double det = a * A + b * B + c * C;
    R[0] = A / det; R[1] = -(b * i - c * h) / det; R[2] = (b * f - c * e) / det;
    R[3] = B / det; R[4] = (a * i - c * g) / det;  R[5] = -(a * f - c * d) / det;
    R[6] = C / det; R[7] = -(a * h - b * g) / det; R[8] = (a * e - b * d) / det;
}

/* ------------------------------------------------------------------------- */
/* Parameters, view and scene as the callers hand them over                   */
/* ------------------------------------------------------------------------- */
typedef struct {
    double gamma_p[3], gain_p;    /* Eq. 1 */
    double gamma_c[3], gain_c;    /* Eq. 5 */
    double wb[3];                 /* Eq. 5 white balance */
    double k_proj;                /* Eq. 2 / Eq. 12 projector scale k (plays 1/phi) */
    double ks, f0;                /* specular lobe weight and Schlick F0 */
    int32_t rr_start;             /* first vertex subject to Russian roulette, 0 = off */
    double rr_q;                  /* survival probability */
    double clip;                  /* Eq. 12 clamp, 0 = off */
    int32_t jitter;               /* 1 = box-filter jitter, 0 = pixel centre */
} or_params;

typedef struct {
    double Kc[9]; int32_t Hc, Wc;                 /* camera at the origin (Eq. 6) */
    double Kp[9], Rp[9], tp[3]; int32_t Hp, Wp;   /* projector (Eq. 6) */
} or_view;

/* timing-mode acceleration: a median-split BVH over the same FP64 triangles */
typedef struct {
    double lo[3], hi[3];  /* box, padded outwards so that culling is conservative */
    int left, right;      /* children, or -1 for a leaf */
    int first, count;     /* leaf: range of bvh_idx */
} bnode;

typedef struct {
    int T;
    d3 *v0, *e1, *e2; /* FP64 copies of the FP32 input: differences are exact */
    double *uv;       /* 6 per triangle */
    bnode *nodes;     /* NULL in parity mode (brute force) */
    int *bvh_idx;     /* triangle indices in leaf order */
    int nnodes;
} dscene;

/* 0 = parity mode (brute force), 1 = timing mode (BVH); set by the caller
 * before a render, read by scene_make */
static int g_accel = 0;
void or_set_accel(int on) { g_accel = on ? 1 : 0; }

/* Adjoint diagnostics: 1 = scatter every projector and albedo contribution
 * to its four bilinear taps with weight 1 instead of the tap's weight.  With
 * dLoss/dIc replaced by its absolute value, every such contribution is
 * nonnegative, and the result is, per texel, the total size of the
 * contributions that reach it through any tap -- the scale by which rounding
 * of a tap's weight (the FP32 position of the hit point in texel units) can
 * move that texel's gradient.  Off in every parity computation. */
static int g_unit_taps = 0;
void or_set_unit_taps(int on) { g_unit_taps = on ? 1 : 0; }
static void bvh_build(dscene *S);

static void scene_make(dscene *S, const float *verts, const int32_t *tris, int32_t T, const float *uv)
{
    S->T = T;
    S->v0 = (d3 *)malloc(sizeof(d3) * (size_t)(T > 0 ? T : 1));
    S->e1 = (d3 *)malloc(sizeof(d3) * (size_t)(T > 0 ? T : 1));
    S->e2 = (d3 *)malloc(sizeof(d3) * (size_t)(T > 0 ? T : 1));
    S->uv = (double *)malloc(sizeof(double) * 6 * (size_t)(T > 0 ? T : 1));
    for (int i = 0; i < T; ++i) {
        const float *a = verts + 3 * tris[3 * i], *b = verts + 3 * tris[3 * i + 1], *c = verts + 3 * tris[3 * i + 2];
        d3 A = mk(a[0], a[1], a[2]), B = mk(b[0], b[1], b[2]), C = mk(c[0], c[1], c[2]);
        S->v0[i] = A; S->e1[i] = sub(B, A); S->e2[i] = sub(C, A);
        for (int k = 0; k < 3; ++k) {
            S->uv[6 * i + 2 * k] = uv[2 * tris[3 * i + k]];
            S->uv[6 * i + 2 * k + 1] = uv[2 * tris[3 * i + k] + 1];
        }
    }
    S->nodes = NULL; S->bvh_idx = NULL; S->nnodes = 0;
    if (g_accel && T > 0) bvh_build(S);
}
static void scene_free(dscene *S)
{
    free(S->v0); free(S->e1); free(S->e2); free(S->uv);
    free(S->nodes); free(S->bvh_idx);
}

/* Moller-Trumbore (1997), two-sided, t in (tmin, tmax) */
static int isect(const dscene *S, int i, d3 o, d3 d, double tmin, double tmax, double *t, double *bu, double *bv)
{
    d3 p = cross(d, S->e2[i]);
    double det = dot(S->e1[i], p);
    if (det == 0.0) return 0;
    double inv = 1.0 / det;
    d3 s = sub(o, S->v0[i]);
    double u = dot(s, p) * inv;
    if (u < 0.0 || u > 1.0) return 0;
    d3 q = cross(s, S->e1[i]);
    double v = dot(d, q) * inv;
    if (v < 0.0 || u + v > 1.0) return 0;
    double tt = dot(S->e2[i], q) * inv;
    if (!(tt > tmin && tt < tmax)) return 0;
    *t = tt; *bu = u; *bv = v;
    return 1;
}

/* brute-force closest hit; strict '<' keeps the lowest index on ties */
static int closest_brute(const dscene *S, d3 o, d3 d, double tmax, double *t, double *bu, double *bv)
{
    int best = -1;
    double bt = tmax, tu = 0, tv = 0;
    for (int i = 0; i < S->T; ++i) {
        double tt, uu, vv;
        if (isect(S, i, o, d, 0.0, bt, &tt, &uu, &vv) && tt < bt) { bt = tt; best = i; tu = uu; tv = vv; }
    }
    if (best >= 0) { *t = bt; *bu = tu; *bv = tv; }
    return best;
}

static int occluded_brute(const dscene *S, d3 o, d3 d, double tmax)
{
    for (int i = 0; i < S->T; ++i) {
        double tt, uu, vv;
        if (isect(S, i, o, d, 0.0, tmax, &tt, &uu, &vv)) return 1;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Timing mode: a median-split BVH (longest centroid axis, leaves of <= 4     */
/* triangles).  It changes which triangles are tested, never how: each test   */
/* is isect() above, and the closest hit is the lexicographic minimum of      */
/* (t, triangle index), which is what the brute-force loop returns.  Boxes    */
/* are padded and the slab test widened, so a box is culled only when no     */
/* point of it can lie on the ray within the current bound.                   */
/* ------------------------------------------------------------------------- */
typedef struct { const dscene *S; double *cen; int *idx; } bvh_ctx;

static void tri_box(const dscene *S, int i, double lo[3], double hi[3])
{
    d3 a = S->v0[i], b = add(S->v0[i], S->e1[i]), c = add(S->v0[i], S->e2[i]);
    double pa[3] = {a.x, a.y, a.z}, pb[3] = {b.x, b.y, b.z}, pc[3] = {c.x, c.y, c.z};
    for (int k = 0; k < 3; ++k) {
        lo[k] = fmin(pa[k], fmin(pb[k], pc[k]));
        hi[k] = fmax(pa[k], fmax(pb[k], pc[k]));
    }
}

/* partial sort of idx[first, last) so that position mid holds the element of
 * rank mid by centroid coordinate `axis` (Hoare's selection) */
static void select_mid(bvh_ctx *B, int first, int last, int mid, int axis)
{
    int *v = B->idx;
    while (last - first > 1) {
        double piv = B->cen[3 * v[(first + last) / 2] + axis];
        int i = first, j = last - 1;
        while (i <= j) {
            while (B->cen[3 * v[i] + axis] < piv) ++i;
            while (B->cen[3 * v[j] + axis] > piv) --j;
            if (i <= j) { int t = v[i]; v[i] = v[j]; v[j] = t; ++i; --j; }
        }
        if (mid <= j) last = j + 1;
        else if (mid >= i) first = i;
        else return;
    }
}

static int bvh_node(bvh_ctx *B, dscene *S, int first, int last)
{
    int id = S->nnodes++;
    bnode *N = &S->nodes[id];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int k = first; k < last; ++k) {
        double tl[3], th[3];
        tri_box(S, B->idx[k], tl, th);
        for (int a = 0; a < 3; ++a) {
            lo[a] = fmin(lo[a], tl[a]); hi[a] = fmax(hi[a], th[a]);
            clo[a] = fmin(clo[a], B->cen[3 * B->idx[k] + a]); chi[a] = fmax(chi[a], B->cen[3 * B->idx[k] + a]);
        }
    }
    for (int a = 0; a < 3; ++a) {  /* pad: far above FP64 rounding of the hit point */
        double pad = 1e-9 * (fabs(lo[a]) + fabs(hi[a]) + (hi[a] - lo[a])) + 1e-12;
        N->lo[a] = lo[a] - pad; N->hi[a] = hi[a] + pad;
    }
    if (last - first <= 4) {
        N->left = N->right = -1; N->first = first; N->count = last - first;
        return id;
    }
    int axis = 0;
    for (int a = 1; a < 3; ++a)
        if (chi[a] - clo[a] > chi[axis] - clo[axis]) axis = a;
    int mid = (first + last) / 2;
    select_mid(B, first, last, mid, axis);
    N->first = first; N->count = 0;
    int l = bvh_node(B, S, first, mid);
    int r = bvh_node(B, S, mid, last);
    S->nodes[id].left = l;
    S->nodes[id].right = r;
    return id;
}

static void bvh_build(dscene *S)
{
    int T = S->T;
    S->nodes = (bnode *)malloc(sizeof(bnode) * (size_t)(2 * T));
    S->bvh_idx = (int *)malloc(sizeof(int) * (size_t)T);
    double *cen = (double *)malloc(sizeof(double) * 3 * (size_t)T);
    for (int i = 0; i < T; ++i) {
        d3 c = add(S->v0[i], scl(add(S->e1[i], S->e2[i]), 1.0 / 3.0));
        cen[3 * i] = c.x; cen[3 * i + 1] = c.y; cen[3 * i + 2] = c.z;
        S->bvh_idx[i] = i;
    }
    bvh_ctx B = {S, cen, S->bvh_idx};
    S->nnodes = 0;
    bvh_node(&B, S, 0, T);
    free(cen);
}

/* ray-box overlap within [0, tmax], conservative (the far bound is widened) */
static int box_hit(const bnode *N, d3 o, d3 d, double tmax, double *tnear)
{
    double oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
    double tn = 0.0, tf = tmax;
    for (int a = 0; a < 3; ++a) {
        if (dd[a] == 0.0) {
            if (oo[a] < N->lo[a] || oo[a] > N->hi[a]) return 0;
            continue;
        }
        double t0 = (N->lo[a] - oo[a]) / dd[a], t1 = (N->hi[a] - oo[a]) / dd[a];
        if (t0 > t1) { double t = t0; t0 = t1; t1 = t; }
        if (t0 > tn) tn = t0;
        if (t1 < tf) tf = t1;
    }
    *tnear = tn;
    return tn <= tf * (1.0 + 1e-12) + 1e-300;
}

static int closest_bvh(const dscene *S, d3 o, d3 d, double tmax, double *t, double *bu, double *bv)
{
    int best = -1;
    double bt = tmax, tu = 0, tv = 0;
    int stack[128], sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const bnode *N = &S->nodes[stack[--sp]];
        double tn;
        if (!box_hit(N, o, d, bt, &tn)) continue;
        if (N->left < 0) {
            for (int k = N->first; k < N->first + N->count; ++k) {
                int i = S->bvh_idx[k];
                double tt, uu, vv;
                if (isect(S, i, o, d, 0.0, tmax, &tt, &uu, &vv) && (tt < bt || (tt == bt && best >= 0 && i < best))) {
                    bt = tt; best = i; tu = uu; tv = vv;
                }
            }
        } else {
            stack[sp++] = N->right;
            stack[sp++] = N->left;
        }
    }
    if (best >= 0) { *t = bt; *bu = tu; *bv = tv; }
    return best;
}

static int occluded_bvh(const dscene *S, d3 o, d3 d, double tmax)
{
    int stack[128], sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const bnode *N = &S->nodes[stack[--sp]];
        double tn;
        if (!box_hit(N, o, d, tmax, &tn)) continue;
        if (N->left < 0) {
            for (int k = N->first; k < N->first + N->count; ++k) {
                double tt, uu, vv;
                if (isect(S, S->bvh_idx[k], o, d, 0.0, tmax, &tt, &uu, &vv)) return 1;
            }
        } else {
            stack[sp++] = N->right;
            stack[sp++] = N->left;
        }
    }
    return 0;
}

static int closest(const dscene *S, d3 o, d3 d, double tmax, double *t, double *bu, double *bv)
{
    return S->nodes ? closest_bvh(S, o, d, tmax, t, bu, bv) : closest_brute(S, o, d, tmax, t, bu, bv);
}

static int occluded(const dscene *S, d3 o, d3 d, double tmax)
{
    return S->nodes ? occluded_bvh(S, o, d, tmax) : occluded_brute(S, o, d, tmax);
}

void or_closest(const float *verts, int32_t V, const int32_t *tris, int32_t T, const float *uv,
                const double *o, const double *d, int64_t n, double *t_out, int32_t *tri_out)
{
    (void)V;
    dscene S;
    scene_make(&S, verts, tris, T, uv);
    for (int64_t r = 0; r < n; ++r) {
        double t = 0, bu, bv;
        int h = closest(&S, mk(o[3 * r], o[3 * r + 1], o[3 * r + 2]), mk(d[3 * r], d[3 * r + 1], d[3 * r + 2]),
                        INFINITY, &t, &bu, &bv);
        tri_out[r] = h;
        t_out[r] = h >= 0 ? t : INFINITY;
    }
    scene_free(&S);
}

/* ------------------------------------------------------------------------- */
/* LBVH reference (integer work must match bit for bit):                       */
/* Morton codes of FP32 centroids, sort of (code, index), binary radix tree   */
/* over the sorted keys built top-down from its definition (each internal     */
/* node splits its key range where the highest differing bit flips; keys are  */
/* augmented by their sorted position), AABBs as FP32 unions.  Node numbering */
/* follows Karras (HPG 2012): the root is 0, a left child that is internal is */
/* numbered by its last key, a right child by its first key.                  */
/* ------------------------------------------------------------------------- */
static uint32_t expand10(uint32_t v)
{
    uint32_t r = 0;
    for (int i = 0; i < 10; ++i) r |= ((v >> i) & 1u) << (3 * i);
    return r;
}

void or_morton(const float *verts, const int32_t *tris, int32_t T, uint32_t *codes)
{
    if (T <= 0) return;
    float *c = (float *)malloc(sizeof(float) * 3 * (size_t)T);
    const float third = 1.0f / 3.0f;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = 0; i < T; ++i)
        for (int k = 0; k < 3; ++k) {
            float a = verts[3 * tris[3 * i] + k], b = verts[3 * tris[3 * i + 1] + k], e = verts[3 * tris[3 * i + 2] + k];
            float s = a + b;
            s = s + e;
            float m = s * third;
            c[3 * i + k] = m;
            if (m < lo[k]) lo[k] = m;
            if (m > hi[k]) hi[k] = m;
        }
    float inv[3];
    for (int k = 0; k < 3; ++k) {
        float ext = hi[k] - lo[k];
        inv[k] = ext > 0.0f ? 1.0f / ext : 0.0f;
    }
    for (int i = 0; i < T; ++i) {
        uint32_t q[3];
        for (int k = 0; k < 3; ++k) {
            float nrmd = (c[3 * i + k] - lo[k]) * inv[k];
            float sc = nrmd * 1024.0f;
            float f = floorf(sc);
            if (f < 0.0f) f = 0.0f;
            if (f > 1023.0f) f = 1023.0f;
            q[k] = (uint32_t)f;
        }
        codes[i] = (expand10(q[0]) << 2) | (expand10(q[1]) << 1) | expand10(q[2]);
    }
    free(c);
}

typedef struct { uint32_t code; int32_t idx; } kv;
static int kv_cmp(const void *a, const void *b)
{
    const kv *x = (const kv *)a, *y = (const kv *)b;
    if (x->code != y->code) return x->code < y->code ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

static int clz64(uint64_t x)
{
    if (x == 0) return 64;
    int n = 0;
    while (!(x & 0x8000000000000000ull)) { x <<= 1; ++n; }
    return n;
}

typedef struct {
    const uint32_t *code;   /* sorted codes */
    int32_t *child;         /* 2 per internal node; >= 0 internal, < 0 leaf ~pos */
} radix_ctx;

static uint64_t akey(const radix_ctx *R, int i) { return ((uint64_t)R->code[i] << 32) | (uint32_t)i; }

static void radix_build(radix_ctx *R, int first, int last, int id)
{
    int common = clz64(akey(R, first) ^ akey(R, last));
    int split = first;
    for (int s = first; s < last; ++s)
        if (clz64(akey(R, first) ^ akey(R, s)) > common) split = s;
    int left = (split == first) ? ~split : split;
    int right = (split + 1 == last) ? ~(split + 1) : split + 1;
    R->child[2 * id] = left;
    R->child[2 * id + 1] = right;
    if (left >= 0) radix_build(R, first, split, left);
    if (right >= 0) radix_build(R, split + 1, last, right);
}

/* box of child reference c: leaf -> triangle bounds, internal -> union */
static void ref_box(const float *verts, const int32_t *tris, const int32_t *order, const int32_t *child, int c,
                    float b[6])
{
    if (c < 0) {
        int t = order[~c];
        for (int k = 0; k < 3; ++k) {
            float x0 = verts[3 * tris[3 * t] + k], x1 = verts[3 * tris[3 * t + 1] + k], x2 = verts[3 * tris[3 * t + 2] + k];
            float lo = x0 < x1 ? x0 : x1, hi = x0 > x1 ? x0 : x1;
            lo = lo < x2 ? lo : x2; hi = hi > x2 ? hi : x2;
            b[k] = lo; b[3 + k] = hi;
        }
        return;
    }
    float l[6], r[6];
    ref_box(verts, tris, order, child, child[2 * c], l);
    ref_box(verts, tris, order, child, child[2 * c + 1], r);
    for (int k = 0; k < 3; ++k) {
        b[k] = l[k] < r[k] ? l[k] : r[k];
        b[3 + k] = l[3 + k] > r[3 + k] ? l[3 + k] : r[3 + k];
    }
}

/* outputs: sorted codes [T], triangle index per sorted position [T],
 * child refs [(T-1)*2], child boxes [(T-1)*2*6] as (lo.xyz, hi.xyz) */
void or_lbvh(const float *verts, const int32_t *tris, int32_t T, uint32_t *sorted_codes, int32_t *order,
             int32_t *child, float *child_box)
{
    if (T <= 0) return;
    uint32_t *codes = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)T);
    or_morton(verts, tris, T, codes);
    kv *a = (kv *)malloc(sizeof(kv) * (size_t)T);
    for (int i = 0; i < T; ++i) { a[i].code = codes[i]; a[i].idx = i; }
    qsort(a, (size_t)T, sizeof(kv), kv_cmp);
    for (int i = 0; i < T; ++i) { sorted_codes[i] = a[i].code; order[i] = a[i].idx; }
    if (T >= 2) {
        radix_ctx R = {sorted_codes, child};
        radix_build(&R, 0, T - 1, 0);
        for (int n = 0; n < T - 1; ++n)
            for (int s = 0; s < 2; ++s) ref_box(verts, tris, order, child, child[2 * n + s], child_box + 12 * n + 6 * s);
    }
    free(a);
    free(codes);
}

/* ------------------------------------------------------------------------- */
/* BRDF (Lambert + GGX), evaluation, derivative in roughness, sampling, pdf   */
/* ------------------------------------------------------------------------- */
static double alpha_of(double r, double *dadr)
{
    double rc = r;
    double d = 2.0 * r;
    if (rc < 0.01) { rc = 0.01; d = 0.0; }
    if (rc > 1.0) { rc = 1.0; d = 0.0; }
    *dadr = d;
    return rc * rc;
}

/* GGX normal distribution D(h) for cos(theta_h) = ch */
static double ggx_D(double ch, double a)
{
    double a2 = a * a;
    double t = ch * ch * (a2 - 1.0) + 1.0;
    return a2 / (OR_PI * t * t);
}
double or_ggx_D(double ch, double a) { return ggx_D(ch, a); }

/* Smith masking for GGX, G1 = 2c / (c + sqrt(a^2 + (1 - a^2) c^2)) */
static double ggx_G1(double c, double a)
{
    double a2 = a * a;
    double s = sqrt(a2 + (1.0 - a2) * c * c);
    return 2.0 * c / (c + s);
}

/* specular term D G F / (4 ci co) (without ks) and its derivative in alpha */
static double spec_term(d3 n, d3 wo, d3 wi, double a, double f0, double *dspec_da)
{
    double co = dot(n, wo), ci = dot(n, wi);
    *dspec_da = 0.0;
    if (co <= 0.0 || ci <= 0.0) return 0.0;
    d3 h = nrm(add(wo, wi));
    double ch = dot(n, h);
    double a2 = a * a;
    double t = ch * ch * (a2 - 1.0) + 1.0;
    double D = a2 / (OR_PI * t * t);
    double si = sqrt(a2 + (1.0 - a2) * ci * ci), so = sqrt(a2 + (1.0 - a2) * co * co);
    double G = (2.0 * ci / (ci + si)) * (2.0 * co / (co + so));
    double m = 1.0 - dot(wo, h);
    if (m < 0.0) m = 0.0;
    double F = f0 + (1.0 - f0) * m * m * m * m * m;
    double spec = D * G * F / (4.0 * ci * co);
    /* d ln D / da = 2/a - 4 a ch^2 / t ; d ln G1 / da = -(a (1 - c^2) / s) / (c + s) */
    double dlnD = 2.0 / a - 4.0 * a * ch * ch / t;
    double dlnG = -(a * (1.0 - ci * ci) / si) / (ci + si) - (a * (1.0 - co * co) / so) / (co + so);
    *dspec_da = spec * (dlnD + dlnG);
    return spec;
}

/* f(wo, wi) per channel; *dfdr = d f / d r (same for all channels) */
static void bsdf_eval(d3 n, d3 wo, d3 wi, const double rho[3], double r, double ks, double f0, double f[3],
                      double *dfdr)
{
    double ci = dot(n, wi), co = dot(n, wo);
    if (ci <= 0.0 || co <= 0.0) { f[0] = f[1] = f[2] = 0.0; *dfdr = 0.0; return; }
    double dadr, a = alpha_of(r, &dadr), dsda = 0.0;
    double sp = ks > 0.0 ? ks * spec_term(n, wo, wi, a, f0, &dsda) : 0.0;
    for (int j = 0; j < 3; ++j) f[j] = rho[j] / OR_PI + sp;
    *dfdr = ks > 0.0 ? ks * dsda * dadr : 0.0;
}

/* Orthonormal basis around n (Duff et al., JCGT 2017).  Every frame field on
 * the sphere has a seam; it is put at n.z = -1/pi instead of n.z = 0 so that
 * the axis-aligned and mirror-symmetric facets common in meshes (n.z exactly
 * 0, or 0 up to rounding) never sit on it.  Both branches stay well
 * conditioned (|sg + n.z| >= 1 - 1/pi). */
static void onb(d3 n, d3 *t, d3 *b)
{
    double sg = n.z >= -0.318309886183790671538 ? 1.0 : -1.0;
    double a = -1.0 / (sg + n.z);
    double bb = n.x * n.y * a;
    *t = mk(1.0 + sg * n.x * n.x * a, sg * bb, -sg * n.x);
    *b = mk(bb, sg + n.y * n.y * a, -n.y);
}

static double spec_prob(double ks) { return ks > 0.0 ? 0.5 : 0.0; }

/* mixture pdf (solid angle) of sampling wi given wo */
static double bsdf_pdf(d3 n, d3 wo, d3 wi, double r, double ks)
{
    double ci = dot(n, wi), co = dot(n, wo);
    if (ci <= 0.0 || co <= 0.0) return 0.0;
    double ps = spec_prob(ks);
    double p = (1.0 - ps) * ci / OR_PI;
    if (ps > 0.0) {
        double dadr, a = alpha_of(r, &dadr);
        d3 h = nrm(add(wo, wi));
        p += ps * ggx_G1(co, a) * ggx_D(dot(n, h), a) / (4.0 * co);
    }
    return p;
}

/* sample wi: u0 picks the lobe, (u1, u2) the direction; returns 0 on failure */
static int bsdf_sample(d3 n, d3 wo, double r, double ks, double u0, double u1, double u2, d3 *wi)
{
    d3 T, B;
    onb(n, &T, &B);
    d3 l;
    if (u0 >= spec_prob(ks)) {
        /* cosine-weighted hemisphere */
        double rr = sqrt(u1), ph = 2.0 * OR_PI * u2;
        l = mk(rr * cos(ph), rr * sin(ph), sqrt(fmax(0.0, 1.0 - u1)));
    } else {
        /* GGX visible-normal sampling (Heitz, JCGT 2018) in the local frame */
        double dadr, a = alpha_of(r, &dadr);
        d3 wl = mk(dot(wo, T), dot(wo, B), dot(wo, n));
        d3 Vh = nrm(mk(a * wl.x, a * wl.y, wl.z));
        double lsq = Vh.x * Vh.x + Vh.y * Vh.y;
        d3 T1 = lsq > 0.0 ? scl(mk(-Vh.y, Vh.x, 0.0), 1.0 / sqrt(lsq)) : mk(1.0, 0.0, 0.0);
        d3 T2 = cross(Vh, T1);
        double rr = sqrt(u1), ph = 2.0 * OR_PI * u2;
        double t1 = rr * cos(ph), t2 = rr * sin(ph);
        double s = 0.5 * (1.0 + Vh.z);
        t2 = (1.0 - s) * sqrt(fmax(0.0, 1.0 - t1 * t1)) + s * t2;
        d3 Nh = add(add(scl(T1, t1), scl(T2, t2)), scl(Vh, sqrt(fmax(0.0, 1.0 - t1 * t1 - t2 * t2))));
        d3 Ne = nrm(mk(a * Nh.x, a * Nh.y, fmax(0.0, Nh.z)));
        l = sub(scl(Ne, 2.0 * dot(wl, Ne)), wl);
    }
    *wi = add(add(scl(T, l.x), scl(B, l.y)), scl(n, l.z));
    return dot(n, *wi) > 0.0;
}

/* exported for the BRDF pins */
void or_bsdf_eval(const double *n, const double *wo, const double *wi, const double *rho, double r, double ks,
                  double f0, double *f, double *dfdr)
{
    bsdf_eval(mk(n[0], n[1], n[2]), mk(wo[0], wo[1], wo[2]), mk(wi[0], wi[1], wi[2]), rho, r, ks, f0, f, dfdr);
}
double or_bsdf_pdf(const double *n, const double *wo, const double *wi, double r, double ks)
{
    return bsdf_pdf(mk(n[0], n[1], n[2]), mk(wo[0], wo[1], wo[2]), mk(wi[0], wi[1], wi[2]), r, ks);
}
int or_bsdf_sample(const double *n, const double *wo, double r, double ks, double u0, double u1, double u2,
                   double *wi)
{
    d3 w;
    int ok = bsdf_sample(mk(n[0], n[1], n[2]), mk(wo[0], wo[1], wo[2]), r, ks, u0, u1, u2, &w);
    wi[0] = w.x; wi[1] = w.y; wi[2] = w.z;
    return ok;
}

/* ------------------------------------------------------------------------- */
/* Principled BRDF with a metallic parameter m (Burley 2012):                 */
/*   f_j = (1 - m) rho_j / pi + ks S F_j,   S = D G / (4 ci co),              */
/*   F_j = F0_j + (1 - F0_j) (1 - wo.h)^5,  F0_j = (1 - m) f0 + m rho_j.      */
/* m = 0 is bsdf_eval.  With it come its partial derivatives in r (through   */
/* alpha), rho_j, m and the shading normal n (wo, wi and h held fixed):      */
/*   d ln S / dn = (d ln D / d ch) h + (d ln G1(co)/d co - 1/co) wo          */
/*               + (d ln G1(ci)/d ci - 1/ci) wi,                             */
/*   d ln D / d ch = -4 ch (a^2 - 1) / t,                                    */
/*   d ln G1(c) / dc - 1/c = -(1 + (1 - a^2) c / s) / (c + s).               */
/* ------------------------------------------------------------------------- */
typedef struct {
    double f[3], dr[3], drho[3], dm[3];
    d3 dn[3];
} pbr_f;

static void pbr_eval(d3 n, d3 wo, d3 wi, const double rho[3], double r, double m, double ks, double f0, pbr_f *o)
{
    memset(o, 0, sizeof *o);
    double ci = dot(n, wi), co = dot(n, wo);
    if (ci <= 0.0 || co <= 0.0) return;
    double S = 0.0, dSda = 0.0, s5 = 0.0, dadr = 0.0;
    d3 dSdn = mk(0.0, 0.0, 0.0);
    if (ks > 0.0) {
        double a = alpha_of(r, &dadr);
        d3 h = nrm(add(wo, wi));
        double ch = dot(n, h);
        double a2 = a * a;
        double t = ch * ch * (a2 - 1.0) + 1.0;
        double D = a2 / (OR_PI * t * t);
        double si = sqrt(a2 + (1.0 - a2) * ci * ci), so = sqrt(a2 + (1.0 - a2) * co * co);
        double G = (2.0 * ci / (ci + si)) * (2.0 * co / (co + so));
        S = D * G / (4.0 * ci * co);
        double dlnD = 2.0 / a - 4.0 * a * ch * ch / t;
        double dlnG = -(a * (1.0 - ci * ci) / si) / (ci + si) - (a * (1.0 - co * co) / so) / (co + so);
        dSda = S * (dlnD + dlnG);
        double kh = -4.0 * ch * (a2 - 1.0) / t;
        double ko = -(1.0 + (1.0 - a2) * co / so) / (co + so);
        double ki = -(1.0 + (1.0 - a2) * ci / si) / (ci + si);
        dSdn = scl(add(add(scl(h, kh), scl(wo, ko)), scl(wi, ki)), S);
        double mm = 1.0 - dot(wo, h);
        if (mm < 0.0) mm = 0.0;
        s5 = mm * mm * mm * mm * mm;
    }
    for (int j = 0; j < 3; ++j) {
        double F0 = (1.0 - m) * f0 + m * rho[j];
        double F = F0 + (1.0 - F0) * s5;
        o->f[j] = (1.0 - m) * rho[j] / OR_PI + ks * S * F;
        o->dr[j] = ks * dSda * dadr * F;
        o->drho[j] = (1.0 - m) / OR_PI + ks * S * (1.0 - s5) * m;
        o->dm[j] = -rho[j] / OR_PI + ks * S * (1.0 - s5) * (rho[j] - f0);
        o->dn[j] = scl(dSdn, ks * F);
    }
}

/* exported for the pins: f[3], dr[3], drho[3], dm[3], dn[3][3] (row j = channel) */
void or_pbr_eval(const double *n, const double *wo, const double *wi, const double *rho, double r, double m,
                 double ks, double f0, double *f, double *dr, double *drho, double *dm, double *dn)
{
    pbr_f o;
    pbr_eval(mk(n[0], n[1], n[2]), mk(wo[0], wo[1], wo[2]), mk(wi[0], wi[1], wi[2]), rho, r, m, ks, f0, &o);
    for (int j = 0; j < 3; ++j) {
        f[j] = o.f[j]; dr[j] = o.dr[j]; drho[j] = o.drho[j]; dm[j] = o.dm[j];
        dn[3 * j] = o.dn[j].x; dn[3 * j + 1] = o.dn[j].y; dn[3 * j + 2] = o.dn[j].z;
    }
}

/* Tangent of triangle (e1, e2) with corner texture coordinates tuv (u0 v0 u1
 * v1 u2 v2): dp/du from e1 = dp/du du1 + dp/dv dv1, e2 = dp/du du2 + dp/dv
 * dv2, made orthogonal to the unit normal N.  A degenerate parameterisation
 * falls back to the shading-frame tangent of onb(). */
static d3 tangent_of(d3 e1, d3 e2, const double *tuv, d3 N)
{
    double du1 = tuv[2] - tuv[0], dv1 = tuv[3] - tuv[1], du2 = tuv[4] - tuv[0], dv2 = tuv[5] - tuv[1];
    double det = du1 * dv2 - du2 * dv1;
    if (det != 0.0) {
        d3 dpdu = scl(sub(scl(e1, dv2), scl(e2, dv1)), 1.0 / det);
        d3 t = sub(dpdu, scl(N, dot(N, dpdu)));
        double l = len(t);
        if (l > 1e-12 * len(dpdu)) return scl(t, 1.0 / l);
    }
    d3 t, b;
    onb(N, &t, &b);
    return t;
}

/* ------------------------------------------------------------------------- */
/* bilinear lookup with texel centres at (i + 1/2), clamp to edge              */
/* ------------------------------------------------------------------------- */
static void bilin(double xp, double yp, int W, int H, int idx[4], double w[4])
{
    double x = xp - 0.5, y = yp - 0.5;
    if (x < -1.0) x = -1.0;
    if (x > (double)W) x = (double)W;
    if (y < -1.0) y = -1.0;
    if (y > (double)H) y = (double)H;
    double fx0 = floor(x), fy0 = floor(y);
    double fx = x - fx0, fy = y - fy0;
    int x0 = (int)fx0, y0 = (int)fy0;
    int xa = clampi(x0, 0, W - 1), xb = clampi(x0 + 1, 0, W - 1);
    int ya = clampi(y0, 0, H - 1), yb = clampi(y0 + 1, 0, H - 1);
    idx[0] = ya * W + xa; idx[1] = ya * W + xb; idx[2] = yb * W + xa; idx[3] = yb * W + xb;
    w[0] = (1.0 - fx) * (1.0 - fy); w[1] = fx * (1.0 - fy); w[2] = (1.0 - fx) * fy; w[3] = fx * fy;
}

/* ------------------------------------------------------------------------- */
/* Eq. 1 (PRF) and Eq. 5 (CRF with white balance)                             */
/* ------------------------------------------------------------------------- */
static double prf_texel(double ip, double gamma, double gain)
{
    return ip > 0.0 ? gain * pow(ip, gamma) : 0.0;
}
void or_prf(const double *Ip, int64_t n_texels, const or_params *P, double *Ep)
{
    for (int64_t t = 0; t < n_texels; ++t)
        for (int j = 0; j < 3; ++j) Ep[3 * t + j] = prf_texel(Ip[3 * t + j], P->gamma_p[j], P->gain_p);
}
static double crf(double ec, int j, const or_params *P)
{
    double a = P->gain_c * P->wb[j] * ec;
    return a > 0.0 ? pow(a, P->gamma_c[j]) : 0.0;
}

/* ------------------------------------------------------------------------- */
/* One camera path (Eq. 10 with NEE to the projector), recording what the     */
/* adjoint needs                                                              */
/* ------------------------------------------------------------------------- */
typedef struct {
    int tex_idx[4]; double tex_w[4];
    double rho[3], m;             /* albedo and metallic at the hit */
    double beta[3];
    d3 T, B, N, ns; double ulen;  /* tangent frame, shading normal ns = u / |u| (normal map) */
    int nee;                      /* NEE light arrived (inside frustum, facing, unoccluded) */
    int proj_idx[4]; double proj_w[4];
    double Ep[3], G;
    pbr_f fp;                     /* f(wo, wp) and its partial derivatives */
    d3 wp_cs;                     /* wp / cos_s */
    int unclipped[3];
    int cont;                     /* a continuation ray was traced from here */
    double cw;                    /* cos_i / (pdf q) */
    pbr_f fi;                     /* f(wo, wi) and its partial derivatives */
    d3 wi_ci;                     /* wi / cos_i */
    d3 x, wo;                     /* the vertex and the direction back along the incoming ray */
    double r;                     /* roughness at the vertex */
    d3 wp, wi;                    /* towards the projector (when nee) and the continuation (when cont) */
    double c[3];                  /* this vertex's contribution to L (after clipping) */
} vrec;

typedef struct {
    const dscene *S;
    const double *albedo, *rough; int Ht, Wt;
    const double *metal, *nmap;   /* Ht x Wt and Ht x Wt x 3, or NULL */
    const double *Ep; int Hp, Wp;
    double Kc[9], Kc_inv[9], Kp[9], Rp[9], tp[3], cp[3];
    const or_params *P;
    int spp, bounces;
    uint64_t seed;
    int Wc;
} rctx;

/* The path that starts with the ray (o, d); continuation b draws its random
 * numbers from counter (pix, s, b, 0).  Returns the number of vertices, the
 * path radiance L (RGB) and the vertex records. */
static int trace_ray(const rctx *C, d3 o, d3 d, uint32_t pix, uint32_t s, double L[3], vrec *rec)
{
    const or_params *P = C->P;
    double u[4];
    L[0] = L[1] = L[2] = 0.0;
    double beta[3] = {1.0, 1.0, 1.0};
    d3 cp = mk(C->cp[0], C->cp[1], C->cp[2]);
    int nv = 0;
    for (int b = 1; b <= C->bounces; ++b) {
        double t, bu, bv;
        int tri = closest(C->S, o, d, INFINITY, &t, &bu, &bv);
        if (tri < 0) break;
        vrec *R = &rec[nv++];
        memset(R, 0, sizeof *R);
        const dscene *S = C->S;
        d3 x = add(add(S->v0[tri], scl(S->e1[tri], bu)), scl(S->e2[tri], bv));
        d3 n = nrm(cross(S->e1[tri], S->e2[tri]));
        if (dot(n, d) > 0.0) n = scl(n, -1.0);
        const double *tuv = S->uv + 6 * tri;
        double w0 = 1.0 - bu - bv;
        double su = w0 * tuv[0] + bu * tuv[2] + bv * tuv[4];
        double sv = w0 * tuv[1] + bu * tuv[3] + bv * tuv[5];
        bilin(su * C->Wt, sv * C->Ht, C->Wt, C->Ht, R->tex_idx, R->tex_w);
        double r = 0.0;
        for (int j = 0; j < 3; ++j) R->rho[j] = 0.0;
        for (int k = 0; k < 4; ++k) {
            for (int j = 0; j < 3; ++j) R->rho[j] += R->tex_w[k] * C->albedo[3 * R->tex_idx[k] + j];
            r += R->tex_w[k] * C->rough[R->tex_idx[k]];
        }
        R->m = 0.0;
        if (C->metal)
            for (int k = 0; k < 4; ++k) R->m += R->tex_w[k] * C->metal[R->tex_idx[k]];
        /* shading normal: the normal map in the triangle's tangent frame */
        d3 ns = n;
        R->N = n;
        R->ulen = 0.0;
        if (C->nmap) {
            double vn[3] = {0.0, 0.0, 0.0};
            for (int k = 0; k < 4; ++k)
                for (int j = 0; j < 3; ++j) vn[j] += R->tex_w[k] * C->nmap[3 * R->tex_idx[k] + j];
            R->T = tangent_of(S->e1[tri], S->e2[tri], tuv, n);
            R->B = cross(n, R->T);
            d3 u = add(add(scl(R->T, 2.0 * vn[0] - 1.0), scl(R->B, 2.0 * vn[1] - 1.0)), scl(n, 2.0 * vn[2] - 1.0));
            R->ulen = len(u);
            if (R->ulen > 1e-12) ns = scl(u, 1.0 / R->ulen);
        }
        R->ns = ns;
        for (int j = 0; j < 3; ++j) R->beta[j] = beta[j];
        d3 wo = scl(d, -1.0);
        R->x = x;
        R->wo = wo;
        R->r = r;

        /* next-event estimation to the pinhole projector (Eqs. 1, 2, 3, 6) */
        d3 X = add(mat3v(C->Rp, x), mk(C->tp[0], C->tp[1], C->tp[2]));
        d3 q = mat3v(C->Kp, X);
        if (q.z > 0.0 && X.z > 0.0) {
            double up = q.x / q.z, vp = q.y / q.z;
            if (up >= 0.0 && up < (double)C->Wp && vp >= 0.0 && vp < (double)C->Hp) {
                d3 v = sub(cp, x);
                double r2 = dot(v, v), dist = sqrt(r2);
                d3 wp = scl(v, 1.0 / dist);
                double cs = dot(ns, wp);
                if (cs > 0.0 && dot(n, wp) > 0.0) {
                    double cpz = X.z / len(X);
                    d3 so = add(x, scl(n, OR_RAY_EPS));
                    d3 sv = sub(cp, so);
                    double sd = len(sv);
                    if (!occluded(S, so, scl(sv, 1.0 / sd), sd - OR_RAY_EPS)) {
                        R->nee = 1;
                        bilin(up, vp, C->Wp, C->Hp, R->proj_idx, R->proj_w);
                        for (int j = 0; j < 3; ++j) {
                            R->Ep[j] = 0.0;
                            for (int k = 0; k < 4; ++k) R->Ep[j] += R->proj_w[k] * C->Ep[3 * R->proj_idx[k] + j];
                        }
                        R->G = P->k_proj * cpz * cs / r2;
                        pbr_eval(ns, wo, wp, R->rho, r, R->m, P->ks, P->f0, &R->fp);
                        R->wp_cs = scl(wp, 1.0 / cs);
                        R->wp = wp;
                        for (int j = 0; j < 3; ++j) {
                            double c = beta[j] * R->fp.f[j] * R->Ep[j] * R->G;
                            R->unclipped[j] = 1;
                            if (P->clip > 0.0 && c > P->clip) { c = P->clip; R->unclipped[j] = 0; }
                            R->c[j] = c;
                            L[j] += c;
                        }
                    }
                }
            }
        }
        if (b == C->bounces) break;

        /* continuation: BSDF sampling, throughput, Russian roulette */
        rand4(C->seed, pix, s, (uint32_t)b, u);
        d3 wi;
        if (!bsdf_sample(ns, wo, r, P->ks, u[0], u[1], u[2], &wi)) break;
        if (!(dot(n, wi) > 0.0)) break; /* below the geometric surface */
        double pdf = bsdf_pdf(ns, wo, wi, r, P->ks);
        if (!(pdf > 0.0)) break;
        double qrr = 1.0;
        if (P->rr_start > 0 && b >= P->rr_start) {
            if (u[3] >= P->rr_q) break;
            qrr = P->rr_q;
        }
        pbr_eval(ns, wo, wi, R->rho, r, R->m, P->ks, P->f0, &R->fi);
        R->cont = 1;
        double ci = dot(ns, wi);
        R->cw = ci / (pdf * qrr);
        R->wi_ci = scl(wi, 1.0 / ci);
        R->wi = wi;
        for (int j = 0; j < 3; ++j) beta[j] *= R->fi.f[j] * R->cw;
        o = add(x, scl(n, OR_RAY_EPS));
        d = wi;
    }
    return nv;
}

/* camera sample s of pixel pix: the jittered ray of Eq. 6 with the Eq. 4 box
 * filter, then trace_ray */
static int trace_sample(const rctx *C, uint32_t pix, uint32_t s, double L[3], vrec *rec)
{
    double u[4];
    rand4(C->seed, pix, s, 0u, u);
    double fx = (double)(pix % (uint32_t)C->Wc) + (C->P->jitter ? u[0] : 0.5);
    double fy = (double)(pix / (uint32_t)C->Wc) + (C->P->jitter ? u[1] : 0.5);
    return trace_ray(C, mk(0.0, 0.0, 0.0), nrm(mat3v(C->Kc_inv, mk(fx, fy, 1.0))), pix, s, L, rec);
}

static void rctx_make(rctx *C, const dscene *S, const double *albedo, const double *rough, int Ht, int Wt,
                      const double *Ep, const or_view *Vw, const or_params *P, int spp, int bounces, uint64_t seed)
{
    C->S = S; C->albedo = albedo; C->rough = rough; C->Ht = Ht; C->Wt = Wt;
    C->metal = NULL; C->nmap = NULL;
    C->Ep = Ep; C->Hp = Vw->Hp; C->Wp = Vw->Wp;
    memcpy(C->Kc, Vw->Kc, sizeof C->Kc);
    inv3(Vw->Kc, C->Kc_inv);
    memcpy(C->Kp, Vw->Kp, sizeof C->Kp);
    memcpy(C->Rp, Vw->Rp, sizeof C->Rp);
    memcpy(C->tp, Vw->tp, sizeof C->tp);
    /* projector centre cp = -Rp^T tp */
    for (int i = 0; i < 3; ++i)
        C->cp[i] = -(Vw->Rp[0 * 3 + i] * Vw->tp[0] + Vw->Rp[1 * 3 + i] * Vw->tp[1] + Vw->Rp[2 * 3 + i] * Vw->tp[2]);
    C->P = P; C->spp = spp; C->bounces = bounces; C->seed = seed; C->Wc = Vw->Wc;
}

static int set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

int or_num_threads(int nthreads) { return set_threads(nthreads); }

/*
 * Forward render of the listed pixels (pixel index = y * Wc + x); NULL list =
 * every pixel.  Ec and Ic are npix x 3.  metal (Ht x Wt) and nmap (Ht x Wt x
 * 3) are the principled material's metallic and normal maps; NULL = metallic
 * 0 and no normal map.  Returns 0, or -1 on bad arguments.
 */
int or_render_m(const float *verts, const int32_t *tris, int32_t T, const float *uv, const double *albedo,
                const double *rough, const double *metal, const double *nmap, int32_t Ht, int32_t Wt,
                const double *Ip, const or_view *Vw, const or_params *P, int32_t spp, int32_t bounces, uint64_t seed,
                const int64_t *pixels, int64_t npix, double *Ec, double *Ic, int32_t nthreads)
{
    if (spp <= 0 || bounces < 0 || bounces > OR_MAX_VERTS || Ht <= 0 || Wt <= 0 || Vw->Hp <= 0 || Vw->Wp <= 0)
        return -1;
    set_threads(nthreads);
    dscene S;
    scene_make(&S, verts, tris, T, uv);
    int64_t ntex = (int64_t)Vw->Hp * Vw->Wp;
    double *Ep = (double *)malloc(sizeof(double) * 3 * (size_t)ntex);
    or_prf(Ip, ntex, P, Ep);
    rctx C;
    rctx_make(&C, &S, albedo, rough, Ht, Wt, Ep, Vw, P, spp, bounces, seed);
    C.metal = metal;
    C.nmap = nmap;
    int64_t n = pixels ? npix : (int64_t)Vw->Hc * Vw->Wc;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; ++i) {
        uint32_t pix = (uint32_t)(pixels ? pixels[i] : i);
        vrec rec[OR_MAX_VERTS];
        double sum[3] = {0.0, 0.0, 0.0}, L[3];
        for (int s = 0; s < spp; ++s) {
            trace_sample(&C, pix, (uint32_t)s, L, rec);
            for (int j = 0; j < 3; ++j) sum[j] += L[j];
        }
        for (int j = 0; j < 3; ++j) {
            Ec[3 * i + j] = sum[j] / spp;
            Ic[3 * i + j] = crf(Ec[3 * i + j], j, P);
        }
    }
    free(Ep);
    scene_free(&S);
    return 0;
}

int or_render(const float *verts, const int32_t *tris, int32_t T, const float *uv, const double *albedo,
              const double *rough, int32_t Ht, int32_t Wt, const double *Ip, const or_view *Vw, const or_params *P,
              int32_t spp, int32_t bounces, uint64_t seed, const int64_t *pixels, int64_t npix, double *Ec, double *Ic,
              int32_t nthreads)
{
    return or_render_m(verts, tris, T, uv, albedo, rough, NULL, NULL, Ht, Wt, Ip, Vw, P, spp, bounces, seed, pixels,
                       npix, Ec, Ic, nthreads);
}

/*
 * Adjoint of or_render_m for the listed pixels: given dLoss/dIc (npix x 3),
 * accumulates (+=) dLoss/dIp [Hp*Wp*3], dLoss/dalbedo [Ht*Wt*3],
 * dLoss/drough [Ht*Wt], dLoss/dmetal [Ht*Wt] and dLoss/dnmap [Ht*Wt*3]
 * (each only where its map was given) and dParams [gamma_p(3), Gp,
 * gamma_c(3), Gc, wb(3)].  The forward is recomputed here; sampled
 * directions are held fixed.
 */
int or_render_backward_m(const float *verts, const int32_t *tris, int32_t T, const float *uv, const double *albedo,
                         const double *rough, const double *metal, const double *nmap, int32_t Ht, int32_t Wt,
                         const double *Ip, const or_view *Vw, const or_params *P, int32_t spp, int32_t bounces,
                         uint64_t seed, const int64_t *pixels, int64_t npix, const double *dIc, double *dIp,
                         double *dAlbedo, double *dRough, double *dMetal, double *dNmap, double *dParams,
                         int32_t nthreads)
{
    if (spp <= 0 || bounces < 0 || bounces > OR_MAX_VERTS || Ht <= 0 || Wt <= 0 || Vw->Hp <= 0 || Vw->Wp <= 0)
        return -1;
    int nt = set_threads(nthreads);
    dscene S;
    scene_make(&S, verts, tris, T, uv);
    int64_t ntex = (int64_t)Vw->Hp * Vw->Wp, nalb = (int64_t)Ht * Wt;
    double *Ep = (double *)malloc(sizeof(double) * 3 * (size_t)ntex);
    or_prf(Ip, ntex, P, Ep);
    rctx C;
    rctx_make(&C, &S, albedo, rough, Ht, Wt, Ep, Vw, P, spp, bounces, seed);
    C.metal = metal;
    C.nmap = nmap;
    int64_t n = pixels ? npix : (int64_t)Vw->Hc * Vw->Wc;
    /* per-thread gradient buffers (Ep, albedo, roughness, metallic, normal
     * map), summed in thread order afterwards */
    size_t per = (size_t)(3 * ntex + 3 * nalb + nalb + nalb + 3 * nalb);
    double *acc = (double *)calloc((size_t)nt * per, sizeof(double));
    double crf_acc[8] = {0};
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *gEp = acc + (size_t)tid * per, *gA = gEp + 3 * ntex, *gR = gA + 3 * nalb, *gM = gR + nalb,
               *gN = gM + nalb;
#pragma omp for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            uint32_t pix = (uint32_t)(pixels ? pixels[i] : i);
            vrec rec[OR_MAX_VERTS];
            double sum[3] = {0.0, 0.0, 0.0}, L[3];
            for (int s = 0; s < spp; ++s) {
                trace_sample(&C, pix, (uint32_t)s, L, rec);
                for (int j = 0; j < 3; ++j) sum[j] += L[j];
            }
            /* Eq. 5 adjoint: dL/dEc and the CRF / white-balance parameters */
            double gE[3];
            for (int j = 0; j < 3; ++j) {
                double ec = sum[j] / spp;
                double a = P->gain_c * P->wb[j] * ec;
                gE[j] = 0.0;
                if (a > 0.0) {
                    double g = dIc[3 * i + j];
                    double da = P->gamma_c[j] * pow(a, P->gamma_c[j] - 1.0); /* dIc/da */
                    gE[j] = g * da * P->gain_c * P->wb[j];
#pragma omp atomic
                    crf_acc[j] += g * pow(a, P->gamma_c[j]) * log(a);            /* gamma_c */
#pragma omp atomic
                    crf_acc[3] += g * da * P->wb[j] * ec;                        /* Gc */
#pragma omp atomic
                    crf_acc[4 + j] += g * da * P->gain_c * ec;                   /* wb */
                }
            }
            /* Eq. 4 adjoint (mean over samples), then the path adjoint */
            double gbar[3] = {gE[0] / spp, gE[1] / spp, gE[2] / spp};
            if (gbar[0] == 0.0 && gbar[1] == 0.0 && gbar[2] == 0.0) continue;
            for (int s = 0; s < spp; ++s) {
                int nv = trace_sample(&C, pix, (uint32_t)s, L, rec);
                /* reverse sweep; A = dL/dbeta_{c+1} in units of beta_{c+1} */
                double A[3] = {0.0, 0.0, 0.0};
                for (int c = nv - 1; c >= 0; --c) {
                    const vrec *R = &rec[c];
                    double An[3] = {A[0], A[1], A[2]};
                    double dr = 0.0, dm = 0.0;
                    d3 gn = mk(0.0, 0.0, 0.0); /* dL / d(shading normal) */
                    for (int j = 0; j < 3; ++j) {
                        double gb = gbar[j] * R->beta[j];
                        double ln_e = (R->nee && R->unclipped[j]) ? R->Ep[j] * R->G : 0.0; /* Ln / f */
                        double cont = R->cont ? R->cw * An[j] : 0.0;                       /* w / f * A */
                        if (R->nee && R->unclipped[j])
                            for (int k = 0; k < 4; ++k)
                                gEp[3 * R->proj_idx[k] + j] +=
                                    gb * R->fp.f[j] * R->G * (g_unit_taps ? 1.0 : R->proj_w[k]);
                        double ga = gb * (R->fp.drho[j] * ln_e + R->fi.drho[j] * cont);
                        for (int k = 0; k < 4; ++k) gA[3 * R->tex_idx[k] + j] += ga * (g_unit_taps ? 1.0 : R->tex_w[k]);
                        dr += gb * (R->fp.dr[j] * ln_e + R->fi.dr[j] * cont);
                        dm += gb * (R->fp.dm[j] * ln_e + R->fi.dm[j] * cont);
                        /* the normal enters f and cos_s (NEE), f and cos_i (continuation) */
                        if (ln_e != 0.0)
                            gn = add(gn, scl(add(R->fp.dn[j], scl(R->wp_cs, R->fp.f[j])), gb * ln_e));
                        if (cont != 0.0)
                            gn = add(gn, scl(add(R->fi.dn[j], scl(R->wi_ci, R->fi.f[j])), gb * cont));
                        A[j] = R->fp.f[j] * ln_e + R->fi.f[j] * cont;
                    }
                    for (int k = 0; k < 4; ++k) gR[R->tex_idx[k]] += dr * R->tex_w[k];
                    if (metal)
                        for (int k = 0; k < 4; ++k) gM[R->tex_idx[k]] += dm * R->tex_w[k];
                    if (nmap && R->ulen > 1e-12) {
                        /* ns = u / |u|, u = T v0 + B v1 + N v2, v = 2 Vn - 1 */
                        d3 gu = scl(sub(gn, scl(R->ns, dot(R->ns, gn))), 1.0 / R->ulen);
                        double gv[3] = {2.0 * dot(R->T, gu), 2.0 * dot(R->B, gu), 2.0 * dot(R->N, gu)};
                        for (int k = 0; k < 4; ++k)
                            for (int j = 0; j < 3; ++j) gN[3 * R->tex_idx[k] + j] += gv[j] * R->tex_w[k];
                    }
                }
            }
        }
    }
    /* Eq. 1 adjoint: dIp, gamma_p, Gp */
    double prf_acc[4] = {0};
    for (int64_t t = 0; t < ntex; ++t)
        for (int j = 0; j < 3; ++j) {
            double g = 0.0;
            for (int th = 0; th < nt; ++th) g += acc[(size_t)th * per + 3 * t + j];
            double ip = Ip[3 * t + j];
            if (ip > 0.0 && g != 0.0) {
                double gm = P->gamma_p[j];
                dIp[3 * t + j] += g * P->gain_p * gm * pow(ip, gm - 1.0);
                prf_acc[j] += g * P->gain_p * pow(ip, gm) * log(ip);
                prf_acc[3] += g * pow(ip, gm);
            }
        }
    for (int64_t t = 0; t < 3 * nalb; ++t) {
        double g = 0.0;
        for (int th = 0; th < nt; ++th) g += acc[(size_t)th * per + 3 * ntex + t];
        dAlbedo[t] += g;
    }
    for (int64_t t = 0; t < nalb; ++t) {
        double g = 0.0;
        for (int th = 0; th < nt; ++th) g += acc[(size_t)th * per + 3 * ntex + 3 * nalb + t];
        dRough[t] += g;
    }
    if (metal && dMetal)
        for (int64_t t = 0; t < nalb; ++t) {
            double g = 0.0;
            for (int th = 0; th < nt; ++th) g += acc[(size_t)th * per + 3 * ntex + 4 * nalb + t];
            dMetal[t] += g;
        }
    if (nmap && dNmap)
        for (int64_t t = 0; t < 3 * nalb; ++t) {
            double g = 0.0;
            for (int th = 0; th < nt; ++th) g += acc[(size_t)th * per + 3 * ntex + 5 * nalb + t];
            dNmap[t] += g;
        }
    dParams[0] += prf_acc[0]; dParams[1] += prf_acc[1]; dParams[2] += prf_acc[2]; dParams[3] += prf_acc[3];
    dParams[4] += crf_acc[0]; dParams[5] += crf_acc[1]; dParams[6] += crf_acc[2]; dParams[7] += crf_acc[3];
    dParams[8] += crf_acc[4]; dParams[9] += crf_acc[5]; dParams[10] += crf_acc[6];
    free(acc);
    free(Ep);
    scene_free(&S);
    return 0;
}

int or_render_backward(const float *verts, const int32_t *tris, int32_t T, const float *uv, const double *albedo,
                       const double *rough, int32_t Ht, int32_t Wt, const double *Ip, const or_view *Vw,
                       const or_params *P, int32_t spp, int32_t bounces, uint64_t seed, const int64_t *pixels,
                       int64_t npix, const double *dIc, double *dIp, double *dAlbedo, double *dRough, double *dParams,
                       int32_t nthreads)
{
    return or_render_backward_m(verts, tris, T, uv, albedo, rough, NULL, NULL, Ht, Wt, Ip, Vw, P, spp, bounces, seed,
                                pixels, npix, dIc, dIp, dAlbedo, dRough, NULL, NULL, dParams, nthreads);
}

/* ------------------------------------------------------------------------- */
/* Guide features of the cross-bilateral denoiser of Eq. 11: what the camera */
/* ray through each pixel centre sees first.  Per pixel 8 values: bilinear   */
/* albedo (3), geometric normal turned towards the camera (3), hit distance  */
/* along the unit ray, and 1 for a hit; all 8 are 0 where the ray misses.    */
/* The paper names the filter but not its guide; these are the noise-free    */
/* first-hit quantities of the renderer itself.                              */
/* ------------------------------------------------------------------------- */
int or_gbuffer(const float *verts, const int32_t *tris, int32_t T, const float *uv, const double *albedo,
               int32_t Ht, int32_t Wt, const or_view *Vw, double *guide, int32_t nthreads)
{
    if (Ht <= 0 || Wt <= 0 || Vw->Hc <= 0 || Vw->Wc <= 0) return -1;
    set_threads(nthreads);
    dscene S;
    scene_make(&S, verts, tris, T, uv);
    double Kc_inv[9];
    inv3(Vw->Kc, Kc_inv);
    const int64_t n = (int64_t)Vw->Hc * Vw->Wc;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < n; ++p) {
        double *g = guide + 8 * p;
        for (int k = 0; k < 8; ++k) g[k] = 0.0;
        double fx = (double)(p % Vw->Wc) + 0.5, fy = (double)(p / Vw->Wc) + 0.5;
        d3 d = nrm(mat3v(Kc_inv, mk(fx, fy, 1.0)));
        double t, bu, bv;
        int tri = closest(&S, mk(0.0, 0.0, 0.0), d, INFINITY, &t, &bu, &bv);
        if (tri < 0) continue;
        d3 nn = nrm(cross(S.e1[tri], S.e2[tri]));
        if (dot(nn, d) > 0.0) nn = scl(nn, -1.0);
        const double *tuv = S.uv + 6 * tri;
        double w0 = 1.0 - bu - bv;
        double su = w0 * tuv[0] + bu * tuv[2] + bv * tuv[4];
        double sv = w0 * tuv[1] + bu * tuv[3] + bv * tuv[5];
        int idx[4];
        double w[4];
        bilin(su * Wt, sv * Ht, Wt, Ht, idx, w);
        for (int k = 0; k < 4; ++k)
            for (int j = 0; j < 3; ++j) g[j] += w[k] * albedo[3 * idx[k] + j];
        g[3] = nn.x; g[4] = nn.y; g[5] = nn.z;
        g[6] = t;
        g[7] = 1.0;
    }
    scene_free(&S);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Camera-pose gradient.  Sec. 3.2 counts the camera pose (Rc, tc) among the  */
/* scene parameters theta of Eq. 9.                                           */
/* ------------------------------------------------------------------------- */
/*
 * Renders keep the camera at the origin, so a pose parameter moves the whole
 * scene (mesh and projector) rigidly in the camera frame: a point y moves
 * with velocity a x y + b (a "twist" (a, b) per parameter).  The pixel mean
 * of Eq. 4 is I_P = integral over pixel P's unit square of the radiance
 * L(u) that reaches image point u.  Written as an integral over the visible
 * surface, the integrand L(x) J(x) (J = image area per unit surface area)
 * travels with the surface, and so do the shadow edges and the projector
 * frustum's border on it: relative to the scene only the camera moves.
 * Differentiating each visible region's integral as its boundary moves
 * (Reynolds transport) leaves three terms, g_P = dLoss/dEc_P:
 *   interior    sum over camera samples of d/dtheta of the sample's
 *               contribution with its first hit held on the surface and the
 *               sampled directions held fixed: the BRDF at the first vertex
 *               through its direction wo to the camera, plus the whole
 *               contribution times d log J / dtheta (divided by spp);
 *   pixel edges for every pixel P, -g_P times the flux out of its square,
 *               the integral over its four edges of L (V.n), n the outward
 *               normal and V the image velocity of the surface point seen
 *               there (the same sum, edge by edge, as L (V.n) (g_Q - g_P)
 *               over the edges between pixels P and Q, g = 0 outside the
 *               image, but estimated pixel by pixel: the four edges' paths
 *               share their random numbers, so opposite edges give a
 *               common-random-number difference across the pixel);
 *   silhouettes where a nearer surface F hides a farther one B, B's visible
 *               part ends at F's edge, which moves with F: integral over the
 *               silhouette of g_P L_B (V_F - V_B).n_BF.
 * Every derivative of a smooth quantity here (the BRDF along wo, log J, the
 * image velocity, the silhouette's image speed) is taken by central
 * differences in FP64; only the split into the three terms is analytic.
 */
static void pose_proj(const double *Kc, d3 y, double s[2])
{
    d3 q = mat3v(Kc, y);
    s[0] = q.x / q.z;
    s[1] = q.y / q.z;
}

static d3 pose_vel(const double *tw, d3 y) { return add(cross(mk(tw[0], tw[1], tw[2]), y), mk(tw[3], tw[4], tw[5])); }

/* image velocity of the scene point y under twist tw */
static void pose_img_vel(const double *Kc, const double *tw, d3 y, double V[2])
{
    const double h = 1e-5;
    double sp[2], sm[2];
    d3 v = pose_vel(tw, y);
    pose_proj(Kc, add(y, scl(v, h)), sp);
    pose_proj(Kc, sub(y, scl(v, h)), sm);
    V[0] = (sp[0] - sm[0]) / (2.0 * h);
    V[1] = (sp[1] - sm[1]) / (2.0 * h);
}

/* log of the image area per unit surface area at x (normal n), the scene
 * moved by th along twist tw: the square of half-side e around x in the
 * surface's plane maps to a quadrilateral (lines stay lines), whose area
 * over the square's is J averaged over the square, J(x) + O(e^2) */
static double pose_logJ(const double *Kc, const double *tw, d3 x, d3 n, double th)
{
    d3 t1, t2;
    onb(n, &t1, &t2);
    const double e = 1e-3 * len(x);
    const double sg[4][2] = {{1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
    d3 c[4];
    double s[4][2], s0[2];
    for (int i = 0; i < 4; ++i) {
        d3 p = add(x, add(scl(t1, e * sg[i][0]), scl(t2, e * sg[i][1])));
        c[i] = add(p, scl(pose_vel(tw, p), th));
    }
    d3 xc = add(x, scl(pose_vel(tw, x), th));
    pose_proj(Kc, xc, s0);
    for (int i = 0; i < 4; ++i) {
        pose_proj(Kc, c[i], s[i]);
        s[i][0] -= s0[0];
        s[i][1] -= s0[1];
    }
    double img = 0.0;
    for (int i = 0; i < 4; ++i) img += s[i][0] * s[(i + 1) % 4][1] - s[(i + 1) % 4][0] * s[i][1];
    img = 0.5 * fabs(img);
    double surf = 0.5 * len(cross(sub(c[0], c[2]), sub(c[1], c[3])));
    return log(img / surf);
}

static double pose_dlogJ(const double *Kc, const double *tw, d3 x, d3 n)
{
    const double h = 1e-5;
    return (pose_logJ(Kc, tw, x, n, h) - pose_logJ(Kc, tw, x, n, -h)) / (2.0 * h);
}

/* directional derivative of the BRDF value f(wo, w) along dwo (tangent to wo) */
static void pose_df(const vrec *R, d3 wo, d3 dwo, d3 w, const or_params *P, double df[3])
{
    const double h = 1e-6;
    pbr_f fp, fm;
    pbr_eval(R->ns, nrm(add(wo, scl(dwo, h))), w, R->rho, R->r, R->m, P->ks, P->f0, &fp);
    pbr_eval(R->ns, nrm(sub(wo, scl(dwo, h))), w, R->rho, R->r, R->m, P->ks, P->f0, &fm);
    for (int j = 0; j < 3; ++j) df[j] = (fp.f[j] - fm.f[j]) / (2.0 * h);
}

/* interior term of one path for twist tw, g = dLoss/dEc of its pixel / spp */
static double pose_interior(const rctx *C, const vrec *rec, int nv, const double *tw, const double g[3])
{
    const vrec *R = &rec[0];
    double rest[3] = {0, 0, 0}, restU[3] = {0, 0, 0};
    for (int v = 1; v < nv; ++v)
        for (int j = 0; j < 3; ++j) {
            rest[j] += rec[v].c[j];
            if (rec[v].unclipped[j]) restU[j] += rec[v].c[j];
        }
    d3 x = R->x, wo = R->wo, b = mk(tw[3], tw[4], tw[5]);
    /* relative to the scene the camera centre moves by -b: wo turns by
     * -(b - wo (wo.b)) / |x| */
    d3 dwo = scl(sub(b, scl(wo, dot(wo, b))), -1.0 / len(x));
    double term = 0.0, df[3];
    if (R->nee) {
        pose_df(R, wo, dwo, R->wp, C->P, df);
        for (int j = 0; j < 3; ++j)
            if (R->unclipped[j]) term += g[j] * df[j] * R->Ep[j] * R->G; /* throughput 1 at the first vertex */
    }
    if (R->cont) {
        pose_df(R, wo, dwo, R->wi, C->P, df);
        for (int j = 0; j < 3; ++j)
            if (R->fi.f[j] > 0.0) term += g[j] * restU[j] * df[j] / R->fi.f[j];
    }
    const double dlj = pose_dlogJ(C->Kc, tw, x, R->N);
    for (int j = 0; j < 3; ++j) term += g[j] * (R->c[j] + rest[j]) * dlj;
    return term;
}

typedef struct { int32_t v0, v1, third[2], nthird; } pose_edge;

static int pose_edge_cmp(const void *pa, const void *pb)
{
    const int32_t *a = (const int32_t *)pa, *b = (const int32_t *)pb;
    for (int k = 0; k < 3; ++k)
        if (a[k] != b[k]) return a[k] < b[k] ? -1 : 1;
    return 0;
}

/* the mesh's edges in increasing (lower vertex, higher vertex) order, each
 * with the third vertices of its triangles (nthird > 2: non-manifold) */
static int64_t pose_edges(const int32_t *tris, int32_t T, pose_edge **out)
{
    int32_t *h = (int32_t *)malloc(sizeof(int32_t) * 9 * (size_t)(T > 0 ? T : 1));
    for (int32_t i = 0; i < T; ++i)
        for (int k = 0; k < 3; ++k) {
            int32_t a = tris[3 * i + k], b = tris[3 * i + (k + 1) % 3], c = tris[3 * i + (k + 2) % 3];
            int32_t *r = h + 3 * (3 * (int64_t)i + k);
            r[0] = a < b ? a : b;
            r[1] = a < b ? b : a;
            r[2] = c;
        }
    qsort(h, (size_t)3 * T, 3 * sizeof(int32_t), pose_edge_cmp);
    pose_edge *E = (pose_edge *)malloc(sizeof(pose_edge) * 3 * (size_t)(T > 0 ? T : 1));
    int64_t n = 0;
    for (int64_t i = 0; i < 3 * (int64_t)T; ++i) {
        const int32_t *r = h + 3 * i;
        if (n == 0 || E[n - 1].v0 != r[0] || E[n - 1].v1 != r[1]) {
            E[n].v0 = r[0]; E[n].v1 = r[1]; E[n].nthird = 0;
            ++n;
        }
        pose_edge *e = &E[n - 1];
        if (e->nthird < 2) e->third[e->nthird] = r[2];
        e->nthird++;
    }
    free(h);
    *out = E;
    return n;
}

static d3 vert_at(const float *verts, int32_t i) { return mk(verts[3 * i], verts[3 * i + 1], verts[3 * i + 2]); }

/*
 * Gradient of a loss with dLoss/dEc = dEc (Hc x Wc x 3) with respect to n_tw
 * pose parameters, each given as the twist tw[6k..6k+5] = (a, b) of the
 * scene's motion in the camera frame.  out (3 x n_tw) receives the interior,
 * pixel-edge and silhouette terms; their sum is the gradient.  Random
 * numbers: camera samples as the render; pixel-edge sample j of pixel p
 * (x0, y0) uses counter (Hc Wc + p, j, vertex, 0) for all four of its paths,
 * which start at (x0 + 1, y0 + t), (x0, y0 + t), (x0 + t, y0 + 1) and
 * (x0 + t, y0), t = (j + u0) / edge_spp; silhouette sample j of mesh edge k
 * (pose_edges order) uses (2 Hc Wc + k, j, vertex, 0) and sits at
 * (j + u0) / sil_spp from the lower-numbered vertex.  Non-manifold edges are
 * skipped.
 * Returns 0, or -1 on bad arguments.
 */
int or_pose_backward_m(const float *verts, const int32_t *tris, int32_t T, const float *uv, const double *albedo,
                       const double *rough, const double *metal, const double *nmap, int32_t Ht, int32_t Wt,
                       const double *Ip, const or_view *Vw, const or_params *P, int32_t spp, int32_t bounces,
                       uint64_t seed, const double *dEc, int32_t n_tw, const double *tw, int32_t edge_spp,
                       int32_t sil_spp, double *out, int32_t nthreads);

int or_pose_backward(const float *verts, const int32_t *tris, int32_t T, const float *uv, const double *albedo,
                     const double *rough, int32_t Ht, int32_t Wt, const double *Ip, const or_view *Vw,
                     const or_params *P, int32_t spp, int32_t bounces, uint64_t seed, const double *dEc, int32_t n_tw,
                     const double *tw, int32_t edge_spp, int32_t sil_spp, double *out, int32_t nthreads)
{
    return or_pose_backward_m(verts, tris, T, uv, albedo, rough, NULL, NULL, Ht, Wt, Ip, Vw, P, spp, bounces, seed,
                              dEc, n_tw, tw, edge_spp, sil_spp, out, nthreads);
}

/* the same with the principled material's metallic (Ht x Wt) and normal
 * (Ht x Wt x 3) maps, each optional (NULL): the first vertex's BRDF is the
 * principled one at its shading normal, which the pose moves with the
 * surface */
int or_pose_backward_m(const float *verts, const int32_t *tris, int32_t T, const float *uv, const double *albedo,
                       const double *rough, const double *metal, const double *nmap, int32_t Ht, int32_t Wt,
                       const double *Ip, const or_view *Vw, const or_params *P, int32_t spp, int32_t bounces,
                       uint64_t seed, const double *dEc, int32_t n_tw, const double *tw, int32_t edge_spp,
                       int32_t sil_spp, double *out, int32_t nthreads)
{
    if (spp <= 0 || bounces < 1 || bounces > OR_MAX_VERTS || Ht <= 0 || Wt <= 0 || Vw->Hp <= 0 || Vw->Wp <= 0 ||
        n_tw < 1 || n_tw > 16 || edge_spp < 0 || sil_spp < 0)
        return -1;
    set_threads(nthreads);
    dscene S;
    scene_make(&S, verts, tris, T, uv);
    int64_t ntex = (int64_t)Vw->Hp * Vw->Wp;
    double *Ep = (double *)malloc(sizeof(double) * 3 * (size_t)ntex);
    or_prf(Ip, ntex, P, Ep);
    rctx C;
    rctx_make(&C, &S, albedo, rough, Ht, Wt, Ep, Vw, P, spp, bounces, seed);
    C.metal = metal;
    C.nmap = nmap;
    const int32_t Hc = Vw->Hc, Wc = Vw->Wc;
    const int64_t npix = (int64_t)Hc * Wc;
    double acc[3][16];
    memset(acc, 0, sizeof acc);

    /* interior */
#pragma omp parallel
    {
        double loc[16] = {0};
        vrec rec[OR_MAX_VERTS];
#pragma omp for schedule(dynamic, 4)
        for (int64_t p = 0; p < npix; ++p) {
            double g[3];
            for (int j = 0; j < 3; ++j) g[j] = dEc[3 * p + j] / spp;
            if (g[0] == 0.0 && g[1] == 0.0 && g[2] == 0.0) continue;
            for (int s = 0; s < spp; ++s) {
                double L[3];
                int nv = trace_sample(&C, (uint32_t)p, (uint32_t)s, L, rec);
                if (nv == 0) continue;
                for (int k = 0; k < n_tw; ++k) loc[k] += pose_interior(&C, rec, nv, tw + 6 * k, g);
            }
        }
#pragma omp critical
        for (int k = 0; k < n_tw; ++k) acc[0][k] += loc[k];
    }

    /* pixel edges: -g_P times the flux out through P's right, left, bottom
     * and top edges (outward normals +x, -x, +y, -y) */
    if (edge_spp > 0) {
#pragma omp parallel
        {
            double loc[16] = {0};
            vrec rec[OR_MAX_VERTS];
#pragma omp for schedule(dynamic, 16)
            for (int64_t p = 0; p < npix; ++p) {
                const double *g = dEc + 3 * p;
                if (g[0] == 0.0 && g[1] == 0.0 && g[2] == 0.0) continue;
                const double x0 = (double)(p % Wc), y0 = (double)(p / Wc);
                const uint32_t vpix = (uint32_t)(npix + p);
                for (int j = 0; j < edge_spp; ++j) {
                    double u[4];
                    rand4(seed, vpix, (uint32_t)j, 0u, u);
                    const double t = ((double)j + u[0]) / edge_spp;
                    const double ex[4] = {x0 + 1.0, x0, x0 + t, x0 + t};
                    const double ey[4] = {y0 + t, y0 + t, y0 + 1.0, y0};
                    const int axis[4] = {0, 0, 1, 1};
                    const double sgn[4] = {1.0, -1.0, 1.0, -1.0};
                    for (int k = 0; k < 4; ++k) {
                        double L[3];
                        d3 d = nrm(mat3v(C.Kc_inv, mk(ex[k], ey[k], 1.0)));
                        int nv = trace_ray(&C, mk(0.0, 0.0, 0.0), d, vpix, (uint32_t)j, L, rec);
                        if (nv == 0) continue;
                        double gl = L[0] * g[0] + L[1] * g[1] + L[2] * g[2];
                        for (int q = 0; q < n_tw; ++q) {
                            double V[2];
                            pose_img_vel(C.Kc, tw + 6 * q, rec[0].x, V);
                            loc[q] -= sgn[k] * gl * V[axis[k]] / edge_spp;
                        }
                    }
                }
            }
#pragma omp critical
            for (int q = 0; q < n_tw; ++q) acc[1][q] += loc[q];
        }
    }

    /* silhouettes */
    if (sil_spp > 0 && T > 0) {
        pose_edge *E;
        int64_t ne = pose_edges(tris, T, &E);
        const int64_t vbase = 2 * npix;
#pragma omp parallel
        {
            double loc[16] = {0};
            vrec rec[OR_MAX_VERTS];
#pragma omp for schedule(dynamic, 16)
            for (int64_t k = 0; k < ne; ++k) {
                const pose_edge *ed = &E[k];
                if (ed->nthird > 2) continue;
                d3 P0 = vert_at(verts, ed->v0), P1 = vert_at(verts, ed->v1);
                d3 m = cross(P0, P1);
                /* a silhouette when every adjacent triangle lies on one side
                 * of the plane through the camera centre and the edge */
                int sgn = 0, ok = 1;
                for (int i = 0; i < ed->nthird; ++i) {
                    double sd = dot(m, vert_at(verts, ed->third[i]));
                    int si = sd > 0.0 ? 1 : (sd < 0.0 ? -1 : 0);
                    if (si == 0 || (sgn != 0 && si != sgn)) ok = 0;
                    sgn = si;
                }
                if (!ok) continue;
                d3 P2 = vert_at(verts, ed->third[0]);
                const uint32_t vpix = (uint32_t)(vbase + k);
                for (int j = 0; j < sil_spp; ++j) {
                    double u[4], L[3], s[2];
                    rand4(seed, vpix, (uint32_t)j, 0u, u);
                    double t = ((double)j + u[0]) / sil_spp;
                    d3 p = add(P0, scl(sub(P1, P0), t));
                    if (!(p.z > 0.0)) continue;
                    pose_proj(C.Kc, p, s);
                    if (!(s[0] >= 0.0 && s[0] < Wc && s[1] >= 0.0 && s[1] < Hc)) continue;
                    double dist = len(p);
                    d3 d = scl(p, 1.0 / dist);
                    if (occluded(&S, mk(0.0, 0.0, 0.0), d, dist * (1.0 - 1e-4))) continue;
                    int nv = trace_ray(&C, scl(d, dist * (1.0 + 1e-4)), d, vpix, (uint32_t)j, L, rec);
                    if (nv == 0) continue;
                    int64_t px = (int64_t)floor(s[1]) * Wc + (int64_t)floor(s[0]);
                    double gl = L[0] * dEc[3 * px] + L[1] * dEc[3 * px + 1] + L[2] * dEc[3 * px + 2];
                    if (gl == 0.0) continue;
                    /* the silhouette's image tangent and speed, and its normal
                     * turned towards F (a point just inside F's triangle) */
                    const double dl = 1e-6;
                    double sp[2], sm[2], sq[2];
                    pose_proj(C.Kc, add(p, scl(sub(P1, P0), dl)), sp);
                    pose_proj(C.Kc, sub(p, scl(sub(P1, P0), dl)), sm);
                    double tx = sp[0] - sm[0], ty = sp[1] - sm[1];
                    double tl = sqrt(tx * tx + ty * ty);
                    double speed = tl / (2.0 * dl);
                    double nx = -ty / tl, ny = tx / tl;
                    pose_proj(C.Kc, add(p, scl(sub(P2, p), 1e-6)), sq);
                    if (nx * (sq[0] - s[0]) + ny * (sq[1] - s[1]) < 0.0) { nx = -nx; ny = -ny; }
                    for (int q = 0; q < n_tw; ++q) {
                        double Vf[2], Vb[2];
                        pose_img_vel(C.Kc, tw + 6 * q, p, Vf);
                        pose_img_vel(C.Kc, tw + 6 * q, rec[0].x, Vb);
                        loc[q] += gl * ((Vf[0] - Vb[0]) * nx + (Vf[1] - Vb[1]) * ny) * speed / sil_spp;
                    }
                }
            }
#pragma omp critical
            for (int q = 0; q < n_tw; ++q) acc[2][q] += loc[q];
        }
        free(E);
    }
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < n_tw; ++k) out[r * n_tw + k] = acc[r][k];
    free(Ep);
    scene_free(&S);
    return 0;
}
