// lbvh.cu -- LBVH construction on the device: FP32 Morton codes of triangle
// centroids, a stable LSD radix sort of (code, index), the Karras (HPG 2012)
// radix tree, and a bottom-up AABB refit that packs 64-byte nodes and 48-byte
// triangles.  Integer results (codes, order, topology) and the FP32 min/max
// boxes are exact and reproducible.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace dpcs {

namespace {

constexpr int kSortTile = 256;  // items (and threads) per radix-sort block

// centroids (v0 + v1 + v2) * (1/3) in FP32 without contraction
__global__ void k_centroids(const float *__restrict__ verts, const int32_t *__restrict__ tris, int T,
                            float *__restrict__ cen) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T) return;
    const float third = 1.0f / 3.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float a = verts[3 * tris[3 * i] + k], b = verts[3 * tris[3 * i + 1] + k], c = verts[3 * tris[3 * i + 2] + k];
        cen[3 * i + k] = __fmul_rn(__fadd_rn(__fadd_rn(a, b), c), third);
    }
}

// single-block min/max of the centroids -> bounds[0..2] lo, [3..5] hi
__global__ void k_bounds(const float *__restrict__ cen, int T, float *__restrict__ bounds) {
    __shared__ float slo[3][32], shi[3][32];
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = threadIdx.x; i < T; i += blockDim.x)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lo[k] = fminf(lo[k], cen[3 * i + k]);
            hi[k] = fmaxf(hi[k], cen[3 * i + k]);
        }
#pragma unroll
    for (int k = 0; k < 3; ++k)
        for (int off = 16; off; off >>= 1) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], off));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], off));
        }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0)
        for (int k = 0; k < 3; ++k) { slo[k][w] = lo[k]; shi[k][w] = hi[k]; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < 3; ++k) {
            float a = INFINITY, b = -INFINITY;
            for (int j = 0; j < (int)(blockDim.x >> 5); ++j) { a = fminf(a, slo[k][j]); b = fmaxf(b, shi[k][j]); }
            bounds[k] = a;
            bounds[3 + k] = b;
        }
    }
}

__device__ __forceinline__ uint32_t expand10(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// 30-bit Morton code of the centroid normalised into the centroid bounds
__global__ void k_morton(const float *__restrict__ cen, const float *__restrict__ bounds, int T,
                         uint32_t *__restrict__ codes, int32_t *__restrict__ idx) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T) return;
    uint32_t q[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float lo = bounds[k], ext = __fsub_rn(bounds[3 + k], lo);
        const float inv = ext > 0.0f ? __frcp_rn(ext) : 0.0f;
        const float nrm = __fmul_rn(__fsub_rn(cen[3 * i + k], lo), inv);
        float f = floorf(__fmul_rn(nrm, 1024.0f));
        f = fminf(fmaxf(f, 0.0f), 1023.0f);
        q[k] = (uint32_t)f;
    }
    codes[i] = (expand10(q[0]) << 2) | (expand10(q[1]) << 1) | expand10(q[2]);
    idx[i] = i;
}

// --- stable LSD radix sort, 8-bit digits -----------------------------------
__global__ void k_radix_hist(const uint32_t *__restrict__ keys, int n, int shift, int nblocks,
                             uint32_t *__restrict__ hist) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int i = blockIdx.x * kSortTile + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xffu], 1u);
    __syncthreads();
    hist[threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of `total` counters in one block
__global__ void k_radix_scan(uint32_t *__restrict__ hist, int total) {
    __shared__ uint32_t part[1024];
    const int per = (total + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per;
    uint32_t s = 0;
    for (int i = b0; i < min(b0 + per, total); ++i) s += hist[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        const uint32_t v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = part[threadIdx.x] - s;
    for (int i = b0; i < min(b0 + per, total); ++i) {
        const uint32_t c = hist[i];
        hist[i] = run;
        run += c;
    }
}

__global__ void k_radix_scatter(const uint32_t *__restrict__ kin, const int32_t *__restrict__ vin,
                                uint32_t *__restrict__ kout, int32_t *__restrict__ vout, int n, int shift,
                                int nblocks, const uint32_t *__restrict__ offs) {
    __shared__ uint32_t cnt[kSortTile / 32][256];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = threadIdx.x; j < (kSortTile / 32) * 256; j += blockDim.x) (&cnt[0][0])[j] = 0u;
    __syncthreads();
    const int i = blockIdx.x * kSortTile + threadIdx.x;
    const bool valid = i < n;
    const uint32_t key = valid ? kin[i] : 0u;
    const uint32_t digit = valid ? ((key >> shift) & 0xffu) : 0x100u;
    const unsigned peers = __match_any_sync(0xffffffffu, digit);
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t rank = __popc(peers & lt);
    if (valid && (peers & lt) == 0u) cnt[w][digit] = __popc(peers);
    __syncthreads();
    if (valid) {
        uint32_t off = rank;
        for (int ww = 0; ww < w; ++ww) off += cnt[ww][digit];
        const uint32_t dst = offs[digit * nblocks + blockIdx.x] + off;
        kout[dst] = key;
        vout[dst] = vin[i];
    }
}

// --- Karras radix tree -------------------------------------------------------
__device__ __forceinline__ int delta(const uint32_t *__restrict__ c, int T, int i, int j) {
    if (j < 0 || j > T - 1) return -1;
    const uint32_t a = c[i], b = c[j];
    if (a == b) return 32 + __clz((uint32_t)(i ^ j));
    return __clz(a ^ b);
}

__global__ void k_karras(const uint32_t *__restrict__ codes, int T, float4 *__restrict__ nodes,
                         int32_t *__restrict__ parent) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T - 1) return;
    const int d = (delta(codes, T, i, i + 1) - delta(codes, T, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = delta(codes, T, i, i - d);
    int lmax = 2;
    while (delta(codes, T, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(codes, T, i, i + (l + t) * d) > dmin) l += t;
    const int j = i + l * d;
    const int dnode = delta(codes, T, i, j);
    int s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (delta(codes, T, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    const int g = i + s * d + min(d, 0);
    const int left = (min(i, j) == g) ? ~g : g;
    const int right = (max(i, j) == g + 1) ? ~(g + 1) : g + 1;
    nodes[4 * i + 3] = make_float4(__int_as_float(left), __int_as_float(right), 0.0f, 0.0f);
    if (left >= 0) parent[left] = i; else parent[T - 1 + g] = i;
    if (right >= 0) parent[right] = i; else parent[T - 1 + g + 1] = i;
}

__device__ __forceinline__ void store_box(float *nd, bool right, const float b[6]) {
    // node float layout: [0..3] left x/y, [4..7] right x/y, [8..11] z of left, right
    float *xy = nd + (right ? 4 : 0);
    float *z = nd + 8 + (right ? 2 : 0);
    __stcg(xy + 0, b[0]);
    __stcg(xy + 1, b[3]);
    __stcg(xy + 2, b[1]);
    __stcg(xy + 3, b[4]);
    __stcg(z + 0, b[2]);
    __stcg(z + 1, b[5]);
}

// one thread per leaf: pack the triangle, then walk up; the second thread to
// reach a node forms the union of its two child boxes and continues
__global__ void k_refit(const float *__restrict__ verts, const int32_t *__restrict__ tris,
                        const float *__restrict__ uv, const int32_t *__restrict__ order, int T,
                        float4 *__restrict__ nodes, const int32_t *__restrict__ parent,
                        int32_t *__restrict__ flags, float4 *__restrict__ tout, float2 *__restrict__ tuv) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= T) return;
    const int t = order[p];
    const int i0 = tris[3 * t], i1 = tris[3 * t + 1], i2 = tris[3 * t + 2];
    const float x0 = verts[3 * i0], y0 = verts[3 * i0 + 1], z0 = verts[3 * i0 + 2];
    const float x1 = verts[3 * i1], y1 = verts[3 * i1 + 1], z1 = verts[3 * i1 + 2];
    const float x2 = verts[3 * i2], y2 = verts[3 * i2 + 1], z2 = verts[3 * i2 + 2];
    // the three vertices as uploaded: a vertex shared by two triangles has
    // the same bits in both, which the watertight hit test relies on
    tout[3 * p + 0] = make_float4(x0, y0, z0, __int_as_float(t));
    tout[3 * p + 1] = make_float4(x1, y1, z1, 0.0f);
    tout[3 * p + 2] = make_float4(x2, y2, z2, 0.0f);
    tuv[3 * p + 0] = make_float2(uv[2 * i0], uv[2 * i0 + 1]);
    tuv[3 * p + 1] = make_float2(uv[2 * i1], uv[2 * i1 + 1]);
    tuv[3 * p + 2] = make_float2(uv[2 * i2], uv[2 * i2 + 1]);
    if (T < 2) return;
    float b[6] = {fminf(fminf(x0, x1), x2), fminf(fminf(y0, y1), y2), fminf(fminf(z0, z1), z2),
                  fmaxf(fmaxf(x0, x1), x2), fmaxf(fmaxf(y0, y1), y2), fmaxf(fmaxf(z0, z1), z2)};
    int child = ~p;
    int node = parent[T - 1 + p];
    while (true) {
        float *nd = reinterpret_cast<float *>(nodes + 4 * node);
        const int cl = __float_as_int(__ldcg(nd + 12));
        store_box(nd, cl != child, b);
        __threadfence();
        if (atomicAdd(&flags[node], 1) == 0) return;
        __threadfence();
        // both children are final: union
        const float lx0 = __ldcg(nd + 0), lx1 = __ldcg(nd + 1), ly0 = __ldcg(nd + 2), ly1 = __ldcg(nd + 3);
        const float rx0 = __ldcg(nd + 4), rx1 = __ldcg(nd + 5), ry0 = __ldcg(nd + 6), ry1 = __ldcg(nd + 7);
        const float lz0 = __ldcg(nd + 8), lz1 = __ldcg(nd + 9), rz0 = __ldcg(nd + 10), rz1 = __ldcg(nd + 11);
        b[0] = fminf(lx0, rx0); b[3] = fmaxf(lx1, rx1);
        b[1] = fminf(ly0, ry0); b[4] = fmaxf(ly1, ry1);
        b[2] = fminf(lz0, rz0); b[5] = fmaxf(lz1, rz1);
        if (node == 0) return;
        child = node;
        node = parent[node];
    }
}

// parent of every internal node and leaf, read back from the child
// references the Karras pass stored in the nodes
__global__ void k_parents(const float4 *__restrict__ nodes, int T, int32_t *__restrict__ parent) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T - 1) return;
    const float4 r = nodes[4 * i + 3];
    const int left = __float_as_int(r.x), right = __float_as_int(r.y);
    parent[left >= 0 ? left : T - 1 + ~left] = i;
    parent[right >= 0 ? right : T - 1 + ~right] = i;
}

inline size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

// --- PLOC: agglomerative clustering over the Morton order -------------------
// (Meister & Bittner, "Parallel Locally-Ordered Clustering for Bounding
// Volume Hierarchy Construction", IEEE TVCG 2018.)  Clusters sit in Morton
// order; each finds its nearest neighbour -- the one whose union with it has
// the smallest surface area -- among the kPlocRadius clusters on either side;
// mutual nearest neighbours merge into a new node, and the survivors are
// compacted in order, until one cluster is left.  Ties go to the smaller
// index, which orders every pair by (area, lower index, higher index): the
// least pair of a round is always mutual, so every round merges.  New nodes
// are numbered downwards from T - 2 by a prefix sum of the merge flags, so
// the last merge (the root) is node 0 and the build is deterministic.
#ifndef DPCS_PLOC_RADIUS
#define DPCS_PLOC_RADIUS 16
#endif
constexpr int kPlocRadius = DPCS_PLOC_RADIUS;
constexpr int kPlocBlock = 128;

__device__ __forceinline__ float union_area(float4 alo, float4 ahi, float4 blo, float4 bhi) {
    const float dx = fmaxf(ahi.x, bhi.x) - fminf(alo.x, blo.x);
    const float dy = fmaxf(ahi.y, bhi.y) - fminf(alo.y, blo.y);
    const float dz = fmaxf(ahi.z, bhi.z) - fminf(alo.z, blo.z);
    return 2.0f * (dx * dy + dy * dz + dz * dx);
}

// leaf clusters: the boxes of the triangle records, in leaf order
__global__ void k_ploc_init(const float4 *__restrict__ tris, int T, int32_t *__restrict__ cid,
                            float4 *__restrict__ cbox) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= T) return;
    const float4 a = tris[3 * p], b = tris[3 * p + 1], c = tris[3 * p + 2];
    cid[p] = ~p;
    cbox[2 * p] = make_float4(fminf(fminf(a.x, b.x), c.x), fminf(fminf(a.y, b.y), c.y), fminf(fminf(a.z, b.z), c.z), 0.f);
    cbox[2 * p + 1] =
        make_float4(fmaxf(fmaxf(a.x, b.x), c.x), fmaxf(fmaxf(a.y, b.y), c.y), fmaxf(fmaxf(a.z, b.z), c.z), 0.f);
}

// nearest neighbour of each of the n clusters within the radius; the block's
// clusters and the radius on either side are staged in shared memory
__global__ void __launch_bounds__(kPlocBlock) k_ploc_nn(const float4 *__restrict__ cbox, int n,
                                                       int32_t *__restrict__ nn) {
    __shared__ float4 sb[2 * (kPlocBlock + 2 * kPlocRadius)];
    const int base = blockIdx.x * kPlocBlock - kPlocRadius;
    for (int k = threadIdx.x; k < kPlocBlock + 2 * kPlocRadius; k += blockDim.x) {
        const int j = base + k;
        if (j >= 0 && j < n) {
            sb[2 * k] = cbox[2 * j];
            sb[2 * k + 1] = cbox[2 * j + 1];
        }
    }
    __syncthreads();
    const int i = blockIdx.x * kPlocBlock + threadIdx.x;
    if (i >= n) return;
    const int li = i - base;
    const float4 lo = sb[2 * li], hi = sb[2 * li + 1];
    float best = INFINITY;
    int bj = i > 0 ? i - 1 : i + 1;
    const int j0 = max(0, i - kPlocRadius), j1 = min(n - 1, i + kPlocRadius);
    for (int j = j0; j <= j1; ++j) {
        if (j == i) continue;
        const float a = union_area(lo, hi, sb[2 * (j - base)], sb[2 * (j - base) + 1]);
        if (a < best) {  // ascending j with a strict comparison: ties to the smaller index
            best = a;
            bj = j;
        }
    }
    nn[i] = bj;
}

// merge flag (the lower of a mutual pair) and keep flag (not the higher one)
__global__ void k_ploc_flags(const int32_t *__restrict__ nn, int n, uint32_t *__restrict__ mflag,
                             uint32_t *__restrict__ kflag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = nn[i];
    const bool mutual = nn[j] == i;
    mflag[i] = (mutual && i < j) ? 1u : 0u;
    kflag[i] = (mutual && i > j) ? 0u : 1u;
}

// with mscan / kscan the exclusive prefix sums of the flags: write the new
// nodes (ids next - 1 - mscan[i]) and the surviving clusters in order;
// counts = (clusters left, merges)
__global__ void k_ploc_compact(const int32_t *__restrict__ nn, int n, const uint32_t *__restrict__ mscan,
                               const uint32_t *__restrict__ kscan, int next, const int32_t *__restrict__ cid,
                               const float4 *__restrict__ cbox, int32_t *__restrict__ cid_out,
                               float4 *__restrict__ cbox_out, float4 *__restrict__ nodes,
                               int32_t *__restrict__ counts) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = nn[i];
    const bool mutual = nn[j] == i;
    if (i == n - 1) {
        counts[0] = (int32_t)(kscan[i] + ((mutual && i > j) ? 0u : 1u));
        counts[1] = (int32_t)(mscan[i] + ((mutual && i < j) ? 1u : 0u));
    }
    if (mutual && i > j) return;  // merged into j
    const uint32_t o = kscan[i];
    const float4 lo = cbox[2 * i], hi = cbox[2 * i + 1];
    if (mutual) {
        const int id = next - 1 - (int)mscan[i];
        const float4 rlo = cbox[2 * j], rhi = cbox[2 * j + 1];
        float4 *nd = nodes + 4 * (int64_t)id;
        nd[0] = make_float4(lo.x, hi.x, lo.y, hi.y);
        nd[1] = make_float4(rlo.x, rhi.x, rlo.y, rhi.y);
        nd[2] = make_float4(lo.z, hi.z, rlo.z, rhi.z);
        nd[3] = make_float4(__int_as_float(cid[i]), __int_as_float(cid[j]), 0.0f, 0.0f);
        cid_out[o] = id;
        cbox_out[2 * o] = make_float4(fminf(lo.x, rlo.x), fminf(lo.y, rlo.y), fminf(lo.z, rlo.z), 0.f);
        cbox_out[2 * o + 1] = make_float4(fmaxf(hi.x, rhi.x), fmaxf(hi.y, rhi.y), fmaxf(hi.z, rhi.z), 0.f);
    } else {
        cid_out[o] = cid[i];
        cbox_out[2 * o] = lo;
        cbox_out[2 * o + 1] = hi;
    }
}

// deepest leaf: internal nodes on its path from the root (stops counting
// past `limit`, so a malformed tree cannot loop)
__global__ void k_tree_depth(const int32_t *__restrict__ parent, int T, int limit, int32_t *__restrict__ depth) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= T) return;
    int d = 1, node = parent[T - 1 + p];
    while (node != 0 && d <= limit) {
        node = parent[node];
        ++d;
    }
    atomicMax(depth, d);
}

}  // namespace

size_t ploc_scratch_bytes(int32_t T) {
    const size_t n = (size_t)(T > 0 ? T : 1);
    return 2 * align256(n * 4) + 2 * align256(n * 32) + align256(n * 4) + 2 * align256(n * 4) +
           align256(n * 64) + align256(2 * n * 4) + align256(4 * 4);
}

int launch_ploc(Scene &sc, void *scratch, size_t scratch_bytes, int max_depth, cudaStream_t st, int32_t *depth_out) {
    const int T = sc.T;
    *depth_out = 0;
    if (T < 3) return 0;  // the radix tree of two leaves is already optimal
    if (scratch_bytes < ploc_scratch_bytes(T)) return DPCS_ERR_INVALID_ARG;
    const size_t n = (size_t)T;
    char *q = (char *)scratch;
    auto take = [&](size_t bytes) {
        char *r = q;
        q += align256(bytes);
        return (void *)r;
    };
    int32_t *cid[2] = {(int32_t *)take(n * 4), (int32_t *)take(n * 4)};
    float4 *cbox[2] = {(float4 *)take(n * 32), (float4 *)take(n * 32)};
    int32_t *nn = (int32_t *)take(n * 4);
    uint32_t *mflag = (uint32_t *)take(n * 4), *kflag = (uint32_t *)take(n * 4);
    float4 *nodes = (float4 *)take(n * 64);
    int32_t *parent = (int32_t *)take(2 * n * 4);
    int32_t *counts = (int32_t *)take(4 * 4);
    const int tb = 256;
    int launches = 0;
    k_ploc_init<<<(T + tb - 1) / tb, tb, 0, st>>>(sc.tris, T, cid[0], cbox[0]);
    ++launches;
    int cur = 0, count = T, next = T - 1;
    while (count > 1) {
        const int g = (count + tb - 1) / tb;
        k_ploc_nn<<<(count + kPlocBlock - 1) / kPlocBlock, kPlocBlock, 0, st>>>(cbox[cur], count, nn);
        k_ploc_flags<<<g, tb, 0, st>>>(nn, count, mflag, kflag);
        k_radix_scan<<<1, 1024, 0, st>>>(mflag, count);
        k_radix_scan<<<1, 1024, 0, st>>>(kflag, count);
        k_ploc_compact<<<g, tb, 0, st>>>(nn, count, mflag, kflag, next, cid[cur], cbox[cur], cid[1 - cur],
                                         cbox[1 - cur], nodes, counts);
        launches += 5;
        int32_t h[2];
        cudaError_t e = cudaMemcpyAsync(h, counts, sizeof h, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return DPCS_ERR_CUDA;
        if (h[1] < 1 || h[0] != count - h[1] || h[1] > next) return DPCS_ERR_DEVICE_CHECK;  // every round merges
        count = h[0];
        next -= h[1];
        cur = 1 - cur;
    }
    if (next != 0) return DPCS_ERR_DEVICE_CHECK;
    // depth of the new tree against the traversal stack
    k_parents<<<(T - 1 + tb - 1) / tb, tb, 0, st>>>(nodes, T, parent);
    cudaMemsetAsync(counts, 0, 4, st);
    k_tree_depth<<<(T + tb - 1) / tb, tb, 0, st>>>(parent, T, max_depth + 1, counts);
    launches += 2;
    int32_t d = 0;
    cudaError_t e = cudaMemcpyAsync(&d, counts, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return DPCS_ERR_CUDA;
    *depth_out = d;
    if (d > max_depth) return launches;  // too deep for the traversal stack: the radix tree stays
    e = cudaMemcpyAsync(sc.nodes, nodes, (n - 1) * 64, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return DPCS_ERR_CUDA;
    sc.root = 0;
    return launches;
}

size_t lbvh_scratch_bytes(int32_t T) {
    const size_t n = (size_t)(T > 0 ? T : 1);
    const size_t nb = (n + kSortTile - 1) / kSortTile;
    return align256(3 * n * 4) + align256(6 * 4) + 4 * align256(n * 4) + align256(256 * nb * 4) +
           align256((2 * n) * 4) + align256(n * 4);
}

size_t lbvh_refit_scratch_bytes(int32_t T) {
    const size_t n = (size_t)(T > 0 ? T : 1);
    return align256((2 * n) * 4) + align256(n * 4);
}

int launch_lbvh_refit(const float *d_verts, Scene &sc, void *scratch, size_t scratch_bytes, cudaStream_t st) {
    const int T = sc.T;
    if (T <= 0) return 0;
    if (scratch_bytes < lbvh_refit_scratch_bytes(T)) return DPCS_ERR_INVALID_ARG;
    const size_t n = (size_t)T;
    int32_t *parent = (int32_t *)scratch;
    int32_t *flags = (int32_t *)((char *)scratch + align256(2 * n * 4));
    const int tb = 256, gb = (T + tb - 1) / tb;
    int launches = 0;
    if (T >= 2) {
        cudaMemsetAsync(flags, 0, n * 4, st);
        k_parents<<<(T - 1 + tb - 1) / tb, tb, 0, st>>>(sc.nodes, T, parent);
        ++launches;
    }
    k_refit<<<gb, tb, 0, st>>>(d_verts, sc.vidx, sc.uv, sc.order, T, sc.nodes, parent, flags, sc.tris, sc.tuv);
    return launches + 1;
}

namespace {
struct Rigid {
    float R[9], t[3];
};
__global__ void k_rigid(const float *__restrict__ in, int32_t V, const Rigid m, float *__restrict__ out) {
    const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    const float x = in[3 * v], y = in[3 * v + 1], z = in[3 * v + 2];
    out[3 * v] = m.R[0] * x + m.R[1] * y + m.R[2] * z + m.t[0];
    out[3 * v + 1] = m.R[3] * x + m.R[4] * y + m.R[5] * z + m.t[1];
    out[3 * v + 2] = m.R[6] * x + m.R[7] * y + m.R[8] * z + m.t[2];
}
}  // namespace

int launch_rigid_transform(const float *in, int32_t V, const float R[9], const float t[3], float *out,
                           cudaStream_t st) {
    if (V <= 0) return 0;
    Rigid m;
    for (int i = 0; i < 9; ++i) m.R[i] = R[i];
    for (int i = 0; i < 3; ++i) m.t[i] = t[i];
    k_rigid<<<(V + 255) / 256, 256, 0, st>>>(in, V, m, out);
    return 1;
}

int launch_lbvh_build(const float *d_verts, int32_t V, const int32_t *d_tris, int32_t T, const float *d_uv,
                      Scene &sc, void *scratch, size_t scratch_bytes, cudaStream_t st) {
    (void)V;
    if (T <= 0) {
        sc.root = kEmptyRoot;
        return 0;
    }
    if (scratch_bytes < lbvh_scratch_bytes(T)) return DPCS_ERR_INVALID_ARG;
    const size_t n = (size_t)T;
    const int nb = (int)((n + kSortTile - 1) / kSortTile);
    char *p = (char *)scratch;
    auto take = [&](size_t bytes) {
        char *r = p;
        p += align256(bytes);
        return (void *)r;
    };
    float *cen = (float *)take(3 * n * 4);
    float *bounds = (float *)take(6 * 4);
    uint32_t *ka = (uint32_t *)take(n * 4), *kb = (uint32_t *)take(n * 4);
    int32_t *va = (int32_t *)take(n * 4), *vb = (int32_t *)take(n * 4);
    uint32_t *hist = (uint32_t *)take(256 * (size_t)nb * 4);
    int32_t *parent = (int32_t *)take(2 * n * 4);
    int32_t *flags = (int32_t *)take(n * 4);
    int launches = 0;
    const int tb = 256, gb = (T + tb - 1) / tb;
    k_centroids<<<gb, tb, 0, st>>>(d_verts, d_tris, T, cen);
    k_bounds<<<1, 1024, 0, st>>>(cen, T, bounds);
    k_morton<<<gb, tb, 0, st>>>(cen, bounds, T, ka, va);
    launches += 3;
    for (int shift = 0; shift < 32; shift += 8) {
        k_radix_hist<<<nb, kSortTile, 0, st>>>(ka, T, shift, nb, hist);
        k_radix_scan<<<1, 1024, 0, st>>>(hist, 256 * nb);
        k_radix_scatter<<<nb, kSortTile, 0, st>>>(ka, va, kb, vb, T, shift, nb, hist);
        launches += 3;
        uint32_t *tk = ka; ka = kb; kb = tk;
        int32_t *tv = va; va = vb; vb = tv;
    }
    // after 4 passes the sorted data is back in (ka, va)
    cudaMemcpyAsync(sc.codes, ka, n * 4, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(sc.order, va, n * 4, cudaMemcpyDeviceToDevice, st);
    if (T >= 2) {
        cudaMemsetAsync(flags, 0, n * 4, st);
        k_karras<<<(T - 1 + tb - 1) / tb, tb, 0, st>>>(ka, T, sc.nodes, parent);
        ++launches;
    }
    k_refit<<<gb, tb, 0, st>>>(d_verts, d_tris, d_uv, va, T, sc.nodes, parent, flags, sc.tris, sc.tuv);
    ++launches;
    sc.root = T >= 2 ? 0 : ~0;
    return launches;
}

}  // namespace dpcs
