// optim.cu -- the compensation step around the renderer (Eq. 13): the L2
// image loss with its gradient, and a bias-corrected Adam update followed by
// the clamp that keeps parameters inside their valid range.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace dpcs {

namespace {

constexpr int kLossBlock = 256;
constexpr int kLossGrid = 296;  // 2 blocks per SM on a 148-152 SM part; fixed so partials need no resizing

// dIc = Ic - target; per-block partial sums of 1/2 (Ic - target)^2
__global__ void k_l2_partial(const float *__restrict__ Ic, const float *__restrict__ tgt, int64_t n,
                             float *__restrict__ dIc, double *__restrict__ partial) {
    __shared__ double red[kLossBlock / 32];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float d = Ic[i] - tgt[i];
        dIc[i] = d;
        s += 0.5 * (double)d * (double)d;
    }
    for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int j = 0; j < kLossBlock / 32; ++j) t += red[j];
        partial[blockIdx.x] = t;
    }
}

__global__ void k_l2_final(const double *__restrict__ partial, int nb, float *__restrict__ loss) {
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partial[i];
    for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int j = 0; j < (int)(blockDim.x >> 5); ++j) t += red[j];
        *loss = (float)t;
    }
}

// Eq. 9's data term with |.| read as an L1 norm: per-block partial sums of
// scale |Ic - target|, and dIc = scale sign(Ic - target) with sign(0) = 0.
__global__ void k_l1_partial(const float *__restrict__ Ic, const float *__restrict__ tgt, int64_t n, float scale,
                             float *__restrict__ dIc, double *__restrict__ partial) {
    __shared__ double red[kLossBlock / 32];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float d = Ic[i] - tgt[i];
        dIc[i] = d > 0.0f ? scale : (d < 0.0f ? -scale : 0.0f);
        s += (double)scale * fabs((double)d);
    }
    for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int j = 0; j < kLossBlock / 32; ++j) t += red[j];
        partial[blockIdx.x] = t;
    }
}

__device__ __forceinline__ float sgnf(float d) { return d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f); }

// Eq. 9's regulariser L(m) read as anisotropic total variation of a texture
// m (H x W x C): weight * sum over texels and channels of |m(x+1,y) - m(x,y)|
// + |m(x,y+1) - m(x,y)|.  Each texel gathers the sign terms of the (up to)
// four differences it takes part in, so the gradient needs no atomics;
// grad += d loss / d m, and per-block partial sums of the loss.
__global__ void k_tv_partial(const float *__restrict__ m, int H, int W, int C, float weight,
                             float *__restrict__ grad, double *__restrict__ partial) {
    __shared__ double red[kLossBlock / 32];
    double s = 0.0;
    const int64_t n = (int64_t)H * W * C;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i / C;
        const int x = (int)(t % W), y = (int)(t / W);
        const float v = m[i];
        float g = 0.0f;
        if (x + 1 < W) {
            const float d = m[i + C] - v;
            g -= sgnf(d);
            s += fabs((double)d);
        }
        if (y + 1 < H) {
            const float d = m[i + (int64_t)W * C] - v;
            g -= sgnf(d);
            s += fabs((double)d);
        }
        if (x > 0) g += sgnf(v - m[i - C]);
        if (y > 0) g += sgnf(v - m[i - (int64_t)W * C]);
        grad[i] += weight * g;
    }
    s *= (double)weight;
    for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int j = 0; j < kLossBlock / 32; ++j) t += red[j];
        partial[blockIdx.x] = t;
    }
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float bc1,
                       float bc2, float lo, float hi) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / bc1, vh = vi / bc2;
    const float pi = p[i] - lr * mh / (sqrtf(vh) + eps);
    p[i] = fminf(fmaxf(pi, lo), hi);
}

}  // namespace

int l2_partial_slots() { return kLossGrid; }

int launch_l2_loss(const float *Ic, const float *target, int64_t n, float *dIc, float *loss, double *partial,
                   cudaStream_t st) {
    k_l2_partial<<<kLossGrid, kLossBlock, 0, st>>>(Ic, target, n, dIc, partial);
    k_l2_final<<<1, 1024, 0, st>>>(partial, kLossGrid, loss);
    return 2;
}

int launch_l1_loss(const float *Ic, const float *target, int64_t n, float scale, float *dIc, float *loss,
                   double *partial, cudaStream_t st) {
    k_l1_partial<<<kLossGrid, kLossBlock, 0, st>>>(Ic, target, n, scale, dIc, partial);
    k_l2_final<<<1, 1024, 0, st>>>(partial, kLossGrid, loss);
    return 2;
}

int launch_tv_loss(const float *m, int H, int W, int C, float weight, float *grad, float *loss, double *partial,
                   cudaStream_t st) {
    k_tv_partial<<<kLossGrid, kLossBlock, 0, st>>>(m, H, W, C, weight, grad, partial);
    k_l2_final<<<1, 1024, 0, st>>>(partial, kLossGrid, loss);
    return 2;
}

int launch_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2, float eps,
                int32_t step, float lo, float hi, cudaStream_t st) {
    const float bc1 = (float)(1.0 - pow((double)b1, (double)step));
    const float bc2 = (float)(1.0 - pow((double)b2, (double)step));
    k_adam<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, bc1, bc2, lo, hi);
    return 1;
}

}  // namespace dpcs
