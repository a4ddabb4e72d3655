// probe.cu -- measured roofs for the rendering kernels, built as a
// measurement library of its own (libdpcs_probe.so; the product library does
// not contain it).  The forward and the adjoint read a scene and textures
// that stay resident in L2, and the adjoint scatters its gradients with
// float4 atomics; neither rate is a published figure, so these two kernels
// measure them on the device at hand.  They are measurement helpers, not
// part of the method.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dpcs_probe.h"

namespace {

constexpr int kProbeBlock = 512;
constexpr int kLoadBlocksPerSM = 2;    // 1024 threads x 4 loads of 16 B in flight per SM covers L2 latency
constexpr int kAtomicBlocksPerSM = 4;  // 2048 resident threads per SM

// Each pass reads every 16-byte word of buf once with loads that cache in L2
// only (ld.global.cg), four independent loads in flight per thread.
__global__ void __launch_bounds__(kProbeBlock, kLoadBlocksPerSM)
    k_probe_l2_load(const uint4 *__restrict__ buf, int64_t n4, int passes, unsigned *__restrict__ sink) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    unsigned acc = 0u;
    for (int p = 0; p < passes; ++p) {
        int64_t i = t0;
        for (; i + 3 * stride < n4; i += 4 * stride) {
            const uint4 a = __ldcg(buf + i), b = __ldcg(buf + i + stride);
            const uint4 c = __ldcg(buf + i + 2 * stride), d = __ldcg(buf + i + 3 * stride);
            acc ^= (a.x ^ a.y ^ a.z ^ a.w) ^ (b.x ^ b.y ^ b.z ^ b.w) ^ (c.x ^ c.y ^ c.z ^ c.w) ^ (d.x ^ d.y ^ d.z ^ d.w);
        }
        for (; i < n4; i += stride) {
            const uint4 a = __ldcg(buf + i);
            acc ^= a.x ^ a.y ^ a.z ^ a.w;
        }
    }
    if (acc == 0x9e3779b9u) sink[0] = acc;  // the buffer is zero, so this never stores; it keeps the loads live
}

// per_thread float4 atomic adds at texels drawn by a per-thread LCG: the
// lanes of a warp hit unrelated texels, as the adjoint's scatters do once
// paths have bounced.  The index (h >> 8) * texels >> 24 lies in [0, texels).
__global__ void __launch_bounds__(kProbeBlock, kAtomicBlocksPerSM)
    k_probe_atomic4(float4 *__restrict__ buf, int32_t texels, int64_t per_thread) {
    uint32_t h = (uint32_t)(blockIdx.x * blockDim.x + threadIdx.x) * 0x9e3779b1u + 0x7f4a7c15u;
    const float4 one = make_float4(1.0f, 1.0f, 1.0f, 1.0f);
    for (int64_t k = 0; k < per_thread; ++k) {
        h = h * 1664525u + 1013904223u;
        const int32_t idx = (int32_t)(((uint64_t)(h >> 8) * (uint64_t)texels) >> 24);
        atomicAdd(buf + idx, one);
    }
}

constexpr int32_t kOk = 0, kBadArg = -1, kOom = -2, kCuda = -3;

// best of `reps` event-timed launches of fn on stream 0, in ms
template <class F>
int32_t time_best(int reps, F fn, float *best) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return kCuda;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return kCuda;
    }
    *best = 0.0f;
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < reps + 1 && e == cudaSuccess; ++r) {  // launch 0 is a warm-up
        cudaEventRecord(e0, 0);
        fn();
        cudaEventRecord(e1, 0);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        float ms = 0.0f;
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && (*best == 0.0f || ms < *best)) *best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return kCuda;
    return *best > 0.0f ? kOk : kCuda;
}

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

int32_t probe_setup(int32_t device, int *sms) {
    if (cudaSetDevice(device) != cudaSuccess) return kCuda;
    if (cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return kCuda;
    return kOk;
}

}  // namespace

extern "C" {

int32_t dpcs_probe_l2_load(int32_t device, size_t bytes, int32_t passes, double *gbs) {
    if (!gbs || bytes == 0 || bytes % 16 != 0 || bytes > ((size_t)64 << 20) || passes < 1 || passes > 4096)
        return kBadArg;
    int sms = 0;
    int32_t s = probe_setup(device, &sms);
    if (s) return s;
    DevBuf buf, sink;
    if (cudaMalloc(&buf.p, bytes) != cudaSuccess || cudaMalloc(&sink.p, 16) != cudaSuccess) {
        cudaGetLastError();
        return kOom;
    }
    if (cudaMemset(buf.p, 0, bytes) != cudaSuccess) return kCuda;
    const int64_t n4 = (int64_t)(bytes / 16);
    const int grid = sms * kLoadBlocksPerSM;
    float ms = 0.0f;
    s = time_best(3, [&] {
        k_probe_l2_load<<<grid, kProbeBlock>>>((const uint4 *)buf.p, n4, passes, (unsigned *)sink.p);
    }, &ms);
    if (s) return s;
    *gbs = (double)bytes * passes / (ms * 1e-3) / 1e9;
    return kOk;
}

int32_t dpcs_probe_atomic4(int32_t device, int32_t texels, int64_t n_atomics, double *gatomics) {
    if (!gatomics || texels < 1 || texels > (1 << 24) || n_atomics < 1 || n_atomics > ((int64_t)1 << 34))
        return kBadArg;
    int sms = 0;
    int32_t s = probe_setup(device, &sms);
    if (s) return s;
    DevBuf buf;
    const size_t bytes = (size_t)texels * 16;
    if (cudaMalloc(&buf.p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return kOom;
    }
    if (cudaMemset(buf.p, 0, bytes) != cudaSuccess) return kCuda;
    const int grid = sms * kAtomicBlocksPerSM;
    const int64_t threads = (int64_t)grid * kProbeBlock;
    const int64_t per_thread = (n_atomics + threads - 1) / threads;
    float ms = 0.0f;
    s = time_best(3, [&] { k_probe_atomic4<<<grid, kProbeBlock>>>((float4 *)buf.p, texels, per_thread); }, &ms);
    if (s) return s;
    *gatomics = (double)(threads * per_thread) / (ms * 1e-3) / 1e9;
    return kOk;
}

}  // extern "C"
