// Memory-bound kernels: the standalone property map (Sec. 3.1 truncation
// rule, Sec. 4.1 lognormal scaling, Appendix B values), the field-mismatch
// loss and its gradient, and a throughput probe of the hardware cosine.
#include <cuda_runtime.h>

#include "device_common.cuh"

namespace grf {

namespace {

constexpr int kMapThreads = 256;
constexpr int kLossThreads = 256;
constexpr int kLossItems = 8;  // elements per thread per block pass

__global__ void __launch_bounds__(kMapThreads) map_kernel(MapDev m, int64_t n,
                                                          const float* __restrict__ Y) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
        map_store(m, i, Y[i]);
}

// L = mean (K - T)^2, g = 2 (K - T) K / n.  Per-block FP64 partial sums go to
// `part`; the last kernel adds them in block order (deterministic).
__global__ void __launch_bounds__(kLossThreads)
    mismatch_kernel(int64_t n, const float* __restrict__ K, const float* __restrict__ T,
                    float* __restrict__ gY, double* __restrict__ part) {
    __shared__ double red[kLossThreads];
    const float scale = 2.0f / static_cast<float>(n);
    double acc = 0.0;
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kLossThreads * kLossItems;
#pragma unroll
    for (int q = 0; q < kLossItems; ++q) {
        const int64_t i = base + q * kLossThreads + threadIdx.x;
        if (i < n) {
            const float k = K[i];
            const float d = k - T[i];
            gY[i] = scale * d * k;
            acc += static_cast<double>(d) * static_cast<double>(d);
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int off = kLossThreads / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(kLossThreads) sum_partials_kernel(const double* __restrict__ part,
                                                                    int64_t nb, double scale,
                                                                    double* __restrict__ out) {
    __shared__ double red[kLossThreads];
    double acc = 0.0;
    for (int64_t k = threadIdx.x; k < nb; k += kLossThreads) acc += part[k];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int off = kLossThreads / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0] * scale;
}

// Independent cos.approx chains, 8 per thread, so the MUFU pipe is the limit.
__global__ void __launch_bounds__(256) mufu_probe_kernel(int32_t iters, float* sink) {
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = 1e-3f * static_cast<float>(threadIdx.x + 37 * k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = hw_cos(v[k]);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += v[k];
    sink[static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x] = s;
}

}  // namespace

int launch_map(const MapDev& m, int64_t n, const float* Y, void* stream) {
    if (n == 0) return cudaSuccess;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (n + kMapThreads - 1) / kMapThreads;
    const int64_t cap = static_cast<int64_t>(sms) * 8;
    if (blocks > cap) blocks = cap;
    map_kernel<<<static_cast<unsigned>(blocks), kMapThreads, 0, st>>>(m, n, Y);
    count_launches(1);
    return cudaGetLastError();
}

size_t mismatch_workspace_bytes(int64_t n) {
    const int64_t nb = (n + int64_t(kLossThreads) * kLossItems - 1) / (int64_t(kLossThreads) * kLossItems);
    return static_cast<size_t>(align256((nb > 0 ? nb : 1) * 8));
}

int launch_mismatch(int64_t n, const float* K, const float* T, float* gY, double* loss, void* ws,
                    void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t nb = (n + int64_t(kLossThreads) * kLossItems - 1) / (int64_t(kLossThreads) * kLossItems);
    double* part = static_cast<double*>(ws);
    if (nb > 0) {
        mismatch_kernel<<<static_cast<unsigned>(nb), kLossThreads, 0, st>>>(n, K, T, gY, part);
        count_launches(1);
    }
    sum_partials_kernel<<<1, kLossThreads, 0, st>>>(part, nb, n > 0 ? 1.0 / static_cast<double>(n) : 0.0,
                                                    loss);
    count_launches(1);
    return cudaGetLastError();
}

int launch_mufu_probe(int32_t blocks, int32_t iters, float* sink, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mufu_probe_kernel<<<blocks, 256, 0, st>>>(iters, sink);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace grf
