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

constexpr int kMapGroups = 2;  // 4-cell groups per thread, loaded before any is processed

// One 4-cell group whose Y, K, P pointers are 16-byte and F 4-byte aligned;
// streaming stores, since nothing reads the outputs back in this launch.
__device__ __forceinline__ void map_store4(const MapDev& m, int64_t i0, float4 y) {
    const float v[4] = {y.x, y.y, y.z, y.w};
    const int bits = m.bits;
    if (bits & GRF_MAP_LOGNORMAL)
        __stcs(reinterpret_cast<float4*>(m.K + i0),
               make_float4(m.k_ref * expf(v[0]), m.k_ref * expf(v[1]), m.k_ref * expf(v[2]),
                           m.k_ref * expf(v[3])));
    if (bits & (GRF_MAP_FACIES | GRF_MAP_VALUES | GRF_MAP_POROSITY)) {
        int lab[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            lab[q] = 0;
            for (int t = 0; t < m.n_thr; ++t) lab[q] += (v[q] > m.thr[t]) ? 1 : 0;
        }
        if (bits & GRF_MAP_FACIES)
            *reinterpret_cast<uchar4*>(m.F + i0) = make_uchar4(lab[0], lab[1], lab[2], lab[3]);
        if (bits & GRF_MAP_VALUES)
            __stcs(reinterpret_cast<float4*>(m.P + i0),
                   make_float4(m.values[lab[0]], m.values[lab[1]], m.values[lab[2]], m.values[lab[3]]));
        if (bits & GRF_MAP_POROSITY) {
            float ph[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                ph[q] = fminf(fmaxf(fmaf(m.phi1, (v[q] - m.mu) * m.sigma_inv, m.phi0), m.phi_min), m.phi_max);
            __stcs(reinterpret_cast<float4*>(m.P + i0), make_float4(ph[0], ph[1], ph[2], ph[3]));
        }
    }
    if (bits & GRF_MAP_Y) __stcs(reinterpret_cast<float4*>(m.Y + i0), y);
}

// kMapGroups groups of four consecutive cells per thread, the groups of a
// block interleaved so that every load of a warp is one contiguous 512-byte
// segment.  All loads of a thread are issued before the first store, which
// doubles the bytes in flight per SM against one group per thread.  A thread
// whose groups run past n, or every thread when a pointer is misaligned
// (vec == 0), stores cell by cell.
__global__ void __launch_bounds__(kMapThreads) map_kernel(MapDev m, int64_t n,
                                                          const float* __restrict__ Y, int vec) {
    const int64_t base = static_cast<int64_t>(blockIdx.x) * (kMapThreads * kMapGroups) + threadIdx.x;
    const int64_t last = (base + static_cast<int64_t>(kMapGroups - 1) * kMapThreads) * 4;
    if (vec && last + 4 <= n) {
        float4 y[kMapGroups];
#pragma unroll
        for (int u = 0; u < kMapGroups; ++u)
            y[u] = __ldg(reinterpret_cast<const float4*>(Y + (base + u * kMapThreads) * 4));
#pragma unroll
        for (int u = 0; u < kMapGroups; ++u) map_store4(m, (base + u * kMapThreads) * 4, y[u]);
        return;
    }
    for (int u = 0; u < kMapGroups; ++u) {
        const int64_t i0 = (base + static_cast<int64_t>(u) * kMapThreads) * 4;
        for (int64_t i = i0; i < n && i < i0 + 4; ++i) map_store(m, i, Y[i]);
    }
}

// Bitruncated truncation rule (Sec. 3.1): region (i, j) of the two fields,
// then the rule's facies and optionally its value.
__global__ void __launch_bounds__(kMapThreads) bimap_kernel(grf_bimap m, int64_t n, const float* __restrict__ Y1,
                                                            const float* __restrict__ Y2,
                                                            uint8_t* __restrict__ F, float* __restrict__ P) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += stride) {
        const float y1 = Y1[k];
        const float y2 = Y2[k];
        int i = 0, j = 0;
        for (int q = 0; q < m.n_t; ++q) i += (y1 > m.t[q]) ? 1 : 0;
        for (int q = 0; q < m.n_s; ++q) j += (y2 > m.s[q]) ? 1 : 0;
        const uint8_t f = m.rule[i][j];
        F[k] = f;
        if (P != nullptr) P[k] = m.values[f];
    }
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

// One block waits on an mbarrier that no thread arrives at and no copy
// completes, through the same bounded wait as the synthesis kernels.
__global__ void selftest_wait_kernel(uint64_t limit_ns, int32_t* status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0u, limit_ns);
    if (threadIdx.x == 0) *status = ok ? 0 : 2;
}

}  // namespace

int launch_selftest_wait(uint64_t limit_ns, int32_t* status, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    selftest_wait_kernel<<<1, 32, 0, st>>>(limit_ns, status);
    count_launches(1);
    return cudaGetLastError();
}

int launch_map(const MapDev& m, int64_t n, const float* Y, void* stream) {
    if (n == 0) return cudaSuccess;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto a16 = [](const void* p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    auto a4 = [](const void* p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 3u) == 0; };
    const int vec = a16(Y) && a16(m.Y) && a16(m.K) && a16(m.P) && a4(m.F) ? 1 : 0;
    const int64_t groups = (n + 3) / 4;
    const int64_t blocks = (groups + kMapThreads * kMapGroups - 1) / (kMapThreads * kMapGroups);
    map_kernel<<<static_cast<unsigned>(blocks), kMapThreads, 0, st>>>(m, n, Y, vec);
    count_launches(1);
    return cudaGetLastError();
}

int launch_bimap(const grf_bimap& m, int64_t n, const float* Y1, const float* Y2, uint8_t* F, float* P,
                 void* stream) {
    if (n == 0) return cudaSuccess;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (n + kMapThreads - 1) / kMapThreads;
    const int64_t cap = static_cast<int64_t>(sms) * 8;
    if (blocks > cap) blocks = cap;
    bimap_kernel<<<static_cast<unsigned>(blocks), kMapThreads, 0, st>>>(m, n, Y1, Y2, F, P);
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

// ---------------------------------------------------------------------------
// Zero-allocation variant of the mismatch loss: the per-block partial sums
// live in a fixed device array owned by the library (see
// grf_mismatch_grad_noalloc in grf.h for the contract).
// ---------------------------------------------------------------------------
static_assert(int64_t(GRF_NOALLOC_MAX_BLOCKS) * kLossThreads * kLossItems == GRF_NOALLOC_MAX_CELLS,
              "cell limit must match the scratch size");
static __device__ __align__(256) double g_noalloc_partials[GRF_NOALLOC_MAX_BLOCKS];

namespace {
// Device address of the scratch array in the current device's context (host
// code cannot use the symbol's own address: on the host it names a stand-in,
// not the device memory).  Looked up on every call rather than cached: the
// lookup is a host-side table search once the module is loaded, and a cached
// address would outlive a context that cudaDeviceReset destroyed and
// recreated (where the module, and the array, may load at a new address).
// On a device's first call the lookup also loads the library's device code
// into the context.
int noalloc_scratch(double** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    *out = static_cast<double*>(p);
    return cudaSuccess;
}
}  // namespace

int launch_mufu_probe(int32_t blocks, int32_t iters, float* sink, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mufu_probe_kernel<<<blocks, 256, 0, st>>>(iters, sink);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace grf

extern "C" int grf_mismatch_grad_noalloc(int64_t n, const float* K, const float* K_target, float* gY,
                                         double* loss, void* stream) {
    if (n < 0) return grf::set_error(GRF_EINVAL, "n must be >= 0");
    if (n > GRF_NOALLOC_MAX_CELLS)
        return grf::set_error(GRF_EINVAL,
                              "n exceeds GRF_NOALLOC_MAX_CELLS (134217728) of the fixed scratch array; "
                              "use grf_mismatch_grad with a caller workspace");
    if (n > 0 && (!K || !K_target || !gY)) return grf::set_error(GRF_EINVAL, "K, K_target or gY is NULL");
    if (!loss) return grf::set_error(GRF_EINVAL, "loss is NULL");
    double* scratch = nullptr;
    int err = grf::noalloc_scratch(&scratch);
    if (err != cudaSuccess)
        return grf::set_error(GRF_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
    err = grf::launch_mismatch(n, K, K_target, gY, loss, scratch, stream);
    if (err != cudaSuccess) return grf::set_error(GRF_ECUDA, cudaGetErrorString(static_cast<cudaError_t>(err)));
    return GRF_OK;
}
