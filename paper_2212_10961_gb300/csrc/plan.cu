// Cell plan: spatial binning of arbitrary cell centres.
//
// The paper evaluates Eq. (DiscreteFT) directly at the cell centres of an
// arbitrary (possibly unstructured) mesh (Sec. 4.1).  The synthesis kernels
// split each phase at a per-warp origin, which is accurate and cheap only when
// a warp's cells are close together.  The plan provides that locality:
//   1. bounding box of every segment (ordered-int atomics, warp-aggregated);
//   2. an isotropic quantisation grid of 2^10 levels along the longest axis;
//   3. 64-bit keys (segment << 30 | Morton code of the quantised position);
//   4. stable LSD radix sort of (key, original index), 8-bit digits;
//   5. gather of the sorted SoA coordinates.
// Everything runs on the stream without host synchronisation and is
// deterministic (the sort is stable, so equal keys keep the input order).
#include <cuda_runtime.h>

#include <cstdint>
#include <new>

#include "device_common.cuh"

namespace grf {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 keys per block
constexpr int kRadix = 256;

__device__ __forceinline__ int32_t float_to_ordered(float f) {
    int32_t b = __float_as_int(f);
    return b >= 0 ? b : b ^ 0x7fffffff;
}
__device__ __forceinline__ float ordered_to_float(int32_t b) {
    return __int_as_float(b >= 0 ? b : b ^ 0x7fffffff);
}

__device__ __forceinline__ int find_segment(const SegInfo* segs, int n_segments, int64_t i) {
    int lo = 0, hi = n_segments - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (segs[mid].begin <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Segment bounding boxes are accumulated as ordered ints in lo/hi.
__global__ void seg_init_kernel(SegInfo* segs, int n_segments) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_segments) return;
    for (int k = 0; k < 3; ++k) {
        reinterpret_cast<int32_t*>(segs[s].lo)[k] = float_to_ordered(INFINITY);
        reinterpret_cast<int32_t*>(segs[s].hi)[k] = float_to_ordered(-INFINITY);
    }
}

__global__ void bbox_kernel(const float* __restrict__ x, const float* __restrict__ y,
                            const float* __restrict__ z, int dim, int64_t n, SegInfo* segs,
                            int n_segments, int32_t* status) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const bool in = i < n;
    const int seg = in ? find_segment(segs, n_segments, i) : -1;
    float v[3] = {0.f, 0.f, 0.f};
    if (in) {
        v[0] = x[i];
        if (dim > 1) v[1] = y[i];
        if (dim > 2) v[2] = z[i];
        for (int k = 0; k < dim; ++k)
            if (!isfinite(v[k])) atomicOr(status, 1);
    }
    const unsigned mask = __ballot_sync(0xffffffffu, in);
    if (!in) return;
    const int seg0 = __shfl_sync(mask, seg, __ffs(mask) - 1);
    const bool uniform = __all_sync(mask, seg == seg0) && mask == 0xffffffffu;
    for (int k = 0; k < dim; ++k) {
        int32_t lo = float_to_ordered(v[k]);
        int32_t hi = lo;
        if (uniform) {
            for (int off = 16; off > 0; off >>= 1) {
                lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, off));
                hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, off));
            }
            if ((threadIdx.x & 31) == 0) {
                atomicMin(reinterpret_cast<int32_t*>(segs[seg].lo) + k, lo);
                atomicMax(reinterpret_cast<int32_t*>(segs[seg].hi) + k, hi);
            }
        } else {
            atomicMin(reinterpret_cast<int32_t*>(segs[seg].lo) + k, lo);
            atomicMax(reinterpret_cast<int32_t*>(segs[seg].hi) + k, hi);
        }
    }
}

// Quantisation grid per segment: cubic cells of side L_max / 2^kMortonBits
// (L_max = largest bounding-box extent), so that the Morton (Z-order) code
// of the quantised position orders cells along a space-filling curve and
// every aligned run of 2^k sorted cells is a compact, roughly cubic block.
__global__ void brick_kernel(SegInfo* segs, int n_segments, int dim) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_segments) return;
    SegInfo& g = segs[s];
    float L[3] = {0.f, 0.f, 0.f};
    float Lmax = 0.f;
    for (int k = 0; k < 3; ++k) {
        float lo = ordered_to_float(reinterpret_cast<int32_t*>(g.lo)[k]);
        float hi = ordered_to_float(reinterpret_cast<int32_t*>(g.hi)[k]);
        if (k >= dim || g.count == 0 || !(hi >= lo)) {
            lo = 0.f;
            hi = 0.f;
        }
        g.lo[k] = lo;
        g.hi[k] = hi;
        L[k] = hi - lo;
        Lmax = fmaxf(Lmax, L[k]);
    }
    const double levels = double(1 << kMortonBits);
    for (int k = 0; k < 3; ++k) {
        int nb = 1;
        float inv = 0.f;
        if (L[k] > 0.f && Lmax > 0.f) {
            const double per_unit = levels / static_cast<double>(Lmax);
            double q = ceil(static_cast<double>(L[k]) * per_unit);
            nb = q < 1.0 ? 1 : (q > levels ? int(levels) : int(q));
            inv = static_cast<float>(per_unit);
        }
        g.nb[k] = nb;
        g.inv_brick[k] = inv;
    }
}

__device__ __forceinline__ uint32_t spread_bits3(uint32_t v) {  // 10 bits -> every 3rd bit
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}
__device__ __forceinline__ uint32_t spread_bits2(uint32_t v) {  // 10 bits -> every 2nd bit
    v &= 0x3ffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

__global__ void key_kernel(const float* __restrict__ x, const float* __restrict__ y,
                           const float* __restrict__ z, int dim, int64_t n,
                           const SegInfo* __restrict__ segs, int n_segments,
                           uint64_t* __restrict__ keys, int32_t* __restrict__ vals) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int s = find_segment(segs, n_segments, i);
    const SegInfo& g = segs[s];
    float v[3] = {x[i], dim > 1 ? y[i] : 0.f, dim > 2 ? z[i] : 0.f};
    uint32_t b[3] = {0u, 0u, 0u};
    for (int k = 0; k < dim; ++k) {
        float f = (v[k] - g.lo[k]) * g.inv_brick[k];
        int q = isfinite(f) ? static_cast<int>(floorf(f)) : 0;
        q = q < 0 ? 0 : (q >= g.nb[k] ? g.nb[k] - 1 : q);
        b[k] = static_cast<uint32_t>(q);
    }
    uint32_t morton;
    if (dim == 3)
        morton = spread_bits3(b[0]) | (spread_bits3(b[1]) << 1) | (spread_bits3(b[2]) << 2);
    else if (dim == 2)
        morton = spread_bits2(b[0]) | (spread_bits2(b[1]) << 1);
    else
        morton = b[0];
    keys[i] = (static_cast<uint64_t>(s) << 30) | morton;
    vals[i] = static_cast<int32_t>(i);
}

// ---- stable LSD radix sort, 8-bit digits -----------------------------------------

__global__ void __launch_bounds__(kSortThreads)
    radix_hist_kernel(const uint64_t* __restrict__ keys, int64_t n, int shift,
                      uint32_t* __restrict__ counts, int nblk) {
    __shared__ uint32_t hist[kRadix];
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) hist[d] = 0u;
    __syncthreads();
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kSortTile;
    for (int r = 0; r < kSortItems; ++r) {
        int64_t i = base + r * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&hist[(keys[i] >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x)
        counts[static_cast<int64_t>(d) * nblk + blockIdx.x] = hist[d];
}

// Exclusive scan of `len` counts in place, one block of 1024 threads.
__global__ void __launch_bounds__(1024) scan_kernel(uint32_t* __restrict__ data, int64_t len) {
    __shared__ uint32_t part[1024];
    const int64_t per = (len + 1023) / 1024;
    const int64_t b = threadIdx.x * per;
    const int64_t e = b + per < len ? b + per : len;
    uint32_t sum = 0u;
    for (int64_t k = b; k < e; ++k) sum += data[k];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        uint32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = threadIdx.x > 0 ? part[threadIdx.x - 1] : 0u;
    for (int64_t k = b; k < e; ++k) {
        uint32_t v = data[k];
        data[k] = run;
        run += v;
    }
}

// Stable scatter: item order inside a tile is (round, warp, lane), which is
// the input order; ranks are counted in that order.
__global__ void __launch_bounds__(kSortThreads)
    radix_scatter_kernel(const uint64_t* __restrict__ keys_in, const int32_t* __restrict__ vals_in,
                         uint64_t* __restrict__ keys_out, int32_t* __restrict__ vals_out,
                         int64_t n, int shift, const uint32_t* __restrict__ offsets, int nblk) {
    constexpr int kWarps = kSortThreads / 32;
    __shared__ uint32_t base[kRadix];           // global start of each digit for this tile
    __shared__ uint32_t running[kRadix];        // items of each digit placed so far
    __shared__ uint32_t warp_cnt[kWarps][kRadix];
    __shared__ uint32_t warp_off[kWarps][kRadix];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) {
        base[d] = offsets[static_cast<int64_t>(d) * nblk + blockIdx.x];
        running[d] = 0u;
    }
    for (int k = threadIdx.x; k < kWarps * kRadix; k += blockDim.x) (&warp_cnt[0][0])[k] = 0u;
    __syncthreads();
    const int64_t tbase = static_cast<int64_t>(blockIdx.x) * kSortTile;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = tbase + r * kSortThreads + threadIdx.x;
        const bool in = i < n;
        uint64_t key = in ? keys_in[i] : 0ull;
        int32_t val = in ? vals_in[i] : 0;
        // out-of-range items get a digit of their own (never stored)
        const int digit = in ? static_cast<int>((key >> shift) & 0xffu) : kRadix;
        const unsigned peers = __match_any_sync(0xffffffffu, digit);
        const int rank = __popc(peers & lt_mask);
        const bool leader = (peers & lt_mask) == 0u;
        if (leader && in) warp_cnt[warp][digit] = __popc(peers);
        __syncthreads();
        for (int d = threadIdx.x; d < kRadix; d += blockDim.x) {
            uint32_t run = running[d];
            for (int w = 0; w < kWarps; ++w) {
                warp_off[w][d] = run;
                run += warp_cnt[w][d];
                warp_cnt[w][d] = 0u;
            }
            running[d] = run;
        }
        __syncthreads();
        if (in) {
            const uint32_t pos = base[digit] + warp_off[warp][digit] + static_cast<uint32_t>(rank);
            keys_out[pos] = key;
            vals_out[pos] = val;
        }
        __syncthreads();
    }
}

__global__ void gather_kernel(const float* __restrict__ x, const float* __restrict__ y,
                              const float* __restrict__ z, int dim, int64_t n,
                              const int32_t* __restrict__ perm, float* __restrict__ xs,
                              float* __restrict__ ys, float* __restrict__ zs) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t o = perm[i];
    xs[i] = x[o];
    if (dim > 1) ys[i] = y[o];
    if (dim > 2) zs[i] = z[o];
}

int64_t sort_blocks(int64_t n) { return (n + kSortTile - 1) / kSortTile; }

}  // namespace

size_t radix_sort_temp_bytes(int64_t n_cells) {
    return static_cast<size_t>(sort_blocks(n_cells)) * kRadix * sizeof(uint32_t);
}

int launch_plan(int32_t dim, int32_t n_segments, const int64_t* seg_offsets_host, const float* x,
                const float* y, const float* z, void* plan, const PlanLayout& L, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* base = static_cast<unsigned char*>(plan);
    const int64_t n = seg_offsets_host[n_segments];
    PlanHeader* hdr = reinterpret_cast<PlanHeader*>(base);
    SegInfo* segs = reinterpret_cast<SegInfo*>(base + L.off_segs);
    float* xs = reinterpret_cast<float*>(base + L.off_xs);
    float* ys = reinterpret_cast<float*>(base + L.off_ys);
    float* zs = reinterpret_cast<float*>(base + L.off_zs);
    int32_t* perm = reinterpret_cast<int32_t*>(base + L.off_perm);
    uint64_t* keys_a = reinterpret_cast<uint64_t*>(base + L.off_keys_in);
    uint64_t* keys_b = reinterpret_cast<uint64_t*>(base + L.off_keys_out);
    int32_t* vals_b = reinterpret_cast<int32_t*>(base + L.off_vals_in);
    uint32_t* counts = reinterpret_cast<uint32_t*>(base + L.off_sort_tmp);

    // header and segment table from the host (small synchronous-staging copies)
    PlanHeader h{};
    h.magic = kPlanMagic;
    h.status = 0;
    h.dim = dim;
    h.n_segments = n_segments;
    h.n_cells = n;
    h.off_segs = L.off_segs;
    h.off_xs = L.off_xs;
    h.off_ys = L.off_ys;
    h.off_zs = L.off_zs;
    h.off_perm = L.off_perm;
    h.off_keys_in = L.off_keys_in;
    h.off_keys_out = L.off_keys_out;
    h.off_vals_in = L.off_vals_in;
    h.off_sort_tmp = L.off_sort_tmp;
    h.sort_tmp_bytes = L.sort_tmp_bytes;
    h.total_bytes = L.total;
    cudaError_t err = cudaMemcpyAsync(hdr, &h, sizeof(h), cudaMemcpyHostToDevice, st);
    if (err != cudaSuccess) return err;
    // cudaMemcpyAsync from pageable memory returns once the source is staged.
    SegInfo* hseg = new (std::nothrow) SegInfo[n_segments];
    if (!hseg) return cudaErrorMemoryAllocation;
    for (int s = 0; s < n_segments; ++s) {
        hseg[s] = SegInfo{};
        hseg[s].begin = seg_offsets_host[s];
        hseg[s].count = seg_offsets_host[s + 1] - seg_offsets_host[s];
    }
    err = cudaMemcpyAsync(segs, hseg, sizeof(SegInfo) * n_segments, cudaMemcpyHostToDevice, st);
    delete[] hseg;
    if (err != cudaSuccess) return err;

    seg_init_kernel<<<(n_segments + 127) / 128, 128, 0, st>>>(segs, n_segments);
    count_launches(1);
    if (n == 0) return cudaGetLastError();
    const int tpb = 256;
    const unsigned grid = static_cast<unsigned>((n + tpb - 1) / tpb);
    bbox_kernel<<<grid, tpb, 0, st>>>(x, y, z, dim, n, segs, n_segments, &hdr->status);
    brick_kernel<<<(n_segments + 127) / 128, 128, 0, st>>>(segs, n_segments, dim);
    key_kernel<<<grid, tpb, 0, st>>>(x, y, z, dim, n, segs, n_segments, keys_a, perm);
    count_launches(3);

    int key_bits = 30;
    if (n_segments > 1) {
        int sb = 0;
        while ((1 << sb) < n_segments) ++sb;
        key_bits += sb;
    } else {
        key_bits = dim * kMortonBits;
    }
    const int passes = (key_bits + 7) / 8;
    const int64_t nblk = sort_blocks(n);
    uint64_t* kin = keys_a;
    uint64_t* kout = keys_b;
    int32_t* vin = perm;
    int32_t* vout = vals_b;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        radix_hist_kernel<<<static_cast<unsigned>(nblk), kSortThreads, 0, st>>>(kin, n, shift, counts,
                                                                                  static_cast<int>(nblk));
        scan_kernel<<<1, 1024, 0, st>>>(counts, nblk * kRadix);
        radix_scatter_kernel<<<static_cast<unsigned>(nblk), kSortThreads, 0, st>>>(
            kin, vin, kout, vout, n, shift, counts, static_cast<int>(nblk));
        count_launches(3);
        uint64_t* tk = kin;
        kin = kout;
        kout = tk;
        int32_t* tv = vin;
        vin = vout;
        vout = tv;
    }
    if (vin != perm) {
        err = cudaMemcpyAsync(perm, vin, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st);
        if (err != cudaSuccess) return err;
    }
    gather_kernel<<<grid, tpb, 0, st>>>(x, y, z, dim, n, perm, xs, ys, zs);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace grf
