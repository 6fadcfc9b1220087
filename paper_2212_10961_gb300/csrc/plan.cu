// Cell plan: spatial binning of arbitrary cell centres.
//
// The paper evaluates Eq. (DiscreteFT) directly at the cell centres of an
// arbitrary (possibly unstructured) mesh (Sec. 4.1).  The synthesis kernels
// split each phase at a per-warp origin, which is accurate and cheap only when
// a warp's cells are close together.  The plan provides that locality:
//   1. bounding box of every segment (ordered-int atomics, warp-aggregated);
//   2. an isotropic quantisation grid along the longest axis, about one
//      level per four cell spacings of the largest segment (at most 2^10);
//   3. 32-bit keys, the segment index above the Morton code of the quantised
//      position, the first digit counted as they are made;
//   4. stable LSD radix sort of (key, original index) in the fewest passes
//      with digits of at most 10 bits;
//   5. gather of the sorted SoA coordinates.
// Everything runs on the stream without host synchronisation and is
// deterministic (the sort is stable, so equal keys keep the input order).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <new>

#include "device_common.cuh"

namespace grf {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 keys per block
constexpr int kMaxDigitBits = 10;  // radix passes use digits of up to 10 bits
constexpr int kMaxRadix = 1 << kMaxDigitBits;
static_assert(kMaxRadix % kSortThreads == 0, "digits are spread evenly over the threads");

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

// Bounding boxes: a block covers kBoxItems consecutive cells.  When they all
// belong to one segment (the usual case) the block reduces them first and
// issues one atomic per axis and bound; blocks that straddle a segment
// boundary fall back to per-thread atomics on change of segment.
constexpr int kBoxThreads = 256;
constexpr int kBoxItems = kBoxThreads * 16;

__device__ __forceinline__ void box_flush(SegInfo* segs, int seg, int dim, const int32_t (&lo)[3],
                                          const int32_t (&hi)[3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (k >= dim) break;
        atomicMin(reinterpret_cast<int32_t*>(segs[seg].lo) + k, lo[k]);
        atomicMax(reinterpret_cast<int32_t*>(segs[seg].hi) + k, hi[k]);
    }
}

__global__ void __launch_bounds__(kBoxThreads)
    bbox_kernel(const float* __restrict__ x, const float* __restrict__ y, const float* __restrict__ z,
                int dim, int64_t n, SegInfo* segs, int n_segments, int32_t* status) {
    __shared__ int32_t red_lo[kBoxThreads / 32][3];
    __shared__ int32_t red_hi[kBoxThreads / 32][3];
    const int64_t c0 = static_cast<int64_t>(blockIdx.x) * kBoxItems;
    const int64_t c1 = c0 + kBoxItems < n ? c0 + kBoxItems : n;
    const int s_first = find_segment(segs, n_segments, c0);
    const int s_last = find_segment(segs, n_segments, c1 - 1);
    const bool single = s_first == s_last;
    const float* src[3] = {x, y, z};
    int32_t lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
        lo[k] = float_to_ordered(INFINITY);
        hi[k] = float_to_ordered(-INFINITY);
    }
    int seg = s_first;
    int64_t seg_end = s_first + 1 < n_segments ? segs[s_first + 1].begin : n;
    bool bad = false;
    if (single) {
        // one segment: every coordinate load of the thread issued before its reductions
        constexpr int kPer = kBoxItems / kBoxThreads;
        float v[3][kPer];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                const int64_t i = c0 + threadIdx.x + static_cast<int64_t>(q) * kBoxThreads;
                v[k][q] = k < dim ? src[k][i < c1 ? i : c0] : 0.f;
            }
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                bad |= !isfinite(v[k][q]);
                const int32_t o = float_to_ordered(v[k][q]);
                lo[k] = min(lo[k], o);
                hi[k] = max(hi[k], o);
            }
    }
    for (int64_t i = c0 + threadIdx.x; !single && i < c1; i += kBoxThreads) {
        if (i >= seg_end) {
            box_flush(segs, seg, dim, lo, hi);
            for (int k = 0; k < 3; ++k) {
                lo[k] = float_to_ordered(INFINITY);
                hi[k] = float_to_ordered(-INFINITY);
            }
            seg = find_segment(segs, n_segments, i);
            seg_end = seg + 1 < n_segments ? segs[seg + 1].begin : n;
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (k >= dim) break;
            const float v = src[k][i];
            bad |= !isfinite(v);
            const int32_t o = float_to_ordered(v);
            lo[k] = min(lo[k], o);
            hi[k] = max(hi[k], o);
        }
    }
    if (bad) atomicOr(status, 1);
    if (!single) {
        box_flush(segs, seg, dim, lo, hi);
        return;
    }
    const int warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (k >= dim) break;
        for (int off = 16; off > 0; off >>= 1) {
            lo[k] = min(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], off));
            hi[k] = max(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], off));
        }
        if ((threadIdx.x & 31) == 0) {
            red_lo[warp][k] = lo[k];
            red_hi[warp][k] = hi[k];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kBoxThreads / 32; ++w)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                if (k >= dim) break;
                lo[k] = min(lo[k], red_lo[w][k]);
                hi[k] = max(hi[k], red_hi[w][k]);
            }
        box_flush(segs, s_first, dim, lo, hi);
    }
}

// Quantisation grid per segment: cubic cells of side L_max / 2^level_bits
// (L_max = largest bounding-box extent, level_bits <= kMortonBits chosen by
// the host from the largest segment's size), so that the Morton (Z-order) code
// of the quantised position orders cells along a space-filling curve and
// every aligned run of 2^k sorted cells is a compact, roughly cubic block.
__global__ void brick_kernel(SegInfo* segs, int n_segments, int dim, int level_bits) {
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
    const double levels = double(1 << level_bits);
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

// Quantisation grid of one segment, held in registers.
struct SegGrid {
    float lo[3], inv[3];
    int nb[3];
};
__device__ __forceinline__ SegGrid seg_grid(const SegInfo& g) {
    SegGrid r;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        r.lo[k] = g.lo[k];
        r.inv[k] = g.inv_brick[k];
        r.nb[k] = g.nb[k];
    }
    return r;
}

// spread[b] = the 10 bits of b moved to every dim-th bit (shared-memory table)
__device__ __forceinline__ uint32_t morton_code(const float (&v)[3], const SegGrid& g, int dim,
                                                const uint32_t* spread) {
    uint32_t code = 0u;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (k >= dim) break;
        const float f = (v[k] - g.lo[k]) * g.inv[k];
        int q = isfinite(f) ? static_cast<int>(floorf(f)) : 0;
        q = q < 0 ? 0 : (q >= g.nb[k] ? g.nb[k] - 1 : q);
        code |= spread[q] << k;
    }
    return code;
}

// Sort keys (segment index above the Morton code), one sort tile per block,
// fused with the digit-0 histogram of the tile (the first radix pass needs no
// separate counting kernel).  The values of the first pass are the input
// indices themselves, so none are stored here.
__global__ void __launch_bounds__(kSortThreads)
    key_kernel(const float* __restrict__ x, const float* __restrict__ y, const float* __restrict__ z,
               int dim, int64_t n, const SegInfo* __restrict__ segs, int n_segments,
               uint32_t* __restrict__ keys, int morton_bits, int digit_bits, uint32_t* __restrict__ counts,
               int nblk) {
    __shared__ uint32_t hist[kMaxRadix];
    __shared__ uint32_t spread[1 << kMortonBits];
    const int radix = 1 << digit_bits;
    const uint32_t mask = static_cast<uint32_t>(radix - 1);
    for (int d = threadIdx.x; d < radix; d += blockDim.x) hist[d] = 0u;
    for (int b = threadIdx.x; b < (1 << kMortonBits); b += blockDim.x)
        spread[b] = dim == 3 ? spread_bits3(b) : (dim == 2 ? spread_bits2(b) : static_cast<uint32_t>(b));
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kSortTile;
    const int64_t c1 = base + kSortTile < n ? base + kSortTile : n;
    const int s_first = find_segment(segs, n_segments, base);
    const bool single = s_first == find_segment(segs, n_segments, c1 - 1);
    const SegGrid g_first = seg_grid(segs[s_first]);
    __syncthreads();
    constexpr int kGroup = 8;  // cells whose loads are in flight together
#pragma unroll 1
    for (int r0 = 0; r0 < kSortItems; r0 += kGroup) {
        float v[kGroup][3];
#pragma unroll
        for (int r = 0; r < kGroup; ++r) {
            const int64_t i = base + (r0 + r) * kSortThreads + threadIdx.x;
            const int64_t j = i < n ? i : base;
            v[r][0] = x[j];
            v[r][1] = dim > 1 ? y[j] : 0.f;
            v[r][2] = dim > 2 ? z[j] : 0.f;
        }
#pragma unroll
        for (int r = 0; r < kGroup; ++r) {
            const int64_t i = base + (r0 + r) * kSortThreads + threadIdx.x;
            if (i >= n) continue;
            uint32_t key;
            if (single) {
                key = (static_cast<uint32_t>(s_first) << morton_bits) | morton_code(v[r], g_first, dim, spread);
            } else {
                const int s = find_segment(segs, n_segments, i);
                key = (static_cast<uint32_t>(s) << morton_bits) | morton_code(v[r], seg_grid(segs[s]), dim, spread);
            }
            keys[i] = key;
            atomicAdd(&hist[key & mask], 1u);
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < radix; d += blockDim.x)
        counts[static_cast<int64_t>(d) * nblk + blockIdx.x] = hist[d];
}

// ---- stable LSD radix sort, digits of up to kMaxDigitBits bits ---------------------

__global__ void __launch_bounds__(kSortThreads)
    radix_hist_kernel(const uint32_t* __restrict__ keys, int64_t n, int shift, int digit_bits,
                      uint32_t* __restrict__ counts, int nblk) {
    __shared__ uint32_t hist[kMaxRadix];
    const int radix = 1 << digit_bits;
    const uint32_t mask = static_cast<uint32_t>(radix - 1);
    for (int d = threadIdx.x; d < radix; d += blockDim.x) hist[d] = 0u;
    __syncthreads();
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kSortTile;
    uint32_t k[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {  // loads first, all in flight together
        const int64_t i = base + r * kSortThreads + threadIdx.x;
        k[r] = i < n ? keys[i] : uint32_t(0);
    }
#pragma unroll
    for (int r = 0; r < kSortItems; ++r)
        if (base + r * kSortThreads + threadIdx.x < n)
            atomicAdd(&hist[(k[r] >> shift) & mask], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < radix; d += blockDim.x)
        counts[static_cast<int64_t>(d) * nblk + blockIdx.x] = hist[d];
}

// Exclusive scan over the block of one value per thread (kSortThreads
// threads), also returning the block total; `warp_tot` is kSortThreads / 32
// words of shared scratch.  Contains block barriers.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_tot, uint32_t& total) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    uint32_t before = 0u;
    total = 0u;
#pragma unroll
    for (int w = 0; w < kSortThreads / 32; ++w) {
        const uint32_t t = warp_tot[w];
        before += w < warp ? t : 0u;
        total += t;
    }
    __syncthreads();  // warp_tot may be reused after the return
    return before + incl - v;
}

// Exclusive scan of each digit's row of per-block counts, one block per
// digit (rows are counts[d * nblk .. (d + 1) * nblk)), plus the row total.
// The row goes through shared memory in chunks of 4096 so that the global
// loads and stores are coalesced while each thread scans 16 consecutive
// counts.
constexpr int kScanThreads = kSortThreads;
constexpr int kScanPer = 16;
constexpr int kScanChunk = kScanThreads * kScanPer;
__global__ void __launch_bounds__(kScanThreads)
    scan_rows_kernel(uint32_t* __restrict__ counts, int nblk, uint32_t* __restrict__ totals) {
    __shared__ uint32_t buf[kScanChunk + kScanChunk / 32];  // one pad word per 32
    __shared__ uint32_t warp_tot[kScanThreads / 32];
    uint32_t* row = counts + static_cast<int64_t>(blockIdx.x) * nblk;
    const auto at = [](int k) { return k + (k >> 5); };
    uint32_t carry = 0u;
    for (int c0 = 0; c0 < nblk; c0 += kScanChunk) {
        const int m = nblk - c0 < kScanChunk ? nblk - c0 : kScanChunk;
        for (int k = threadIdx.x; k < kScanChunk; k += kScanThreads) buf[at(k)] = k < m ? row[c0 + k] : 0u;
        __syncthreads();
        uint32_t v[kScanPer];
        uint32_t sum = 0u;
#pragma unroll
        for (int q = 0; q < kScanPer; ++q) {
            v[q] = buf[at(threadIdx.x * kScanPer + q)];
            sum += v[q];
        }
        uint32_t chunk = 0u;
        uint32_t run = carry + block_exclusive_scan(sum, warp_tot, chunk);
#pragma unroll
        for (int q = 0; q < kScanPer; ++q) {
            buf[at(threadIdx.x * kScanPer + q)] = run;
            run += v[q];
        }
        __syncthreads();
        for (int k = threadIdx.x; k < m; k += kScanThreads) row[c0 + k] = buf[at(k)];
        __syncthreads();  // buf is refilled by the next chunk
        carry += chunk;
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

// Stable scatter.  Warp w owns items [512 w, 512 (w + 1)) of the tile, in
// 16 rounds of 32 consecutive items, so (warp, round, lane) is the input
// order.  Each warp ranks its items per digit on its own (match_any within a
// round, all rounds' matches issued first; a warp-private running count
// across rounds, advanced by one shared atomic per digit group); one block barrier then
// turns the per-warp counts into offsets, and every item is stored at the
// digit's global start + its warp's offset + its rank within the warp.
// kFirst: the values are the input indices (nothing to read); kLast: only
// the values are stored.
template <bool kFirst, bool kLast>
__global__ void __launch_bounds__(kSortThreads, kFirst ? 3 : 2)
    radix_scatter_kernel(const uint32_t* __restrict__ keys_in, const int32_t* __restrict__ vals_in,
                         uint32_t* __restrict__ keys_out, int32_t* __restrict__ vals_out,
                         int64_t n64, int shift, int digit_bits, const uint32_t* __restrict__ offsets,
                         const uint32_t* __restrict__ totals, int nblk) {
    constexpr int kWarps = kSortThreads / 32;
    constexpr int kRounds = kSortTile / kSortThreads;  // rounds of 32 items per warp
    static_assert(kRounds % 2 == 0 && kRounds * 32 <= 65536, "ranks are packed two per register");
    __shared__ uint32_t warp_cnt[kWarps][kMaxRadix];  // per-warp digit counts, then offsets
    __shared__ uint32_t digit_start[kMaxRadix];       // global start of each digit for this tile
    __shared__ uint32_t warp_tot[kWarps];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int radix = 1 << digit_bits;
    const uint32_t mask = static_cast<uint32_t>(radix - 1);
    // plans hold at most 2^31 - 1 cells, so item indices fit in 32 bits
    const uint32_t n = static_cast<uint32_t>(n64);
    const uint32_t i0 = blockIdx.x * static_cast<uint32_t>(kSortTile) + warp * (kRounds * 32) + lane;
    uint32_t key[kRounds];
    int32_t val[kFirst ? 1 : kRounds];
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {  // loads first, all in flight together
        const uint32_t i = i0 + r * 32;
        key[r] = i < n ? keys_in[i] : 0u;
        if (!kFirst) val[r] = i < n ? vals_in[i] : 0;
    }
    for (int w = 0; w < kWarps; ++w)
        for (int d = threadIdx.x; d < radix; d += kSortThreads) warp_cnt[w][d] = 0u;
    // digit starts: exclusive scan of the digit totals in slabs of kSortThreads
    // digits (the slab loop is uniform over the block)
    {
        uint32_t carry = 0u;
        for (int d0 = 0; d0 < radix; d0 += kSortThreads) {
            const int d = d0 + threadIdx.x;
            const uint32_t t = d < radix ? totals[d] : 0u;
            uint32_t slab = 0u;
            const uint32_t ex = block_exclusive_scan(t, warp_tot, slab);
            if (d < radix) digit_start[d] = carry + ex + offsets[static_cast<int64_t>(d) * nblk + blockIdx.x];
            carry += slab;
        }
    }
    const unsigned lt_mask = (1u << lane) - 1u;
    uint32_t loc[kRounds / 2];  // rank of each item among its warp's items of the same digit
    unsigned peer[kRounds];
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {  // the rounds' matches are independent: all in flight
        const bool in = i0 + r * 32 < n;
        // out-of-range items get a digit of their own (never counted or stored)
        const int digit = in ? static_cast<int>((key[r] >> shift) & mask) : kMaxRadix;
        peer[r] = __match_any_sync(0xffffffffu, digit);
    }
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const bool in = i0 + r * 32 < n;
        const unsigned peers = peer[r];
        const int leader = __ffs(peers) - 1;
        uint32_t before = 0u;
        if (lane == leader && in)
            before = atomicAdd(&warp_cnt[warp][(key[r] >> shift) & mask], static_cast<uint32_t>(__popc(peers)));
        before = __shfl_sync(0xffffffffu, before, leader);
        const uint32_t rank = before + static_cast<uint32_t>(__popc(peers & lt_mask));
        if (r % 2 == 0)
            loc[r / 2] = rank;
        else
            loc[r / 2] |= rank << 16;
        __syncwarp();  // this round's counts are visible to the next round's leaders
    }
    __syncthreads();
    for (int d = threadIdx.x; d < radix; d += kSortThreads) {
        uint32_t run = digit_start[d];
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t c = warp_cnt[w][d];
            warp_cnt[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const uint32_t i = i0 + r * 32;
        if (i >= n) continue;
        const uint32_t rank = r % 2 == 0 ? (loc[r / 2] & 0xffffu) : (loc[r / 2] >> 16);
        const uint32_t pos = warp_cnt[warp][(key[r] >> shift) & mask] + rank;
        if (!index_ok(pos, n)) continue;
        if (!kLast) keys_out[pos] = key[r];
        vals_out[pos] = kFirst ? static_cast<int32_t>(i) : val[r];
    }
}

// Sorted coordinates: four cells per thread, index and coordinate loads
// issued before the stores.
constexpr int kGatherPer = 4;
__global__ void gather_kernel(const float* __restrict__ x, const float* __restrict__ y,
                              const float* __restrict__ z, int dim, int64_t n,
                              const int32_t* __restrict__ perm, float* __restrict__ xs,
                              float* __restrict__ ys, float* __restrict__ zs) {
    const int64_t i0 = static_cast<int64_t>(blockIdx.x) * blockDim.x * kGatherPer + threadIdx.x;
    int64_t o[kGatherPer];
#pragma unroll
    for (int q = 0; q < kGatherPer; ++q) {
        const int64_t i = i0 + static_cast<int64_t>(q) * blockDim.x;
        o[q] = i < n ? perm[i] : 0;
        if (!index_ok(o[q], n)) o[q] = 0;  // checked builds: read a valid cell instead
    }
    float v[kGatherPer][3];
#pragma unroll
    for (int q = 0; q < kGatherPer; ++q) {
        v[q][0] = x[o[q]];
        v[q][1] = dim > 1 ? y[o[q]] : 0.f;
        v[q][2] = dim > 2 ? z[o[q]] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < kGatherPer; ++q) {
        const int64_t i = i0 + static_cast<int64_t>(q) * blockDim.x;
        if (i >= n) continue;
        xs[i] = v[q][0];
        if (dim > 1) ys[i] = v[q][1];
        if (dim > 2) zs[i] = v[q][2];
    }
}

int64_t sort_blocks(int64_t n) { return (n + kSortTile - 1) / kSortTile; }

}  // namespace

size_t radix_sort_temp_bytes(int64_t n_cells) {
    return static_cast<size_t>(sort_blocks(n_cells) + 1) * kMaxRadix * sizeof(uint32_t);
}

namespace {

// Keys of the sort tiles (first digit counted on the fly), then one
// histogram / scan / scatter triple per further digit.  The index array
// ping-pongs between vals_b and perm so that the last pass writes perm.
void run_sort(const float* x, const float* y, const float* z, int dim, int64_t n, const SegInfo* segs,
              int n_segments, int morton_bits, int passes, int digit_bits, int64_t nblk, uint32_t* keys_a,
              uint32_t* keys_b, int32_t* vals_b, int32_t* perm, uint32_t* counts, uint32_t* totals,
              cudaStream_t st) {
    uint32_t* kin = keys_a;
    uint32_t* kout = keys_b;
    const unsigned grid = static_cast<unsigned>(nblk);
    const int nb = static_cast<int>(nblk);
    key_kernel<<<grid, kSortThreads, 0, st>>>(x, y, z, dim, n, segs, n_segments, kin, morton_bits, digit_bits,
                                              counts, nb);
    count_launches(1);
    const int32_t* vin = nullptr;
    for (int p = 0; p < passes; ++p) {
        const int shift = digit_bits * p;
        if (p > 0) {
            radix_hist_kernel<<<grid, kSortThreads, 0, st>>>(kin, n, shift, digit_bits, counts, nb);
            count_launches(1);
        }
        scan_rows_kernel<<<1u << digit_bits, kScanThreads, 0, st>>>(counts, nb, totals);
        int32_t* vout = (passes - 1 - p) % 2 == 0 ? perm : vals_b;
        const bool first = p == 0, last = p == passes - 1;
        if (first && last)
            radix_scatter_kernel<true, true><<<grid, kSortThreads, 0, st>>>(kin, vin, kout, vout, n, shift,
                                                                            digit_bits, counts, totals, nb);
        else if (first)
            radix_scatter_kernel<true, false><<<grid, kSortThreads, 0, st>>>(kin, vin, kout, vout, n, shift,
                                                                             digit_bits, counts, totals, nb);
        else if (last)
            radix_scatter_kernel<false, true><<<grid, kSortThreads, 0, st>>>(kin, vin, kout, vout, n, shift,
                                                                             digit_bits, counts, totals, nb);
        else
            radix_scatter_kernel<false, false><<<grid, kSortThreads, 0, st>>>(kin, vin, kout, vout, n, shift,
                                                                              digit_bits, counts, totals, nb);
        count_launches(2);
        uint32_t* tk = kin;
        kin = kout;
        kout = tk;
        vin = vout;
    }
}

// ---- Cartesian-grid check of a single-segment plan --------------------------
// Cells given x-fastest on the tensor product of three axes, cell
// n = i + nx (k + ny l) at (X_i, Y_k, Z_l), let the synthesis use the tensor-
// core grid path.  Pass 1 finds nx (the first cell whose (y, z) differs from
// cell 0's) and nx ny (the first whose z differs); pass 2 checks every cell
// against those axes and writes X, Y, Z.  The host reads the result later.
constexpr int kGridThreads = 256;
constexpr int kGridPer = 16;

__device__ __forceinline__ unsigned long long block_min_u64(unsigned long long v, unsigned long long* red) {
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, off);
        v = o < v ? o : v;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < kGridThreads / 32; ++w) v = red[w] < v ? red[w] : v;
    return v;  // valid in thread 0
}

__global__ void __launch_bounds__(kGridThreads) grid_scan_kernel(const float* y, const float* z, int32_t dim,
                                                                 int64_t n, GridCheck* gc) {
    __shared__ unsigned long long red1[kGridThreads / 32], red2[kGridThreads / 32];
    const int64_t base = static_cast<int64_t>(blockIdx.x) * (kGridThreads * kGridPer);
    // blocks past the current candidates cannot lower them
    const unsigned long long lim =
        dim > 2 ? *reinterpret_cast<volatile unsigned long long*>(&gc->c2)
                : *reinterpret_cast<volatile unsigned long long*>(&gc->c1);
    if (static_cast<unsigned long long>(base) >= lim) return;
    const float y0 = __ldg(y);
    const float z0 = dim > 2 ? __ldg(z) : 0.0f;
    unsigned long long m1 = ~0ull, m2 = ~0ull;
#pragma unroll 4
    for (int q = 0; q < kGridPer; ++q) {
        const int64_t i = base + static_cast<int64_t>(q) * kGridThreads + threadIdx.x;
        if (i >= 1 && i < n) {
            const bool zd = dim > 2 && __ldg(z + i) != z0;
            if (zd || __ldg(y + i) != y0) m1 = m1 < static_cast<unsigned long long>(i) ? m1 : i;
            if (zd) m2 = m2 < static_cast<unsigned long long>(i) ? m2 : i;
        }
    }
    m1 = block_min_u64(m1, red1);
    m2 = block_min_u64(m2, red2);
    if (threadIdx.x == 0) {
        if (m1 != ~0ull) atomicMin(&gc->c1, m1);
        if (m2 != ~0ull) atomicMin(&gc->c2, m2);
    }
}

__global__ void __launch_bounds__(kGridThreads) grid_verify_kernel(const float* x, const float* y, const float* z,
                                                                   int32_t dim, int64_t n, GridCheck* gc,
                                                                   float* axes) {
    const int64_t nx = static_cast<int64_t>(gc->c1);
    const int64_t nxy = dim > 2 ? static_cast<int64_t>(gc->c2) : n;
    // a shape that is not a tensor product is rejected on the host
    if (nx < 1 || nxy < nx || nxy % nx != 0 || n % nxy != 0) return;
    const int64_t ny = nxy / nx, nz = n / nxy;
    const bool room = nx + ny + nz <= n;  // the axes go over the keys scratch (n floats)
    bool ok = true;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t ix = i % nx;
        const int64_t r = i / nx;
        const int64_t k = r % ny;
        const int64_t l = r / ny;
        const float xv = __ldg(x + i), yv = __ldg(y + i);
        const float zv = dim > 2 ? __ldg(z + i) : 0.0f;
        ok = ok && xv == __ldg(x + ix) && yv == __ldg(y + k * nx);
        if (dim > 2) ok = ok && zv == __ldg(z + l * nxy);
        if (room) {
            if (i < nx) axes[i] = xv;
            if (ix == 0 && l == 0) axes[nx + k] = yv;
            if (ix == 0 && k == 0) axes[nx + ny + l] = zv;
        }
    }
    if (!__all_sync(0xffffffffu, ok) && (threadIdx.x & 31) == 0) atomicOr(&gc->bad, 1);
}

}  // namespace

int launch_grid_check(int32_t dim, int64_t n, const float* x, const float* y, const float* z, void* plan,
                      const PlanLayout& L, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* base = static_cast<unsigned char*>(plan);
    GridCheck* gc = &reinterpret_cast<PlanHeader*>(base)->grid;
    float* axes = reinterpret_cast<float*>(base + L.off_keys_in);
    const int64_t per = int64_t(kGridThreads) * kGridPer;
    grid_scan_kernel<<<static_cast<unsigned>((n + per - 1) / per), kGridThreads, 0, st>>>(y, z, dim, n, gc);
    const int64_t vb = std::min<int64_t>((n + kGridThreads - 1) / kGridThreads, 152 * 16);
    grid_verify_kernel<<<static_cast<unsigned>(vb), kGridThreads, 0, st>>>(x, y, z, dim, n, gc, axes);
    count_launches(2);
    return cudaGetLastError();
}

int launch_plan(int32_t dim, int32_t n_segments, const int64_t* seg_offsets_host, const float* x,
                const float* y, const float* z, void* plan, const PlanLayout& L, uint64_t tag, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* base = static_cast<unsigned char*>(plan);
    const int64_t n = seg_offsets_host[n_segments];
    PlanHeader* hdr = reinterpret_cast<PlanHeader*>(base);
    SegInfo* segs = reinterpret_cast<SegInfo*>(base + L.off_segs);
    float* xs = reinterpret_cast<float*>(base + L.off_xs);
    float* ys = reinterpret_cast<float*>(base + L.off_ys);
    float* zs = reinterpret_cast<float*>(base + L.off_zs);
    int32_t* perm = reinterpret_cast<int32_t*>(base + L.off_perm);
    uint32_t* keys_a = reinterpret_cast<uint32_t*>(base + L.off_keys_in);
    uint32_t* keys_b = reinterpret_cast<uint32_t*>(base + L.off_keys_out);
    int32_t* vals_b = reinterpret_cast<int32_t*>(base + L.off_vals_in);
    uint32_t* counts = reinterpret_cast<uint32_t*>(base + L.off_sort_tmp);
    uint32_t* totals = counts + sort_blocks(n) * kMaxRadix;  // digit totals

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
    h.grid.c1 = static_cast<unsigned long long>(n);
    h.grid.c2 = static_cast<unsigned long long>(n);
    h.grid.bad = (n_segments == 1 && dim >= 2 && n >= 4) ? 0 : 1;
    h.grid.tag = tag;
    cudaError_t err = cudaMemcpyAsync(hdr, &h, sizeof(h), cudaMemcpyHostToDevice, st);
    if (err != cudaSuccess) return err;
    // cudaMemcpyAsync from pageable memory returns once the source is staged.
    alloc_point();
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
    bbox_kernel<<<static_cast<unsigned>((n + kBoxItems - 1) / kBoxItems), kBoxThreads, 0, st>>>(
        x, y, z, dim, n, segs, n_segments, &hdr->status);
    count_launches(1);
    // Quantisation levels along the longest axis: about one level per four
    // cell spacings of the largest segment (n^(1/dim) / 4 rounded up to a
    // power of two, 16 .. 2^kMortonBits), so that no sort pass is spent on
    // key bits finer than a lane's group of cells; cells that share a level
    // keep their input order (the sort is stable).
    int64_t n_max = 0;
    for (int s = 0; s < n_segments; ++s) {
        const int64_t c = seg_offsets_host[s + 1] - seg_offsets_host[s];
        if (c > n_max) n_max = c;
    }
    int level_bits = 4;
    while (level_bits < kMortonBits &&
           std::pow(2.0, static_cast<double>(level_bits * dim)) * std::pow(4.0, dim) < static_cast<double>(n_max))
        ++level_bits;
    // 32-bit keys: with very many segments (more than 2^(32 - 4 dim)) the
    // grid is made coarser so that the segment index still fits above it.
    int sb = 0;
    while ((int64_t(1) << sb) < n_segments) ++sb;
    if (level_bits * dim + sb > 32) level_bits = (32 - sb) / dim;
    const int morton_bits = dim * level_bits;
    const int key_bits = morton_bits + sb;
    // fewest passes with digits of at most kMaxDigitBits bits, the bits spread
    // evenly over them (18-bit keys: two passes of 9 bits)
    const int passes = key_bits > kMaxDigitBits ? (key_bits + kMaxDigitBits - 1) / kMaxDigitBits : 1;
    const int digit_bits = key_bits > 0 ? (key_bits + passes - 1) / passes : 1;
    const int64_t nblk = sort_blocks(n);
    brick_kernel<<<(n_segments + 127) / 128, 128, 0, st>>>(segs, n_segments, dim, level_bits);
    count_launches(1);
    run_sort(x, y, z, dim, n, segs, n_segments, morton_bits, passes, digit_bits, nblk, keys_a, keys_b, vals_b,
             perm, counts, totals, st);
    const int gtpb = 256;
    const unsigned ggrid = static_cast<unsigned>((n + gtpb * kGatherPer - 1) / (gtpb * kGatherPer));
    gather_kernel<<<ggrid, gtpb, 0, st>>>(x, y, z, dim, n, perm, xs, ys, zs);
    count_launches(1);
    if (n_segments == 1 && dim >= 2 && n >= 4) {
        const int e = launch_grid_check(dim, n, x, y, z, plan, L, st);
        if (e != cudaSuccess) return static_cast<cudaError_t>(e);
    }
    return cudaGetLastError();
}

unsigned long long take_index_faults_plan() { return take_tu_index_faults(); }

}  // namespace grf
