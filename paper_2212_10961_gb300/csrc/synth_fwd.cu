// Forward synthesis kernel: Y_i = mu + sum_j A_j cos(2 pi (a_j . x_i + psi_j))
// at arbitrary cell centres (Icardi et al., arXiv 2212.10961, Sec. 4.1,
// Eq. DiscreteFT), with the property maps of Sec. 3.1 / Sec. 4.1 fused into
// the epilogue.
//
// Work decomposition.  Cells arrive spatially sorted (cell plan).  A warp owns
// 32*C consecutive sorted cells (C per lane, in registers) and takes the
// midpoint of their bounding box as its origin x0, with half-extent E.  The
// phase of mode j at cell i is split as
//     theta_ij = 2 pi (a_j . x0 + psi_j  mod 1)  +  (2 pi a_j) . (x_i - x0),
// the first term computed once per (warp, mode) in compensated FP32
// (phase_exact_turns), the second per cell-mode with three FFMAs.  Modes whose
// phase span over the warp, |a_j|_1 * E, exceeds tau turns (a prefix of the
// table, which is sorted by |a_j|_1) take the exact per-cell path instead.
// The hot loop is one MUFU cosine, one FMUL (radian scaling inside
// cos.approx), DIM FFMAs for the phase and one FFMA to accumulate.
//
// Mode chunks (kChunk modes, 48 B each) are staged in shared memory by 1-D
// bulk copies into two buffers completed on mbarriers; every wait is bounded
// and reports GRF_ETIMEOUT through the status word instead of hanging.
// Per-chunk FP32 partials are folded into a TwoSum-compensated accumulator.
#include <cuda_runtime.h>

#include "device_common.cuh"

namespace grf {

namespace {

constexpr int kChunkBytes = kChunk * 48;  // hot (16 B) + cold (32 B) per mode
constexpr int kMaxSplit = 8;              // most mode splits of one launch

template <int C, int W>
struct FwdSmem {
    float4 buf[2][kChunk * 3];  // [hot kChunk][cold 2*kChunk]
    float t0[W][kChunk];        // per-warp origin phase (radians)
    uint64_t full[2];
    int32_t abort_flag;
    int32_t work;               // batched: current work index
    FwdDesc desc;               // batched: current descriptor
};

// Issue the bulk copies of chunk `ch` of descriptor d into buffer `bi`.
__device__ __forceinline__ void issue_chunk(const FwdDesc& d, int ch, float4* dst, uint64_t* bar) {
    mbar_arrive_expect_tx(bar, kChunkBytes);
    bulk_g2s(dst, d.hot + static_cast<int64_t>(ch) * kChunk, kChunk * 16, bar);
    bulk_g2s(dst + kChunk, d.cold + static_cast<int64_t>(ch) * kChunk * 2, kChunk * 32, bar);
}

// Conservative extent bucket: smallest b with 2^((b - bias)/4) >= E (one
// extra step covers the approximate log2).  kpref[b] counts the modes with
// |a_j|_1 * 2^((b - bias)/4) > 1, so querying with E / tau gives the modes
// whose phase span over a box of half-extent E exceeds tau turns.
__device__ __forceinline__ int prefix_for(const int32_t* kpref, int n_pad, float E_over_tau) {
    if (!(E_over_tau > 0.0f)) return 0;
    const int b = static_cast<int>(ceilf(4.0f * __log2f(E_over_tau))) + kBucketBias + 1;
    if (b >= kBuckets) return n_pad;
    return b < 0 ? 0 : __ldg(kpref + b);
}

// Warp-wide min / max.
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

// One tile: W warps x 32 lanes x C cells starting at sorted cell `tile_base`.
// Lane l of a warp owns the C consecutive sorted cells wbase + C l + c, a
// compact block of the Z-order (2x2x2 for C = 8).  Three classes of modes,
// all prefixes of the table (sorted by |a|_1, descending):
//   super  : span over the lane's block > tau2 turns -> exact phase per cell;
//   medium : span over the warp's block > tau1 turns -> exact phase at the
//            lane origin xt once per (lane, mode), FP32 offsets per cell;
//   light  : the rest -> exact phase at the warp origin x0 once per
//            (warp, mode), FP32 offsets per cell (the hot loop).
// `uses` counts completed waits per buffer (parity tracking across tiles).
template <int DIM, int C, int W>
__device__ __forceinline__ void synth_tile(const FwdDesc& d, int64_t tile_base, int cb, int ce,
                                           float2* partial, FwdSmem<C, W>& sm, uint32_t (&uses)[2],
                                           int32_t* status) {
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t n = d.n_cells;
    const int64_t wbase = tile_base + static_cast<int64_t>(warp) * 32 * C;
    const bool warp_active = wbase < n;
    // this block's modes: chunks [cb, ce) of the table (the whole table unless
    // the modes are split over blocks, see synth_split_finalize)
    const int jlo = cb * kChunk;
    const int jhi = ce * kChunk;

    // Prefetch the first two chunks (previous tile's buffers are free: the
    // tile ended with a block barrier).
    if (threadIdx.x == 0) {
        fence_proxy_async_smem();
        issue_chunk(d, cb, sm.buf[0], &sm.full[0]);
        if (cb + 1 < ce) issue_chunk(d, cb + 1, sm.buf[1], &sm.full[1]);
    }

    // ---- load cells (lane-contiguous), bounding boxes, origins ------------
    const int64_t lbase = wbase + static_cast<int64_t>(lane) * C;
    float x[C][DIM];
    bool valid[C];
    {
        const float* src[3] = {d.xs, d.ys, d.zs};
        const int64_t safe = warp_active ? wbase : 0;  // a valid cell of this warp
#pragma unroll
        for (int c = 0; c < C; ++c) valid[c] = lbase + c < n;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            // vector loads only when all C cells exist and the address is
            // 16-byte aligned (a segment may start at any cell index)
            const bool vec = (C % 4) == 0 && lbase + C <= n &&
                             (reinterpret_cast<uintptr_t>(src[k] + lbase) & 15u) == 0;
            if (vec) {
#pragma unroll
                for (int q = 0; q < C / 4; ++q) {
                    const float4 v = __ldg(reinterpret_cast<const float4*>(src[k] + lbase) + q);
                    x[4 * q + 0][k] = v.x;
                    x[4 * q + 1][k] = v.y;
                    x[4 * q + 2][k] = v.z;
                    x[4 * q + 3][k] = v.w;
                }
            } else {
                // ragged tail: invalid cells repeat the lane's first valid cell
                // (or the warp's first cell) so that bounding boxes are unaffected
                const int64_t first = lbase < n ? lbase : safe;
#pragma unroll
                for (int c = 0; c < C; ++c) x[c][k] = __ldg(src[k] + (valid[c] ? lbase + c : first));
            }
        }
    }
    float x0[DIM], xt[DIM];
    float Ew = 0.0f, Et = 0.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        float mn = x[0][k], mx = x[0][k];
#pragma unroll
        for (int c = 1; c < C; ++c) {
            mn = fminf(mn, x[c][k]);
            mx = fmaxf(mx, x[c][k]);
        }
        xt[k] = 0.5f * mn + 0.5f * mx;
        Et = fmaxf(Et, fmaxf(mx - xt[k], xt[k] - mn));
        mn = warp_min(mn);
        mx = warp_max(mx);
        x0[k] = 0.5f * mn + 0.5f * mx;
        Ew = fmaxf(Ew, fmaxf(mx - x0[k], x0[k] - mn));
    }
    Et = warp_max(Et);
    int k_med = 0, k_sup = 0;
    if (warp_active) {
        k_med = prefix_for(d.kpref, d.n_pad, Ew * d.inv_tau1);
        k_sup = min(k_med, prefix_for(d.kpref, d.n_pad, Et * d.inv_tau2));
    }

    float s[C], e[C], p[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        s[c] = 0.0f;
        e[c] = 0.0f;
        p[c] = 0.0f;
    }

    // ---- super class: exact phase at every cell ---------------------------------
    const int sup_end = min(k_sup, jhi);
    for (int j = jlo; j < sup_end; ++j) {
        const float4 c0 = __ldg(d.cold + 2 * j);
        const float4 c1 = __ldg(d.cold + 2 * j + 1);
        const float A = __ldg(&d.hot[j].w);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float r = phase_exact_turns<DIM>(x[c], c0, c1);
            p[c] = fmaf(A, hw_cos(kTwoPiF * r), p[c]);
        }
        if ((j & 63) == 63) {
#pragma unroll
            for (int c = 0; c < C; ++c) {
                two_sum_acc(s[c], e[c], p[c]);
                p[c] = 0.0f;
            }
        }
    }

    // ---- medium class: exact phase at the lane origin -------------------------
    float dx[C][DIM];  // offsets from the lane origin, then from the warp origin
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
        for (int k = 0; k < DIM; ++k) dx[c][k] = x[c][k] - xt[k];
    const int med_end = min(k_med, jhi);
    for (int j = max(k_sup, jlo); j < med_end; ++j) {
        const float4 c0 = __ldg(d.cold + 2 * j);
        const float4 c1 = __ldg(d.cold + 2 * j + 1);
        const float4 h = __ldg(d.hot + j);
        const float t0 = kTwoPiF * phase_exact_turns<DIM>(xt, c0, c1);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            float th = fmaf(h.x, dx[c][0], t0);
            if (DIM > 1) th = fmaf(h.y, dx[c][1], th);
            if (DIM > 2) th = fmaf(h.z, dx[c][2], th);
            p[c] = fmaf(h.w, hw_cos(th), p[c]);
        }
        if (((j - k_sup) & 63) == 63) {
#pragma unroll
            for (int c = 0; c < C; ++c) {
                two_sum_acc(s[c], e[c], p[c]);
                p[c] = 0.0f;
            }
        }
    }
    // re-base the offsets on the warp origin: dx = (x - xt) + (xt - x0)
    {
        float D[DIM];
#pragma unroll
        for (int k = 0; k < DIM; ++k) D[k] = xt[k] - x0[k];
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int k = 0; k < DIM; ++k) dx[c][k] += D[k];
    }

    // ---- light class over staged chunks ------------------------------------------
    int ch = cb;
    for (; ch < ce; ++ch) {
        const int bi = (ch - cb) & 1;
        const uint32_t parity = uses[bi] & 1u;
        bool ok = mbar_wait_bounded(&sm.full[bi], parity);
        if (!ok) {
            sm.abort_flag = 1;
            atomicOr(status, 2);
        }
        uses[bi] += 1;
        const float4* hotS = sm.buf[bi];
        const float4* coldS = sm.buf[bi] + kChunk;
        float* t0S = sm.t0[warp];
        const int jbase = ch * kChunk;
        if (ok && warp_active && jbase + kChunk > k_med) {
            const int m0 = k_med > jbase ? k_med - jbase : 0;
            for (int m = m0 + lane; m < kChunk; m += 32)
                t0S[m] = kTwoPiF * phase_exact_turns<DIM>(x0, coldS[2 * m], coldS[2 * m + 1]);
            __syncwarp();
#pragma unroll 4
            for (int m = m0; m < kChunk; ++m) {
                const float4 h = hotS[m];
                const float t0 = t0S[m];
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    float th = fmaf(h.x, dx[c][0], t0);
                    if (DIM > 1) th = fmaf(h.y, dx[c][1], th);
                    if (DIM > 2) th = fmaf(h.z, dx[c][2], th);
                    p[c] = fmaf(h.w, hw_cos(th), p[c]);
                }
            }
#pragma unroll
            for (int c = 0; c < C; ++c) {
                two_sum_acc(s[c], e[c], p[c]);
                p[c] = 0.0f;
            }
        }
        __syncthreads();
        if (sm.abort_flag) break;
        if (threadIdx.x == 0 && ch + 2 < ce) {
            fence_proxy_async_smem();
            issue_chunk(d, ch + 2, sm.buf[bi], &sm.full[bi]);
        }
    }
    if (sm.abort_flag) {
        // Give the copies still in flight (chunks ch and ch + 1) a bounded
        // chance to land before the block's shared memory is released.
        if (threadIdx.x == 0) {
            const int b0 = (ch - cb) & 1;
            mbar_wait_bounded(&sm.full[b0], (uses[b0] - 1u) & 1u);
            if (ch + 1 < ce) mbar_wait_bounded(&sm.full[b0 ^ 1], uses[b0 ^ 1] & 1u);
        }
        return;
    }

    // ---- epilogue: field value and fused maps ------------------------------------
#pragma unroll
    for (int c = 0; c < C; ++c) {
        two_sum_acc(s[c], e[c], p[c]);
        if (warp_active && valid[c]) {
            const int64_t i = lbase + c;
            if (partial != nullptr) {
                partial[i] = make_float2(s[c], e[c]);
            } else {
                const float y = (s[c] + e[c]) + d.map.mu;
                map_store(d.map, static_cast<int64_t>(__ldg(d.perm + i)) - d.perm_base, y);
            }
        }
    }
}

template <int DIM, int C, int W>
__device__ __forceinline__ void init_smem(FwdSmem<C, W>& sm) {
    if (threadIdx.x == 0) {
        mbar_init(&sm.full[0], 1);
        mbar_init(&sm.full[1], 1);
        sm.abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
}

// blockIdx.x: cell tile; blockIdx.y: mode split (gridDim.y splits of the
// chunk range; with more than one split every block writes its TwoSum
// partial (s, e) per sorted cell to partial[split * n_cells + i]).
template <int DIM, int C, int W>
__global__ void __launch_bounds__(W * 32) synth_fwd_kernel(FwdDesc d, float2* partial, int32_t* status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    auto& sm = *reinterpret_cast<FwdSmem<C, W>*>(smem_raw);
    init_smem<DIM, C, W>(sm);
    uint32_t uses[2] = {0u, 0u};
    const int64_t tile_base = static_cast<int64_t>(blockIdx.x) * (W * 32 * C);
    const int n_chunks = d.n_pad / kChunk;
    const int split = blockIdx.y, n_split = gridDim.y;
    const int cb = static_cast<int>(static_cast<int64_t>(n_chunks) * split / n_split);
    const int ce = static_cast<int>(static_cast<int64_t>(n_chunks) * (split + 1) / n_split);
    float2* part = n_split > 1 ? partial + static_cast<int64_t>(split) * d.n_cells : nullptr;
    synth_tile<DIM, C, W>(d, tile_base, cb, ce, part, sm, uses, status);
}

// Combine the per-split partials of every sorted cell in split order (a
// fixed order, so results are deterministic) and apply the maps.
__global__ void __launch_bounds__(256) synth_split_finalize(FwdDesc d, const float2* __restrict__ partial,
                                                            int n_split) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= d.n_cells) return;
    float s = 0.0f, e = 0.0f;
    for (int k = 0; k < n_split; ++k) {
        const float2 v = partial[static_cast<int64_t>(k) * d.n_cells + i];
        two_sum_acc(s, e, v.x);
        e += v.y;
    }
    const float y = (s + e) + d.map.mu;
    map_store(d.map, static_cast<int64_t>(__ldg(d.perm + i)) - d.perm_base, y);
}

// Persistent batched kernel: blocks pull (realisation, tile) work items from
// a counter until the list is exhausted.  DIM is the plan's dimension; a
// realisation of lower dimension has zero frequencies on the extra axes.
template <int DIM, int C, int W>
__global__ void __launch_bounds__(W * 32) synth_batched_kernel(const FwdDesc* __restrict__ descs,
                                                                const WorkItem* __restrict__ work,
                                                                int32_t n_work, int32_t* counter,
                                                                int32_t* status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    auto& sm = *reinterpret_cast<FwdSmem<C, W>*>(smem_raw);
    init_smem<DIM, C, W>(sm);
    uint32_t uses[2] = {0u, 0u};
    for (;;) {
        if (threadIdx.x == 0) sm.work = atomicAdd(counter, 1);
        __syncthreads();
        const int w = sm.work;
        if (w >= n_work) break;
        const WorkItem it = work[w];
        // copy the descriptor into shared memory (word by word)
        {
            const int nwords = static_cast<int>(sizeof(FwdDesc) / 4);
            const int32_t* src = reinterpret_cast<const int32_t*>(descs + it.r);
            int32_t* dst = reinterpret_cast<int32_t*>(&sm.desc);
            for (int k = threadIdx.x; k < nwords; k += blockDim.x) dst[k] = src[k];
        }
        __syncthreads();
        const int64_t tile_base = static_cast<int64_t>(it.t) * (W * 32 * C);
        synth_tile<DIM, C, W>(sm.desc, tile_base, 0, sm.desc.n_pad / kChunk, nullptr, sm, uses, status);
        if (sm.abort_flag) break;
        __syncthreads();
    }
}

// Mode splits for a launch of `tiles` blocks: enough to fill about eight
// waves of resident blocks, at most kMaxSplit, at least two chunks per split,
// and only as many as the workspace holds.
int choose_split(int64_t tiles, int n_chunks, int resident, int64_t n_cells, size_t ws_bytes) {
    if (tiles <= 0) return 1;
    int64_t want = (8 * static_cast<int64_t>(resident) + tiles - 1) / tiles;
    if (want > kMaxSplit) want = kMaxSplit;
    if (want > n_chunks / 2) want = n_chunks / 2;
    const int64_t fits = n_cells > 0 ? static_cast<int64_t>(ws_bytes / (sizeof(float2) * n_cells)) : 0;
    if (want > fits) want = fits;
    return want < 2 ? 1 : static_cast<int>(want);
}

template <int DIM, int C, int W>
int launch_fwd_cfg(const FwdDesc& d, void* workspace, size_t ws_bytes, int32_t* status, cudaStream_t st) {
    const size_t smem = sizeof(FwdSmem<C, W>);
    auto kern = synth_fwd_kernel<DIM, C, W>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    const int64_t per_cta = int64_t(W) * 32 * C;
    const int64_t grid = (d.n_cells + per_cta - 1) / per_cta;
    if (grid == 0) return cudaSuccess;
    int n_split = 1;
    if (workspace != nullptr) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, W * 32, smem);
        n_split = choose_split(grid, d.n_pad / kChunk, sms * (per_sm > 0 ? per_sm : 1), d.n_cells, ws_bytes);
    }
    float2* partial = static_cast<float2*>(workspace);
    kern<<<dim3(static_cast<unsigned>(grid), n_split), W * 32, smem, st>>>(d, partial, status);
    count_launches(1);
    if (n_split > 1) {
        synth_split_finalize<<<static_cast<unsigned>((d.n_cells + 255) / 256), 256, 0, st>>>(d, partial, n_split);
        count_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace

// Configuration used by the single-realisation path: C = 8 cells per lane,
// W = 4 warps (1024 cells per block).
int fwd_tile_cells(int cfg) {
    switch (cfg) {
        case 0: return 4 * 32 * 8;
        case 1: return 8 * 32 * 8;
        case 2: return 4 * 32 * 4;
        default: return 0;
    }
}

size_t synth_workspace_bytes(int64_t n_cells) {
    return static_cast<size_t>(align256(int64_t(kMaxSplit) * n_cells * int64_t(sizeof(float2))));
}

int launch_synth_fwd(const FwdDesc& d, void* workspace, size_t ws_bytes, int32_t* status, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (d.dim) {
        case 1: return launch_fwd_cfg<1, 8, 4>(d, workspace, ws_bytes, status, st);
        case 2: return launch_fwd_cfg<2, 8, 4>(d, workspace, ws_bytes, status, st);
        case 3: return launch_fwd_cfg<3, 8, 4>(d, workspace, ws_bytes, status, st);
        default: return cudaErrorInvalidValue;
    }
}

namespace {
template <int DIM, int C, int W>
int launch_batched_cfg(const FwdDesc* descs, const WorkItem* work, int32_t n_work,
                       int32_t* counter, int32_t* status, cudaStream_t st) {
    const size_t smem = sizeof(FwdSmem<C, W>);
    auto kern = synth_batched_kernel<DIM, C, W>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, W * 32, smem);
    if (per_sm < 1) per_sm = 1;
    kern<<<sms * per_sm, W * 32, smem, st>>>(descs, work, n_work, counter, status);
    count_launches(1);
    return cudaGetLastError();
}

template <int DIM>
int launch_batched_dim(int cfg, const FwdDesc* descs, const WorkItem* work, int32_t n_work,
                       int32_t* counter, int32_t* status, cudaStream_t st) {
    switch (cfg) {
        case 0: return launch_batched_cfg<DIM, 8, 4>(descs, work, n_work, counter, status, st);
        case 1: return launch_batched_cfg<DIM, 8, 8>(descs, work, n_work, counter, status, st);
        case 2: return launch_batched_cfg<DIM, 4, 4>(descs, work, n_work, counter, status, st);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace

int launch_synth_batched(const void* workspace, const BatchHeader& h, int32_t* status,
                         int32_t* counter, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const unsigned char* base = static_cast<const unsigned char*>(workspace);
    const FwdDesc* descs = reinterpret_cast<const FwdDesc*>(base + h.off_desc);
    const WorkItem* work = reinterpret_cast<const WorkItem*>(base + h.off_work);
    cudaError_t err = cudaMemsetAsync(counter, 0, sizeof(int32_t), st);
    if (err != cudaSuccess) return err;
    switch (h.dim_max) {
        case 1: return launch_batched_dim<1>(h.cfg, descs, work, h.n_work, counter, status, st);
        case 2: return launch_batched_dim<2>(h.cfg, descs, work, h.n_work, counter, status, st);
        case 3: return launch_batched_dim<3>(h.cfg, descs, work, h.n_work, counter, status, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace grf
