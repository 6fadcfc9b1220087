// Forward synthesis kernel: Y_i = mu + sum_j A_j cos(2 pi (a_j . x_i + psi_j))
// at arbitrary cell centres (Icardi et al., arXiv 2212.10961, Sec. 4.1,
// Eq. DiscreteFT), with the property maps of Sec. 3.1 / Sec. 4.1 fused into
// the epilogue.
//
// Work decomposition.  Cells arrive spatially sorted (cell plan, Z-order).
// Every warp works on its own: it owns 32*C consecutive sorted cells (C per
// lane, in registers), takes the midpoint of their bounding box as origin x0
// (half-extent E), and streams the mode table through its own two shared-
// memory buffers filled by 1-D bulk copies completed on its own mbarriers.
// There is no block-wide barrier, so warps never wait for one another.
//
// Phase split.  For mode j at cell i
//     theta_ij = 2 pi frac(a_j . x0 + psi_j)  +  (2 pi a_j) . (x_i - x0),
// the first term once per (warp, mode) in compensated FP32
// (phase_exact_turns), the second per cell-mode with DIM FFMAs.  Three classes
// of modes, all prefixes of the table (sorted by |a|_1, descending):
//   super  : span over the lane's block > tau2 turns -> exact phase per cell;
//   medium : span over the warp's block > tau1 turns -> exact phase at the
//            lane origin xt once per (lane, mode), FP32 offsets per cell;
//   light  : the rest, the hot loop: DIM FFMA, 1 FMUL (radian scaling inside
//            cos.approx), 1 MUFU cosine, 1 FFMA accumulate per cell-mode.
// Per-chunk FP32 partials are folded into TwoSum-compensated accumulators.
// Every mbarrier wait is bounded and reports through the status word.
#include <cuda_runtime.h>

#include "device_common.cuh"

namespace grf {

// Warp tiles of 2-D and 3-D synthesis launches (single-field and batched)
// that took the general path [0] and the lattice path [1] since the last
// grf_take_path_counts (diagnostics).
static __device__ unsigned long long g_path_warps[2];

namespace {

constexpr int kWChunk = 128;                 // modes per warp chunk
constexpr int kWChunkBytes = kWChunk * 16;   // hot records only (16 B per mode)
constexpr int kStages = 3;                   // chunk buffers per warp (prefetch distance 2)
constexpr int kMaxSplit = 8;                 // most mode splits of one launch
constexpr float kInvTwoPiF = 0.159154943091895335769f;
static_assert(kChunk % kWChunk == 0, "table padding must be a multiple of the warp chunk");

// Shared memory of one warp: a ring of hot-record chunks filled by bulk
// copies, and the warp-origin phases of the current chunk.  The hi/lo
// records needed for those phases are read through L1 by the lanes.
struct WarpSmem {
    float4 buf[kStages][kWChunk];  // (2 pi a_x, 2 pi a_y, 2 pi a_z, A)
    float t0[kWChunk];             // warp-origin phase of the chunk's modes (radians)
    uint64_t full[kStages];
};

// NS > 0 (lattice path enabled): per warp, NS step phasors per mode of the
// current chunk (see lattice_chunk); NS = 0 keeps one unused entry.
template <int W, int NS = 0>
struct FwdSmem {
    WarpSmem w[W];
    FwdDesc desc[W];  // batched: each warp's current realisation
    float4 stp[W][NS > 0 ? NS * kWChunk / 2 : 1];
};

// Phase a v in turns, reduced to [-1/2, 1/2], of a = ah + al (FP32 pair) at a
// point v of one axis: the product ah v split exactly by an FMA, integer
// parts removed exactly (as phase_exact_turns, without psi).
__device__ __forceinline__ float axis_turns(float ah, float al, float v) {
    const float pr = ah * v;
    const float e = fmaf(ah, v, -pr);
    return frac_turn(frac_turn(pr) + fmaf(al, v, e));
}

// Lattice lanes.  When every lane's C cells are the 4 x NY block
//     (xl + i hx, yl + k hy, zl),  cell c = i + 4 k,
// of one Cartesian grid (the same hx, hy in every lane of the warp), a term
// of the sum at cell c is the real part of
//     A e^{i theta(lane corner)} * e^{2 pi i a_x i hx} * e^{2 pi i a_y k hy},
// so one hardware sine/cosine pair per (lane, mode) and two exact step
// phasors per axis shared by the warp replace the per-cell phase and cosine:
// per cell-mode two FFMA (one FADD for i = 0) and a quarter of a complex
// product.  The step phasors come from exact reduced phases (axis_turns),
// the corner phase as in the general path: from the warp-origin phase plus
// the corner offset for light modes, exactly for the modes of the medium
// and super classes (j < k_med).  Adds this chunk's terms to p[].
template <int DIM, int C, int NS>
__device__ __forceinline__ void lattice_chunk(const FwdDesc& d, int jbase, int k_med, const float (&x0)[DIM],
                                              const float (&xl)[DIM], float hx, float hy, const float4* hotS,
                                              float* t0s, float4* stp, float (&p)[C], int lane) {
    constexpr int NY = C / 4;
    static_assert(NS == NY + 2, "step phasors: 3 along x, NY - 1 along y");
    for (int m = lane; m < kWChunk; m += 32) {
        const int j = jbase + m;
        const float4 c0 = __ldg(d.cold + 2 * j);
        const float4 c1 = __ldg(d.cold + 2 * j + 1);
        t0s[m] = kTwoPiF * phase_exact_turns<DIM>(x0, c0, c1);
        float ph[NS];
#pragma unroll
        for (int k = 1; k <= 3; ++k) ph[k - 1] = kTwoPiF * axis_turns(c0.x, c0.y, static_cast<float>(k) * hx);
#pragma unroll
        for (int k = 1; k < NY; ++k) ph[2 + k] = kTwoPiF * axis_turns(c0.z, c0.w, static_cast<float>(k) * hy);
        float4* sm = stp + m * (NS / 2);
#pragma unroll
        for (int k = 0; k < NS / 2; ++k)
            sm[k] = make_float4(hw_cos(ph[2 * k]), hw_sin(ph[2 * k]), hw_cos(ph[2 * k + 1]), hw_sin(ph[2 * k + 1]));
    }
    __syncwarp();
    float dl[DIM];  // lane corner relative to the warp origin
#pragma unroll
    for (int k = 0; k < DIM; ++k) dl[k] = xl[k] - x0[k];
    auto mode = [&](const float4 h, const float th, const float4* sm) {
        const float er = h.w * hw_cos(th);
        const float ei = h.w * hw_sin(th);
        const float4 s01 = sm[0];  // step x 1, step x 2
        const float4 s23 = sm[1];  // step x 3, step y 1
#pragma unroll
        for (int k = 0; k < NY; ++k) {
            float zr = er, zi = ei;
            if (k > 0) {
                const float4 q = k == 1 ? s23 : sm[1 + k / 2];
                const float qr = (k == 1 || k == 3) ? q.z : q.x;
                const float qi = (k == 1 || k == 3) ? q.w : q.y;
                zr = fmaf(er, qr, -ei * qi);
                zi = fmaf(er, qi, ei * qr);
            }
            p[4 * k + 0] += zr;
            p[4 * k + 1] = fmaf(zr, s01.x, fmaf(-zi, s01.y, p[4 * k + 1]));
            p[4 * k + 2] = fmaf(zr, s01.z, fmaf(-zi, s01.w, p[4 * k + 2]));
            p[4 * k + 3] = fmaf(zr, s23.x, fmaf(-zi, s23.y, p[4 * k + 3]));
        }
    };
    const int mh = min(max(k_med - jbase, 0), kWChunk);
    for (int m = 0; m < mh; ++m) {
        const int j = jbase + m;
        const float th = kTwoPiF * phase_exact_turns<DIM>(xl, __ldg(d.cold + 2 * j), __ldg(d.cold + 2 * j + 1));
        mode(hotS[m], th, stp + m * (NS / 2));
    }
#pragma unroll 2
    for (int m = mh; m < kWChunk; ++m) {
        const float4 h = hotS[m];
        float th = fmaf(h.x, dl[0], t0s[m]);
        if (DIM > 1) th = fmaf(h.y, dl[1], th);
        if (DIM > 2) th = fmaf(h.z, dl[2], th);
        mode(h, th, stp + m * (NS / 2));
    }
}

__device__ __forceinline__ void warp_init_barriers(WarpSmem& ws) {
    if ((threadIdx.x & 31) == 0) {
        for (int b = 0; b < kStages; ++b) mbar_init(&ws.full[b], 1);
        fence_mbar_init();
    }
    __syncwarp();
}

// Lane 0: bulk copy of the hot records of warp chunk `ch` into buffer b.
__device__ __forceinline__ void issue_wchunk(const FwdDesc& d, int ch, WarpSmem& ws, int b) {
    mbar_arrive_expect_tx(&ws.full[b], kWChunkBytes);
    bulk_g2s(ws.buf[b], d.hot + static_cast<int64_t>(ch) * kWChunk, kWChunkBytes, &ws.full[b]);
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

// One warp tile: the 32*C sorted cells starting at wbase, modes of warp
// chunks [cb, ce).  `uses` counts completed waits per buffer (parity across
// tiles).  Returns false if a bounded wait expired (status bit 2 set).
// With `partial` the TwoSum pair (s, e) of every cell is written to
// partial[i] instead of the maps (mode split over blocks).
// POLY: cells per lane whose cosine is evaluated on the FMA pipe (polynomial)
// instead of the MUFU pipe in the light loop.  It pays only where the MUFU
// pipe, not instruction issue, limits the kernel (the persistent batched
// kernel); the single-realisation kernel uses 0.
// MM: the epilogue also forms the mismatch gradient of every cell and writes
// the warp's sum of (K - T)^2 to d.map.lpart[wbase / (32 C)] (kMapMismatch).
template <int DIM, int C, int POLY, bool MM = false, int NS = 0>
__device__ __forceinline__ bool synth_warp_tile(const FwdDesc& d, int64_t wbase, int cb, int ce,
                                                float2* partial, WarpSmem& ws, uint32_t (&uses)[kStages],
                                                int32_t* status, float4* stp = nullptr) {
    const int lane = threadIdx.x & 31;
    const int64_t n = d.n_cells;
    const int jlo = cb * kWChunk;
    const int jhi = ce * kWChunk;

    // Prefetch the first chunks (this warp's buffers are free: its previous
    // tile waited for every copy it issued).
    if (lane == 0) {
        fence_proxy_async_smem();
        for (int q = 0; q < kStages - 1 && cb + q < ce; ++q) issue_wchunk(d, cb + q, ws, q);
    }

    // ---- load cells (lane-contiguous), bounding boxes, origins ------------
    const int64_t lbase = wbase + static_cast<int64_t>(lane) * C;
    float x[C][DIM];
    bool valid[C];
    {
        const float* src[3] = {d.xs, d.ys, d.zs};
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
                const int64_t first = lbase < n ? lbase : wbase;
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
    const int k_med = prefix_for(d.kpref, d.n_pad, Ew * d.inv_tau1);
    const int k_sup = min(k_med, prefix_for(d.kpref, d.n_pad, Et * d.inv_tau2));

    float s[C], e[C], p[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        s[c] = 0.0f;
        e[c] = 0.0f;
        p[c] = 0.0f;
    }

    // ---- lattice lanes (see lattice_chunk): every lane's cells are the 4 x C/4
    // block of one grid spacing (hx, hy), the same in the whole warp ----------------
    bool lat = false;
    float hx = 0.0f, hy = 0.0f;
    float xl[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) xl[k] = x[0][k];
    if constexpr (NS > 0) {
        static_assert(DIM >= 2 && C >= 8 && C % 4 == 0, "lattice lanes are 4 x C/4 blocks");
        bool ok = true;
#pragma unroll
        for (int c = 0; c < C; ++c) ok = ok && valid[c];
        hx = x[1][0] - x[0][0];
        hy = x[4][1] - x[0][1];
        ok = ok && hx > 0.0f && hy > 0.0f;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float ox = static_cast<float>(c & 3) * hx;
            const float oy = static_cast<float>(c >> 2) * hy;
            ok = ok && (x[c][0] - x[0][0] == ox) && (x[0][0] + ox == x[c][0]) && (x[c][1] - x[0][1] == oy) &&
                 (x[0][1] + oy == x[c][1]);
            if (DIM > 2) ok = ok && (x[c][2] == x[0][2]);
        }
        // every lane takes part in the shuffles (no short-circuit around them)
        const float hx0 = __shfl_sync(0xffffffffu, hx, 0);
        const float hy0 = __shfl_sync(0xffffffffu, hy, 0);
        ok = ok && hx == hx0 && hy == hy0;
        lat = __all_sync(0xffffffffu, ok);
        if (lane == 0) atomicAdd(&g_path_warps[lat ? 1 : 0], 1ull);
    }

    // Chunk pipeline: waits for each of this warp's chunks in turn, keeping
    // kStages - 1 bulk copies in flight, and hands it to body(hotS, jbase).
    // If a bounded wait expires it records that in the status word, gives the
    // copies still in flight a bounded chance to land before this warp's
    // shared memory is reused, and returns false.
    auto run_chunks = [&](auto&& body) -> bool {
        bool ok = true;
        int ch = cb;
        for (; ch < ce; ++ch) {
            const int b = (ch - cb) % kStages;
            // keep kStages - 1 chunks in flight: refill the buffer freed last
            if (lane == 0 && ch + kStages - 1 < ce) {
                fence_proxy_async_smem();
                issue_wchunk(d, ch + kStages - 1, ws, (ch - cb + kStages - 1) % kStages);
            }
            // the hi/lo records of the next chunk (128 modes x 32 B = 32 lines,
            // one per lane) are pulled into L1 while this chunk is summed
            if (ch + 1 < ce) prefetch_l1(d.cold + 2 * ((ch + 1) * kWChunk + lane * (kWChunk / 32)));
            const uint32_t parity = uses[b] & 1u;
            ok = __all_sync(0xffffffffu, mbar_wait_bounded(&ws.full[b], parity));
            uses[b] += 1;
            if (!ok) break;
            body(ws.buf[b], ch * kWChunk);
            __syncwarp();  // every lane is done with buffer b and the chunk's tables
        }
        if (!ok) {
            if (lane == 0) {
                atomicOr(status, 2);
                for (int q = 0; q < kStages && ch + q < ce; ++q) {
                    const int bq = (ch - cb + q) % kStages;
                    mbar_wait_bounded(&ws.full[bq], (q == 0 ? uses[bq] - 1u : uses[bq]) & 1u);
                }
            }
            __syncwarp();
        }
        return ok;
    };
    auto fold = [&]() {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            two_sum_acc(s[c], e[c], p[c]);
            p[c] = 0.0f;
        }
    };

    bool handled = false;
    if constexpr (NS > 0) {
        if (lat) {
            handled = true;
            if (!run_chunks([&](float4* hotS, int jbase) {
                    lattice_chunk<DIM, C, NS>(d, jbase, k_med, x0, xl, hx, hy, hotS, ws.t0, stp, p, lane);
                    fold();
                }))
                return false;
        }
    }
    if (!handled) {
        // ---- super class: exact phase at every cell -----------------------------
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
            if ((j & 63) == 63) fold();
        }

        // ---- medium class: exact phase at the lane origin ---------------------
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
            if (((j - k_sup) & 63) == 63) fold();
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

        // ---- light class over this warp's staged chunks --------------------------
        const bool done = run_chunks([&](float4* hotS, int jbase) {
            if (jbase + kWChunk <= k_med) return;
            const int m0 = k_med > jbase ? k_med - jbase : 0;
            auto mode = [&](const float4 h, const float t0) {
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    float th = fmaf(h.x, dx[c][0], t0);
                    if (DIM > 1) th = fmaf(h.y, dx[c][1], th);
                    if (DIM > 2) th = fmaf(h.z, dx[c][2], th);
                    float cv;
                    if (c >= C - POLY) {
                        const float u = th * kInvTwoPiF;
                        cv = cos_turns_poly(u - ((u + kRoundMagic) - kRoundMagic));
                    } else {
                        cv = hw_cos(th);
                    }
                    p[c] = fmaf(h.w, cv, p[c]);
                }
            };
            if constexpr (C >= 16) {
                // groups of 4 modes share one 16-byte load of t0; the modes of
                // the first group that belong to the medium class (summed
                // already) get amplitude 0 in this warp's copy of the chunk
                const int m0a = m0 & ~3;
                for (int m = m0a + lane; m < kWChunk; m += 32) {
                    const int j = jbase + m;
                    float t = 0.0f;
                    if (m >= m0)
                        t = kTwoPiF * phase_exact_turns<DIM>(x0, __ldg(d.cold + 2 * j), __ldg(d.cold + 2 * j + 1));
                    else
                        hotS[m].w = 0.0f;
                    ws.t0[m] = t;
                }
                __syncwarp();
#pragma unroll 2
                for (int m = m0a; m < kWChunk; m += 4) {
                    const float4 t4 = *reinterpret_cast<const float4*>(&ws.t0[m]);
                    mode(hotS[m + 0], t4.x);
                    mode(hotS[m + 1], t4.y);
                    mode(hotS[m + 2], t4.z);
                    mode(hotS[m + 3], t4.w);
                }
            } else {
                for (int m = m0 + lane; m < kWChunk; m += 32) {
                    const int j = jbase + m;
                    ws.t0[m] = kTwoPiF * phase_exact_turns<DIM>(x0, __ldg(d.cold + 2 * j), __ldg(d.cold + 2 * j + 1));
                }
                __syncwarp();
#pragma unroll 8
                for (int m = m0; m < kWChunk; ++m) mode(hotS[m], ws.t0[m]);
            }
            fold();
        });
        if (!done) return false;
    }

    // ---- epilogue: field value and fused maps ------------------------------------
    double lsum = 0.0;  // MM: this lane's sum of (K - T)^2
#pragma unroll
    for (int c = 0; c < C; ++c) {
        two_sum_acc(s[c], e[c], p[c]);
        if (valid[c]) {
            const int64_t i = lbase + c;
            if (partial != nullptr) {
                partial[i] = make_float2(s[c], e[c]);
            } else {
                const float y = (s[c] + e[c]) + d.map.mu;
                const int64_t o = static_cast<int64_t>(__ldg(d.perm + i)) - d.perm_base;
                if (index_ok(o, d.n_cells)) {
                    map_store(d.map, o, y);
                    if constexpr (MM) lsum += mismatch_store(d.map, o, y);
                }
            }
        }
    }
    if constexpr (MM) {
        if (partial == nullptr) {
            // fixed butterfly order: the warp's sum does not depend on timing
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
            if (lane == 0) d.map.lpart[wbase / (32 * C)] = lsum;
        }
    }
    return true;
}

// blockIdx.x: W warp tiles; blockIdx.y: mode split (gridDim.y splits of the
// warp-chunk range; with more than one split every warp writes its TwoSum
// partial (s, e) per sorted cell to partial[split * n_cells + i]).
// Lattice path in the single-field kernel for 2-D and 3-D fields (NS step
// phasors per mode); the 2-D kernel then holds 5 blocks per SM (shared memory).
template <int DIM, int C>
__host__ __device__ constexpr int lattice_ns() { return DIM >= 2 && C >= 8 ? C / 4 + 2 : 0; }
template <int DIM, int C>
__host__ __device__ constexpr int fwd_min_blocks() { return C >= 16 ? 4 : (lattice_ns<DIM, C>() > 0 ? 5 : 6); }

template <int DIM, int C, int W, bool MM>
__global__ void __launch_bounds__(W * 32, (fwd_min_blocks<DIM, C>())) synth_fwd_kernel(FwdDesc d, float2* partial,
                                                                                   int32_t* status) {
    constexpr int NS = lattice_ns<DIM, C>();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    auto& sm = *reinterpret_cast<FwdSmem<W, NS>*>(smem_raw);
    const int warp = threadIdx.x >> 5;
    WarpSmem& ws = sm.w[warp];
    warp_init_barriers(ws);
    const int64_t wbase = (static_cast<int64_t>(blockIdx.x) * W + warp) * (32 * C);
    if (wbase >= d.n_cells) return;
    uint32_t uses[kStages] = {};
    const int n_chunks = d.n_pad / kWChunk;
    const int split = blockIdx.y, n_split = gridDim.y;
    const int cb = static_cast<int>(static_cast<int64_t>(n_chunks) * split / n_split);
    const int ce = static_cast<int>(static_cast<int64_t>(n_chunks) * (split + 1) / n_split);
    float2* part = n_split > 1 ? partial + static_cast<int64_t>(split) * d.n_cells : nullptr;
    const bool ok = synth_warp_tile<DIM, C, 0, MM, NS>(d, wbase, cb, ce, part, ws, uses, status, sm.stp[warp]);
    if (MM && !ok && part == nullptr && (threadIdx.x & 31) == 0)
        d.map.lpart[wbase / (32 * C)] = __longlong_as_double(0x7ff8000000000000ll);  // NaN: no loss
}

// Combine the per-split partials of every sorted cell in split order (a
// fixed order, so results are deterministic) and apply the maps; with the
// mismatch bit every block also writes its sum of (K - T)^2 to lpart.
__global__ void __launch_bounds__(256) synth_split_finalize(FwdDesc d, const float2* __restrict__ partial,
                                                            int n_split) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (i < d.n_cells) {
        float s = 0.0f, e = 0.0f;
        for (int k = 0; k < n_split; ++k) {
            const float2 v = partial[static_cast<int64_t>(k) * d.n_cells + i];
            two_sum_acc(s, e, v.x);
            e += v.y;
        }
        const float y = (s + e) + d.map.mu;
        const int64_t o = static_cast<int64_t>(__ldg(d.perm + i)) - d.perm_base;
        if (index_ok(o, d.n_cells)) {
            map_store(d.map, o, y);
            if (d.map.bits & kMapMismatch) l = mismatch_store(d.map, o, y);
        }
    }
    if (d.map.bits & kMapMismatch) {
        __shared__ double red[8];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < 8; ++w) t += red[w];
            d.map.lpart[blockIdx.x] = t;
        }
    }
}

// loss = (sum of the nb partial sums of (K - T)^2) / n_mean, one block,
// fixed order.
__global__ void __launch_bounds__(256) loss_sum_kernel(const double* __restrict__ part, int64_t nb,
                                                       double inv_n, double* __restrict__ out) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int64_t k = threadIdx.x; k < nb; k += 256) acc += part[k];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0] * inv_n;
}

// Persistent batched kernel: every warp pulls (realisation, warp tile) work
// items from a counter until the list is exhausted.  DIM is the plan's
// dimension; a realisation of lower dimension has zero frequencies on the
// extra axes.
template <int DIM, int C, int W>
__global__ void __launch_bounds__(W * 32, C >= 16 ? 4 : 5) synth_batched_kernel(const FwdDesc* __restrict__ descs,
                                                                const WorkItem* __restrict__ work,
                                                                int32_t n_work, int32_t* counter,
                                                                int32_t* status) {
    // lattice lanes (lattice_chunk) for the realisations of 2 or 3 dimensions
    constexpr int NS = lattice_ns<2, C>();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    auto& sm = *reinterpret_cast<FwdSmem<W, NS>*>(smem_raw);
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    WarpSmem& ws = sm.w[warp];
    FwdDesc& d = sm.desc[warp];
    warp_init_barriers(ws);
    uint32_t uses[kStages] = {};
    for (;;) {
        int w = 0;
        if (lane == 0) w = atomicAdd(counter, 1);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= n_work) break;
        const WorkItem it = work[w];
        {
            constexpr int kWords = static_cast<int>(sizeof(FwdDesc) / 4);
            const int32_t* src = reinterpret_cast<const int32_t*>(descs + it.r);
            int32_t* dst = reinterpret_cast<int32_t*>(&d);
            for (int k = lane; k < kWords; k += 32) dst[k] = src[k];
        }
        __syncwarp();
        const int64_t wbase = static_cast<int64_t>(it.t) * (32 * C);
        // a realisation of lower dimension than the plan (e.g. 2-D fields on a
        // plan whose third coordinate is 0) runs the tile of its own dimension
        bool ok;
        constexpr int NSD = DIM >= 2 ? NS : 0;
        if (DIM > 1 && d.dim == 1)
            ok = synth_warp_tile<1, C, 1>(d, wbase, 0, d.n_pad / kWChunk, nullptr, ws, uses, status);
        else if (DIM > 2 && d.dim == 2)
            ok = synth_warp_tile<(DIM > 2 ? 2 : DIM), C, 1, false, (DIM > 2 ? NS : 0)>(
                d, wbase, 0, d.n_pad / kWChunk, nullptr, ws, uses, status, sm.stp[warp]);
        else
            ok = synth_warp_tile<DIM, C, 1, false, NSD>(d, wbase, 0, d.n_pad / kWChunk, nullptr, ws, uses, status,
                                                        sm.stp[warp]);
        if (!ok) break;
        __syncwarp();  // every lane is done with the descriptor
    }
}

// Mode splits for a launch of `tiles` blocks: enough to fill about eight
// waves of resident blocks, at most kMaxSplit, at least two warp chunks per
// split, and only as many as the workspace holds.
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
    const size_t smem = sizeof(FwdSmem<W, lattice_ns<DIM, C>()>);
    const bool mm = (d.map.bits & kMapMismatch) != 0;
    auto kern = mm ? synth_fwd_kernel<DIM, C, W, true> : synth_fwd_kernel<DIM, C, W, false>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    const int64_t per_cta = int64_t(W) * 32 * C;
    const int64_t grid = (d.n_cells + per_cta - 1) / per_cta;
    if (grid == 0) {
        if (mm) {  // no cells: the loss is 0
            loss_sum_kernel<<<1, 256, 0, st>>>(d.map.lpart, 0, 0.0, d.map.loss);
            count_launches(1);
        }
        return cudaGetLastError();
    }
    int n_split = 1;
    if (workspace != nullptr) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, W * 32, smem);
        n_split = choose_split(grid, d.n_pad / kWChunk, sms * (per_sm > 0 ? per_sm : 1), d.n_cells, ws_bytes);
    }
    float2* partial = static_cast<float2*>(workspace);
    kern<<<dim3(static_cast<unsigned>(grid), n_split), W * 32, smem, st>>>(d, partial, status);
    count_launches(1);
    const int64_t fin_blocks = (d.n_cells + 255) / 256;
    if (n_split > 1) {
        synth_split_finalize<<<static_cast<unsigned>(fin_blocks), 256, 0, st>>>(d, partial, n_split);
        count_launches(1);
    }
    if (mm) {
        const int64_t nb = n_split > 1 ? fin_blocks : (d.n_cells + 32 * C - 1) / (32 * C);
        loss_sum_kernel<<<1, 256, 0, st>>>(d.map.lpart, nb, d.map.inv_n_mean, d.map.loss);
        count_launches(1);
    }
    return cudaGetLastError();
}

template <int DIM, int C, int W>
int launch_batched_cfg(const FwdDesc* descs, const WorkItem* work, int32_t n_work, int32_t* counter,
                       int32_t* status, cudaStream_t st) {
    const size_t smem = sizeof(FwdSmem<W, lattice_ns<2, C>()>);
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
        case 1: return launch_batched_cfg<DIM, 4, 4>(descs, work, n_work, counter, status, st);
        case 2: return launch_batched_cfg<DIM, 16, 4>(descs, work, n_work, counter, status, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// Cells per work item (one warp tile) of the batched configurations.
int fwd_tile_cells(int cfg) {
    switch (cfg) {
        case 0: return 32 * 8;
        case 1: return 32 * 4;
        case 2: return 32 * 16;
        default: return 0;
    }
}

size_t synth_workspace_bytes(int64_t n_cells) {
    return static_cast<size_t>(align256(int64_t(kMaxSplit) * n_cells * int64_t(sizeof(float2))));
}

// One entry per warp tile of at least 128 cells, or per 256-cell block of the
// split finalize, whichever is more.
int64_t mismatch_partials(int64_t n_cells) { return (n_cells + 127) / 128 + 1; }

int launch_loss_sum(const double* part, int64_t nb, double inv_n, double* out, void* stream) {
    loss_sum_kernel<<<1, 256, 0, static_cast<cudaStream_t>(stream)>>>(part, nb, inv_n, out);
    count_launches(1);
    return cudaGetLastError();
}

int launch_synth_fwd(const FwdDesc& d, void* workspace, size_t ws_bytes, int32_t* status, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (d.dim) {
        case 1: return launch_fwd_cfg<1, 8, 4>(d, workspace, ws_bytes, status, st);
        case 2: return launch_fwd_cfg<2, 8, 4>(d, workspace, ws_bytes, status, st);
        case 3: return launch_fwd_cfg<3, 16, 4>(d, workspace, ws_bytes, status, st);
        default: return cudaErrorInvalidValue;
    }
}

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

unsigned long long take_index_faults_fwd() { return take_tu_index_faults(); }

int take_path_counts(unsigned long long* general, unsigned long long* lattice) {
    unsigned long long v[2] = {0ull, 0ull};
    const unsigned long long zero[2] = {0ull, 0ull};
    cudaError_t e = cudaMemcpyFromSymbol(v, g_path_warps, sizeof(v));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_path_warps, zero, sizeof(zero));
    *general = v[0];
    *lattice = v[1];
    return e;
}

}  // namespace grf
