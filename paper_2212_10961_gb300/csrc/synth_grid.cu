// Spectral synthesis on Cartesian grids with the fifth-generation tensor
// cores (Icardi et al., arXiv 2212.10961, Sec. 4.1, Eq. DiscreteFT).
//
// When the cells are the tensor product of three axes -- cell (i, k, l) at
// (X_i, Y_k, Z_l) -- every term of the sum factorises,
//     A_j cos(2 pi (a_j . x + psi_j)) = Re[ Xp_ij W_jc ],
//     Xp_ij = e^{2 pi i a_jx X_i},  W_jc = A_j e^{2 pi i (psi_j + a_jy Y_k + a_jz Z_l)},
// so on a block of 128 x-cells (rows i) by 128 (y, z) cells (columns c) the
// field is a real matrix product over K = 2N:
//     Y[i, c] - mu = sum_j ( Re Xp_ij Re W_jc - Im Xp_ij Im W_jc ).
// The x phasors (operand A) are the same for every block of one x range:
// they are tabulated once per call, already in the tensor core's shared-
// memory layout, and copied in chunk by chunk.  Operand B:
//   * 3-D grids: a tile's columns are a patch of 2^p y-cells by 128 / 2^p
//     z-cells; per chunk the loader copies the patch's y phasors and
//     (amplitude, psi, z) phasors (tables stored chunk by chunk) next to A,
//     and the epilogue warps form B = WZ * Yp in shared memory;
//   * 2-D grids (and 3-D grids of one z layer): B = W * Yp is tabulated like
//     A and copied in as well.
// All phases are exactly reduced (hi/lo frequencies, FMA-split products)
// before an accurate sincospi.
//
// Precision.  Each operand value v (|v| <= 1 after scaling the amplitudes
// by a power of two S) is split into FP16 numbers hi + lo with
// |v - hi - lo| <= 2^-24; a term costs three tensor-core products
// hi.hi + hi.lo + lo.hi (the dropped lo.lo is below 2^-24).  The hi.hi
// products go to an FP32 accumulator in TMEM that takes `fc` chunks of 32
// modes and is then folded into a running FP32 sum (a few tens of folds per
// cell), so the accumulator's own rounding acts on short partial sums only;
// the two correction products, 2^-11 smaller, go to a second accumulator
// that spans the whole tile.
//
// Kernel structure (one CTA per SM, persistent over work items: tiles, or
// for grids of at most 64 tiles (tile, mode split) pairs of whole fold
// intervals whose partial fields a finalize kernel adds in split order):
//   warps 0-15: form B for each chunk (3-D; a thread forms 4 modes of two
//               columns that share a y cell), fold the accumulator, write the
//               maps (warp w reads TMEM lanes 32 (w mod 4) .., columns 32 (w / 4) ..);
//   warp 16   : one thread issues the MMAs (tcgen05.mma kind::f16, M = N = 128);
//   warp 17   : one thread issues the bulk copies; the warp owns TMEM.
// A ring of `sa` stages (A hi/lo and the chunk's tables, or A and B) and,
// in 3-D, a ring of 3 formed B stages.  TMEM (512 columns): the hi.hi
// accumulator double-buffered (2 x 128), the correction accumulator (128) and
// the running sums (128).  Every mbarrier wait is bounded and reports through
// the status word.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "device_common.cuh"
#include "grid_common.cuh"
#include "tcgen05.cuh"

namespace grf {

// Tiles computed by the grid path since the last grf_take_grid_tiles.
static __device__ unsigned long long g_grid_tiles;

namespace {

using gridc::gwait;
using gridc::psi_z_turns;
using gridc::tile_off;

constexpr int kGM = 128;                    // x cells per tile (TMEM lanes)
constexpr int kGN = 128;                    // (y, z) cells per tile (accumulator columns)
constexpr int kGModes = 32;                 // modes per chunk
constexpr int kGK = 2 * kGModes;            // K elements per chunk (re, im)
constexpr int kGOpBytes = kGM * kGK * 2;    // one FP16 operand tile (128 x 64): 16 KB
constexpr int kGPair = 2 * kGOpBytes;       // hi and lo tiles of one operand
constexpr int kGRowBytes = kGModes * 8 + 16;  // one table row of a chunk: 32 float2 + 16 bytes of padding
                                              // (consecutive rows start in different shared-memory banks)
constexpr int kGMaxSA = 4;
constexpr int kGSB = 3;                     // formed B stages (3-D)
constexpr int kGEpiWarps = 16;
constexpr int kGThreads = 32 * (kGEpiWarps + 2);
constexpr int kGColsPerWarp = kGN / (kGEpiWarps / 4);    // TMEM columns a warp folds (4 lane quarters)
// B formation: thread t forms one 4-mode group (t / 64) of two columns that
// share a y cell (z cells 2 q and 2 q + 1 of the patch, pair t mod 64), so the
// y row is read once for both
constexpr int kGFormPairs = kGN / 2;
static_assert(kGColsPerWarp % 32 == 0 && 32 * kGEpiWarps == kGFormPairs * (kGModes / 4), "epilogue warp layout");
constexpr uint32_t kGSbo = 1024;            // 8-row groups of a tile: one 128-byte-swizzle atom apart
constexpr uint32_t kGKStep = 32;            // bytes of 16 K elements inside an atom row
constexpr uint32_t kGTmemCols = 512;
constexpr uint32_t kGCorrCol = 256;         // hi.lo + lo.hi accumulator of the tile
constexpr uint32_t kGSumCol = 384;          // running FP32 sum of the folded hi.hi intervals
constexpr int kGBarBytes = 256;
constexpr int kGAlignPad = 1024;            // room to start the stages on a 1024-byte boundary
constexpr int kGSmemMax = gridc::kSmemMax;
static_assert(kGM == 128 && kGN == 128, "tile shape is fixed by the TMEM layout");

// Amplitude scale: the smallest power of two S >= max |A_j| (1 when all
// amplitudes vanish), so that |W| <= 1.
__device__ __forceinline__ float grid_scale(const TableHeader* h) {
    const float m = h->amp_max;
    if (!(m > 0.0f)) return 1.0f;
    int e;
    frexpf(m, &e);
    return ldexpf(1.0f, e);
}

// B of one chunk for the columns n0 and n1 (one y cell, two z cells):
// W_jc = WZ[l, j] * Yp[k, j] for the 4 modes of group kk8, from the staged
// table rows ty (y) and tw0, tw1 ((amplitude, psi, z) of the two z cells),
// written as (re, im) FP16 pairs into rows n0 and n1 of the hi and lo tiles,
// K segment kk8.
__device__ __forceinline__ void form_b(unsigned char* bhi, const float4* ty, const float4* tw0, const float4* tw1,
                                       int n0, int n1, int kk8) {
    const float4 ya = ty[0], yb = ty[1];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float4* tw = h == 0 ? tw0 : tw1;
        const uint32_t boff = tile_off(h == 0 ? n0 : n1, kk8);
        const float4 wa = tw[0], wb = tw[1];
        const float r0 = fmaf(wa.x, ya.x, -wa.y * ya.y), i0 = fmaf(wa.x, ya.y, wa.y * ya.x);
        const float r1 = fmaf(wa.z, ya.z, -wa.w * ya.w), i1 = fmaf(wa.z, ya.w, wa.w * ya.z);
        const float r2 = fmaf(wb.x, yb.x, -wb.y * yb.y), i2 = fmaf(wb.x, yb.y, wb.y * yb.x);
        const float r3 = fmaf(wb.z, yb.z, -wb.w * yb.w), i3 = fmaf(wb.z, yb.w, wb.w * yb.z);
        uint4 H, L;
        tc::split_f16x2(r0, i0, H.x, L.x);
        tc::split_f16x2(r1, i1, H.y, L.y);
        tc::split_f16x2(r2, i2, H.z, L.z);
        tc::split_f16x2(r3, i3, H.w, L.w);
        *reinterpret_cast<uint4*>(bhi + boff) = H;
        *reinterpret_cast<uint4*>(bhi + kGOpBytes + boff) = L;
    }
}

struct TileIdx {
    int mt, kt, k0, l0, pkv, plv;  // x tile, y tile, first y and z cell, valid y and z cells of the patch
};
__device__ __forceinline__ TileIdx tile_idx(const GridDesc& d, int64_t tile) {
    TileIdx t;
    t.mt = static_cast<int>(tile % d.n_mt);
    const int64_t rest = tile / d.n_mt;
    t.kt = static_cast<int>(rest % d.n_kt);
    t.k0 = t.kt << d.pk_log2;
    t.l0 = static_cast<int>(rest / d.n_kt) * (kGN >> d.pk_log2);
    t.pkv = min(1 << d.pk_log2, d.ny - t.k0);
    t.plv = min(kGN >> d.pk_log2, d.nz - t.l0);
    return t;
}

template <bool kSplit>
__global__ void __launch_bounds__(kGThreads, 1) grid_mma_kernel(GridDesc d, int32_t* status) {
    extern __shared__ __align__(1024) unsigned char gsm_raw[];
    // stages on a 1024-byte boundary of the shared window (swizzle atoms)
    unsigned char* gsm = gsm_raw + ((1024u - (smem_u32(gsm_raw) & 1023u)) & 1023u);
    uint64_t* bars = reinterpret_cast<uint64_t*>(gsm + d.off_bar);
    uint64_t* afull = bars;                // [sa] stage's copies landed (transaction bytes)
    uint64_t* afree = bars + kGMaxSA;      // [sa] stage's MMAs completed
    uint64_t* bfull = bars + 2 * kGMaxSA;  // [kGSB] B formed (one arrival per epilogue warp)
    uint64_t* bfree = bfull + kGSB;        // [kGSB] B's MMAs completed
    uint64_t* accfull = bfree + kGSB;      // [2] interval's MMAs completed
    uint64_t* accfree = accfull + 2;       // [2] accumulator read by every epilogue warp
    uint64_t* corrfree = accfree + 2;      // correction accumulator read (tile end)
    uint64_t* done = corrfree + 1;         // all MMAs of this CTA completed
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int32_t* abort = reinterpret_cast<volatile int32_t*>(done + 2);
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const bool form = d.form != 0;
    const bool mm = (d.map.bits & kMapMismatch) != 0;
    const int SA = d.sa;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kGMaxSA; ++s) {
            mbar_init(afull + s, 1);
            mbar_init(afree + s, 1);
        }
        for (int b = 0; b < kGSB; ++b) {
            mbar_init(bfull + b, kGEpiWarps);
            mbar_init(bfree + b, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accfull + b, 1);
            mbar_init(accfree + b, kGEpiWarps);
        }
        mbar_init(corrfree, kGEpiWarps);
        mbar_init(done, 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == kGEpiWarps + 1) tc::alloc(tslot, kGTmemCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = *tslot;
    const int NI = d.nc / d.fc;  // fold intervals per tile
    const int n_split = kSplit ? d.n_split : 1;
    const int pkm = (1 << d.pk_log2) - 1;

    if (warp < kGEpiWarps) {
        // ---- B formation (3-D), folds, maps ---------------------------------------
        const int q = warp & 3;           // TMEM lane quarter (rows 32 q .. 32 q + 31)
        const int h = warp >> 2;          // column block (kGColsPerWarp h ..)
        const int t = threadIdx.x;        // 0 .. 255
        const int fp = t & (kGFormPairs - 1);  // column pair this thread forms
        const int fg = t / kGFormPairs;        // 4-mode group of the chunk it forms
        const int fk = fp & pkm;               // y cell of the pair in the patch
        const int fz = (fp >> d.pk_log2) * 2;  // first z cell of the pair in the patch
        const int n0 = fk + (fz << d.pk_log2), n1 = n0 + (1 << d.pk_log2);
        const uint32_t lane_off = static_cast<uint32_t>(32 * q) << 16;
        const float S = grid_scale(d.thdr);
        uint32_t g = 0, gi = 0;
        for (int64_t item = blockIdx.x; item < (kSplit ? d.n_items : d.n_tiles); item += gridDim.x) {
            const int64_t tile = kSplit ? item / n_split : item;
            const int split = kSplit ? static_cast<int>(item - tile * n_split) : 0;
            // the item's fold intervals iv0 .. iv1 - 1 (all of the tile's without a split)
            const int iv0 = kSplit ? NI * split / n_split : 0;
            const int NIl = kSplit ? NI * (split + 1) / n_split - iv0 : NI;
            const TileIdx ti = tile_idx(d, tile);
            // staged table rows this thread reads: y row and (amplitude, psi, z) row
            const int ry = min(fk, ti.pkv - 1);
            const int rz0 = min(fz, ti.plv - 1), rz1 = min(fz + 1, ti.plv - 1);
            const int toff_y = kGPair + ry * kGRowBytes + 32 * fg;
            const int toff_w0 = kGPair + ((1 << d.pk_log2) + rz0) * kGRowBytes + 32 * fg;
            const int toff_w1 = kGPair + ((1 << d.pk_log2) + rz1) * kGRowBytes + 32 * fg;

            // fold of interval gidx: the hi.hi accumulator into the running sum
            // (plain FP32: a few tens of folds per cell); the last fold of a
            // tile adds the correction accumulator and writes the cells
            double lsum = 0.0;  // kMapMismatch: this lane's sum of (K - T)^2 over the tile
            auto fold = [&](uint32_t gidx, bool first, bool last) -> bool {
                const uint32_t b = gidx & 1u;
                // warp-uniform outcome: the TMEM moves below are warp-wide
                if (!__all_sync(0xffffffffu, gwait(accfull + b, (gidx >> 1) & 1u, abort, status))) return false;
                tc::fence_after();
                if (!last) {
#pragma unroll 1
                    for (int blk = 0; blk < kGColsPerWarp / 16; ++blk) {  // 16 columns per TMEM round trip
                        const uint32_t col = static_cast<uint32_t>(kGColsPerWarp * h + 16 * blk);
                        uint32_t p[16], sm[16];
                        tc::ld16(tbase + lane_off + b * kGN + col, p);
                        if (!first) tc::ld16(tbase + lane_off + kGSumCol + col, sm);
                        tc::wait_ld();
                        if (blk == kGColsPerWarp / 16 - 1) {
                            tc::fence_before();
                            __syncwarp();
                            if (lane == 0) tc::mbar_arrive(accfree + b);
                        }
#pragma unroll
                        for (int cc = 0; cc < 16; ++cc)
                            sm[cc] = first ? p[cc] : __float_as_uint(__uint_as_float(sm[cc]) + __uint_as_float(p[cc]));
                        tc::st16(tbase + lane_off + kGSumCol + col, sm);
                    }
                    tc::wait_st();
                } else {
                    const int i = ti.mt * kGM + 32 * q + lane;
#pragma unroll 1
                    for (int blk = 0; blk < kGColsPerWarp / 8; ++blk) {  // 8 columns at a time, then the maps
                        const uint32_t col = static_cast<uint32_t>(kGColsPerWarp * h + 8 * blk);
                        uint32_t p[8], sm[8], cr[8];
                        tc::ld8(tbase + lane_off + b * kGN + col, p);
                        tc::ld8(tbase + lane_off + kGCorrCol + col, cr);
                        if (!first) tc::ld8(tbase + lane_off + kGSumCol + col, sm);
                        tc::wait_ld();
                        if (blk == kGColsPerWarp / 8 - 1) {
                            tc::fence_before();
                            __syncwarp();
                            if (lane == 0) {
                                tc::mbar_arrive(accfree + b);
                                tc::mbar_arrive(corrfree);
                            }
                        }
#pragma unroll
                        for (int cc = 0; cc < 8; ++cc) {
                            float v = __uint_as_float(p[cc]);
                            if (!first) v = __uint_as_float(sm[cc]) + v;
                            v += __uint_as_float(cr[cc]);
                            const int c = static_cast<int>(col) + cc;
                            const int k = ti.k0 + (c & pkm);
                            const int l = ti.l0 + (c >> d.pk_log2);
                            if (i < d.nx && k < d.ny && l < d.nz) {
                                const int64_t o = i + static_cast<int64_t>(d.nx) *
                                                          (k + static_cast<int64_t>(d.ny) * l);
                                if (kSplit) {
                                    d.part[static_cast<int64_t>(split) * d.nx * d.ny * d.nz + o] = v * S;
                                } else {
                                    const float y = v * S + d.map.mu;
                                    map_store(d.map, o, y);
                                    if (mm) lsum += mismatch_store(d.map, o, y);
                                }
                            }
                        }
                    }
                }
                return true;
            };

            bool ok = true;
            if (form) {
                const int c_end = kSplit ? (iv0 + NIl) * d.fc : d.nc;
                for (int c = kSplit ? iv0 * d.fc : 0; c < c_end; ++c, ++g) {
                    const int sb = static_cast<int>(g % kGSB);
                    const int sa = static_cast<int>(g % SA);
                    if (g >= kGSB &&
                        !__all_sync(0xffffffffu, gwait(bfree + sb, ((g / kGSB) - 1u) & 1u, abort, status))) {
                        ok = false;
                        break;
                    }
                    if (!__all_sync(0xffffffffu, gwait(afull + sa, (g / SA) & 1u, abort, status))) {
                        ok = false;
                        break;
                    }
                    const unsigned char* st = gsm + sa * d.a_stage;
                    form_b(gsm + d.off_b + sb * kGPair, reinterpret_cast<const float4*>(st + toff_y),
                           reinterpret_cast<const float4*>(st + toff_w0), reinterpret_cast<const float4*>(st + toff_w1),
                           n0, n1, fg);
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(bfull + sb);
                    if ((c + 1) % d.fc == 0) {
                        const int iv = (c + 1) / d.fc - 1 - (kSplit ? iv0 : 0);  // the item's interval whose chunks are all formed
                        if (iv >= 1) {
                            if (!fold(gi, iv == 1, false)) {
                                ok = false;
                                break;
                            }
                            ++gi;
                        }
                    }
                }
                if (!ok || !fold(gi, NIl == 1, true)) break;
                ++gi;
            } else {
                for (int iv = 0; iv < NIl; ++iv, ++gi) {
                    if (!fold(gi, iv == 0, iv == NIl - 1)) {
                        ok = false;
                        break;
                    }
                }
                if (!ok) break;
            }
            if (mm && !kSplit) {
                // fixed butterfly order, one partial per (tile, warp): the loss
                // does not depend on which CTA took the tile
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
                if (lane == 0) d.map.lpart[tile * kGEpiWarps + warp] = lsum;
            }
        }
    } else if (warp == kGEpiWarps) {
        // ---- MMA issue ------------------------------------------------------------
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_f16_f32(kGM, kGN);
            constexpr uint32_t dhi = tc::smem_desc_sw128_hi(kGSbo);
            constexpr uint32_t tstep = kGOpBytes >> 4;  // one operand tile in descriptor units
            const uint32_t alo0 = tc::smem_desc_sw128_lo(smem_u32(gsm));
            const uint32_t blo0 = tc::smem_desc_sw128_lo(smem_u32(gsm + d.off_b));
            uint32_t g = 0, gi = 0, tile_count = 0;
            uint32_t sa = 0, pa = 0, sb = 0, pb = 0;  // ring stages and their phase parities
            bool ok = true;
            const uint32_t dc = tbase + kGCorrCol;
            for (int64_t item = blockIdx.x; item < (kSplit ? d.n_items : d.n_tiles) && ok; item += gridDim.x, ++tile_count) {
                const int split = kSplit ? static_cast<int>(item % n_split) : 0;
                const int NIl = kSplit ? NI * (split + 1) / n_split - NI * split / n_split : NI;
                // the previous item's correction accumulator has been read
                if (tile_count >= 1 && !gwait(corrfree, (tile_count - 1u) & 1u, abort, status)) {
                    ok = false;
                    break;
                }
                for (int iv = 0; iv < NIl && ok; ++iv, ++gi) {
                    const uint32_t b = gi & 1u;
                    if (gi >= 2 && !gwait(accfree + b, ((gi >> 1) - 1u) & 1u, abort, status)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after();
                    const uint32_t dt = tbase + b * kGN;
                    for (int cc = 0; cc < d.fc; ++cc, ++g) {
                        if (!gwait(afull + sa, pa, abort, status) || (form && !gwait(bfull + sb, pb, abort, status))) {
                            ok = false;
                            break;
                        }
                        tc::fence_after();
                        const uint32_t alo = alo0 + sa * (static_cast<uint32_t>(d.a_stage) >> 4);
                        const uint32_t blo = form ? blo0 + sb * (kGPair >> 4) : alo + (kGPair >> 4);
#pragma unroll
                        for (int ks = 0; ks < kGK / 16; ++ks) {
                            const uint32_t ko = static_cast<uint32_t>(ks) * (kGKStep >> 4);  // 16 K elements
                            const uint64_t ah = tc::desc_of(alo + ko, dhi);
                            const uint64_t al = tc::desc_of(alo + tstep + ko, dhi);
                            const uint64_t bh = tc::desc_of(blo + ko, dhi);
                            const uint64_t bl = tc::desc_of(blo + tstep + ko, dhi);
                            tc::mma_f16(dt, ah, bh, idesc, (cc | ks) != 0 ? 1u : 0u);
                            tc::mma_f16(dc, ah, bl, idesc, (iv | cc | ks) != 0 ? 1u : 0u);
                            tc::mma_f16(dc, al, bh, idesc, 1u);
                        }
                        tc::commit(afree + sa);
                        if (form) tc::commit(bfree + sb);
                        if (++sa == static_cast<uint32_t>(SA)) {
                            sa = 0;
                            pa ^= 1u;
                        }
                        if (++sb == kGSB) {
                            sb = 0;
                            pb ^= 1u;
                        }
                    }
                    if (ok) tc::commit(accfull + b);
                }
                if (ok) atomicAdd(&g_grid_tiles, 1ull);
            }
            // every MMA this CTA issued has completed before TMEM is released
            tc::commit(done);
            mbar_wait_bounded(done, 0);
        }
        __syncwarp();
    } else {
        // ---- bulk copies: A chunks and, per chunk, the tables or B ---------------------
        if (lane == 0) {
            uint32_t g = 0;
            bool ok = true;
            for (int64_t item = blockIdx.x; item < (kSplit ? d.n_items : d.n_tiles) && ok; item += gridDim.x) {
                const int64_t tile = kSplit ? item / n_split : item;
                const int split = kSplit ? static_cast<int>(item - tile * n_split) : 0;
                const TileIdx ti = tile_idx(d, tile);
                const unsigned char* asrc = d.atab + static_cast<int64_t>(ti.mt) * d.nc * kGPair;
                const int c_end = kSplit ? NI * (split + 1) / n_split * d.fc : d.nc;
                for (int c = kSplit ? NI * split / n_split * d.fc : 0; c < c_end; ++c, ++g) {
                    const int sa = static_cast<int>(g % SA);
                    if (g >= static_cast<uint32_t>(SA) &&
                        !gwait(afree + sa, ((g / SA) - 1u) & 1u, abort, status)) {
                        ok = false;
                        break;
                    }
                    unsigned char* dst = gsm + sa * d.a_stage;
                    const unsigned char* ac = asrc + static_cast<int64_t>(c) * kGPair;
                    if (form) {
                        const uint32_t by = static_cast<uint32_t>(ti.pkv) * kGRowBytes;
                        const uint32_t bw = static_cast<uint32_t>(ti.plv) * kGRowBytes;
                        mbar_arrive_expect_tx(afull + sa, kGPair + by + bw);
                        bulk_g2s(dst, ac, kGOpBytes, afull + sa);
                        bulk_g2s(dst + kGOpBytes, ac + kGOpBytes, kGOpBytes, afull + sa);
                        bulk_g2s(dst + kGPair, d.ytab + (static_cast<int64_t>(c) * d.ny + ti.k0) * (kGRowBytes / 8), by,
                                 afull + sa);
                        bulk_g2s(dst + kGPair + (1 << d.pk_log2) * kGRowBytes,
                                 d.wztab + (static_cast<int64_t>(c) * d.nz + ti.l0) * (kGRowBytes / 8), bw,
                                 afull + sa);
                    } else {
                        const unsigned char* bc = d.btab + (static_cast<int64_t>(ti.kt) * d.nc + c) * kGPair;
                        mbar_arrive_expect_tx(afull + sa, 2 * kGPair);
                        bulk_g2s(dst, ac, kGOpBytes, afull + sa);
                        bulk_g2s(dst + kGOpBytes, ac + kGOpBytes, kGOpBytes, afull + sa);
                        bulk_g2s(dst + kGPair, bc, kGOpBytes, afull + sa);
                        bulk_g2s(dst + kGPair + kGOpBytes, bc + kGOpBytes, kGOpBytes, afull + sa);
                    }
                }
            }
            // copies still in flight land before the CTA's shared memory goes away
            for (uint32_t q = g > static_cast<uint32_t>(SA) ? g - SA : 0u; q < g; ++q)
                mbar_wait_bounded(afull + q % SA, (q / SA) & 1u);
        }
        __syncwarp();
    }
    tc::fence_before();
    __syncthreads();
    if (warp == kGEpiWarps + 1) {
        tc::fence_after();
        tc::dealloc(tbase, kGTmemCols);
    }
}

// Tables of one call (workspace).  Work items, flattened:
//   A : (mt, chunk, row, quad of 4 modes) -> one 16-byte row segment of the
//       hi and of the lo tile ((re, -im) pairs of e^{2 pi i a_x X_i}; rows
//       beyond nx are zero);
//   3-D (form):  Y : (chunk, k, m) -> e^{2 pi i a_jy Y_k},
//                W : (chunk, l, m) -> (A_j / S) e^{2 pi i (psi_j + a_jz Z_l)}, j = 32 chunk + m;
//   2-D (load):  B : (kt, chunk, column, quad) -> (A_j / S) e^{2 pi i (psi_j + a_jy Y_k + a_jz Z_0)}
//                as (re, im) hi and lo tiles (columns beyond ny are zero).
__global__ void grid_prep_kernel(GridPrep p) {
    const int64_t nA = static_cast<int64_t>(p.n_mt) * p.nc * kGM * 8;
    const int64_t nY = p.form ? static_cast<int64_t>(p.ny) * p.n_pad : static_cast<int64_t>(p.n_kt) * p.nc * kGN * 8;
    const int64_t nW = p.form ? static_cast<int64_t>(p.nz) * p.n_pad : 0;
    const float s_inv = 1.0f / grid_scale(p.thdr);  // exact: a power of two
    const bool has_z = p.dim > 2;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; idx < nA + nY + nW;
         idx += stride) {
        if (idx < nA || (!p.form && idx < nA + nY)) {
            // an operand tile row segment: A (x phasors) or, in 2-D, B
            const bool is_a = idx < nA;
            const int64_t u = is_a ? idx : idx - nA;
            const int quad = static_cast<int>(u & 7);
            const int r = static_cast<int>((u >> 3) & 127);
            const int64_t rest = u >> 10;
            const int c = static_cast<int>(rest % p.nc);
            const int64_t tt = rest / p.nc;  // mt or kt
            const int64_t i = tt * kGM + r;  // x or y cell
            float v[8];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int j = c * kGModes + quad * 4 + m;
                float cs = 0.0f, sn = 0.0f;
                if (is_a) {
                    if (i < p.nx) {
                        const float4 c0 = __ldg(p.cold + 2 * j);
                        sincospif(2.0f * turns_axis(c0.x, c0.y, __ldg(p.X + i)), &sn, &cs);
                    }
                    v[2 * m] = cs;
                    v[2 * m + 1] = -sn;
                } else {
                    if (i < p.ny) {
                        const float4 c0 = __ldg(p.cold + 2 * j);
                        const float4 c1 = __ldg(p.cold + 2 * j + 1);
                        const float tz = psi_z_turns(c1, has_z ? __ldg(p.Z) : 0.0f, has_z);
                        const float t = frac_turn(turns_axis(c0.z, c0.w, __ldg(p.Y + i)) + tz);
                        sincospif(2.0f * t, &sn, &cs);
                        const float amp = __ldg(&p.hot[j].w) * s_inv;
                        cs *= amp;
                        sn *= amp;
                    }
                    v[2 * m] = cs;
                    v[2 * m + 1] = sn;
                }
            }
            uint4 H, L;
            tc::split_f16x2(v[0], v[1], H.x, L.x);
            tc::split_f16x2(v[2], v[3], H.y, L.y);
            tc::split_f16x2(v[4], v[5], H.z, L.z);
            tc::split_f16x2(v[6], v[7], H.w, L.w);
            unsigned char* o = (is_a ? p.atab : p.btab) + (tt * p.nc + c) * static_cast<int64_t>(kGPair) +
                               tile_off(r, quad);
            *reinterpret_cast<uint4*>(o) = H;
            *reinterpret_cast<uint4*>(o + kGOpBytes) = L;
        } else if (idx < nA + nY) {
            const int64_t u = idx - nA;  // (chunk, k, m)
            const int m = static_cast<int>(u % kGModes);
            const int64_t k = (u / kGModes) % p.ny;
            const int c = static_cast<int>(u / (static_cast<int64_t>(kGModes) * p.ny));
            const int j = c * kGModes + m;
            const float4 c0 = __ldg(p.cold + 2 * j);
            float cs, sn;
            sincospif(2.0f * turns_axis(c0.z, c0.w, __ldg(p.Y + k)), &sn, &cs);
            p.ytab[(u / kGModes) * (kGRowBytes / 8) + m] = make_float2(cs, sn);
        } else {
            const int64_t u = idx - nA - nY;  // (chunk, l, m)
            const int m = static_cast<int>(u % kGModes);
            const int64_t l = (u / kGModes) % p.nz;
            const int c = static_cast<int>(u / (static_cast<int64_t>(kGModes) * p.nz));
            const int j = c * kGModes + m;
            const float4 c1 = __ldg(p.cold + 2 * j + 1);
            const float amp = __ldg(&p.hot[j].w) * s_inv;
            float cs, sn;
            sincospif(2.0f * psi_z_turns(c1, has_z ? __ldg(p.Z + l) : 0.0f, has_z), &sn, &cs);
            p.wztab[(u / kGModes) * (kGRowBytes / 8) + m] = make_float2(amp * cs, amp * sn);
        }
    }
}

// Mode-split grids: per cell the partial fields of the splits, added in split
// order (a fixed order), plus mu, then the maps; with the mismatch bit every
// block also writes its sum of (K - T)^2 to lpart.
__global__ void __launch_bounds__(256) grid_split_finalize(const float* __restrict__ part, int n_split, int64_t n,
                                                           MapDev map) {
    const int64_t o = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const bool mm = (map.bits & kMapMismatch) != 0;
    double l = 0.0;
    if (o < n) {
        float s = 0.0f, e = 0.0f;
        for (int k = 0; k < n_split; ++k) two_sum_acc(s, e, part[static_cast<int64_t>(k) * n + o]);
        const float y = (s + e) + map.mu;
        map_store(map, o, y);
        if (mm) l = mismatch_store(map, o, y);
    }
    if (mm) {
        __shared__ double red[8];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < 8; ++w) t += red[w];
            map.lpart[blockIdx.x] = t;
        }
    }
}

// D[128][128] = sum_K A[128][K] B[128][K] (FP16 inputs, K-contiguous rows,
// K = 64 k_chunks, FP32 result row-major) through the same layout,
// descriptors and TMEM path as the grid kernel.  One CTA of 128 threads.
__global__ void __launch_bounds__(128, 1) mma_probe_kernel(const uint16_t* A, const uint16_t* B, int32_t k_chunks,
                                                             float* D, int32_t* status) {
    __shared__ __align__(1024) unsigned char sm_raw[2 * kGOpBytes + 1024];
    // operand tiles on a 1024-byte boundary of the shared window (swizzle atoms)
    unsigned char* sm = sm_raw + ((1024u - (smem_u32(sm_raw) & 1023u)) & 1023u);
    __shared__ uint64_t bar;
    __shared__ uint32_t slot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    if (warp == 0) tc::alloc(&slot, 128);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = slot;
    const int K = kGK * k_chunks;
    bool ok = true;
    for (int ch = 0; ch < k_chunks; ++ch) {
        // canonical layout of the 128 x 64 chunk of A and of B
        for (int e = threadIdx.x; e < kGM * kGK; e += blockDim.x) {
            const int r = e / kGK, kk = e % kGK;
            const uint32_t off = tile_off(r, kk >> 3) + static_cast<uint32_t>(kk & 7) * 2u;
            *reinterpret_cast<uint16_t*>(sm + off) = A[static_cast<int64_t>(r) * K + ch * kGK + kk];
            *reinterpret_cast<uint16_t*>(sm + kGOpBytes + off) = B[static_cast<int64_t>(r) * K + ch * kGK + kk];
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc::fence_after();
            const uint32_t sa = smem_u32(sm);
            for (int ks = 0; ks < kGK / 16; ++ks) {
                const uint32_t ko = static_cast<uint32_t>(ks) * kGKStep;
                tc::mma_f16(tbase, tc::smem_desc_sw128(sa + ko, kGSbo), tc::smem_desc_sw128(sa + kGOpBytes + ko, kGSbo),
                            tc::idesc_f16_f32(kGM, kGN), (ch | ks) != 0 ? 1u : 0u);
            }
            tc::commit(&bar);
        }
        if (!mbar_wait_bounded(&bar, static_cast<uint32_t>(ch) & 1u)) {
            if (threadIdx.x == 0) atomicOr(status, 2);
            ok = false;
        }
        tc::fence_after();
        __syncthreads();  // the chunk's shared data is no longer read
        if (!ok) break;
    }
    if (ok) {
        for (int cb = 0; cb < kGN; cb += 32) {
            uint32_t r[32];
            tc::ld32(tbase + (static_cast<uint32_t>(32 * warp) << 16) + cb, r);
            tc::wait_ld();
            const int row = 32 * warp + lane;
            for (int c = 0; c < 32; ++c) D[row * kGN + cb + c] = __uint_as_float(r[c]);
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::dealloc(tbase, 128);
    }
}

int g_num_sms = 0;

// Layout of one grid synthesis: mode, patch, tiles, shared-memory rings and
// workspace tables.
struct GridPlan {
    bool form;
    int pk_log2, n_mt, n_kt, n_lt, nc, sa, a_stage, off_b, off_bar, smem;
    int max_split;  // mode splits for grids of few tiles (the launch takes at most one per fold interval)
    int64_t n_tiles, a_bytes, y_bytes, w_bytes, b_bytes, part_bytes;
};

// Grids of at most 64 tiles split each tile's modes over up to 8 CTAs, so
// that about 128 work items fill the GPU.
constexpr int kGMaxSplit = 8;
constexpr int64_t kGSplitItems = 128;

GridPlan grid_plan(int32_t nx, int32_t ny, int32_t nz, int64_t n_pad) {
    GridPlan g{};
    g.form = nz > 1;
    g.nc = static_cast<int>(n_pad / kGModes);
    g.n_mt = (nx + kGM - 1) / kGM;
    if (g.form) {
        // patch 2^p y-cells by 128 / 2^p z-cells (p = 2 .. 6): fewest wasted
        // columns, then the fewest staged table rows
        double best = 1e300;
        for (int pk = 2; pk <= 6; ++pk) {
            const int64_t PK = int64_t(1) << pk, PL = kGN / PK;
            const double cols = double((ny + PK - 1) / PK * PK) * double((nz + PL - 1) / PL * PL);
            const double w = cols / (double(ny) * double(nz)) + 1e-4 * double(PK + PL);
            if (w < best) {
                best = w;
                g.pk_log2 = pk;
            }
        }
        const int tb = ((1 << g.pk_log2) + (kGN >> g.pk_log2)) * kGRowBytes;
        g.a_stage = (kGPair + tb + 1023) / 1024 * 1024;  // swizzle atoms start on 1024-byte boundaries
        g.sa = std::min(kGMaxSA, (kGSmemMax - kGAlignPad - kGBarBytes - kGSB * kGPair) / g.a_stage);
        g.off_b = g.sa * g.a_stage;
        g.off_bar = g.off_b + kGSB * kGPair;
    } else {
        g.pk_log2 = 7;
        g.a_stage = 2 * kGPair;
        g.sa = std::min(kGMaxSA, (kGSmemMax - kGAlignPad - kGBarBytes) / g.a_stage);
        g.off_b = g.sa * g.a_stage;
        g.off_bar = g.off_b;
    }
    g.smem = g.off_bar + kGBarBytes + kGAlignPad;
    g.n_kt = (ny + (1 << g.pk_log2) - 1) >> g.pk_log2;
    const int PL = kGN >> g.pk_log2;
    g.n_lt = (nz + PL - 1) / PL;
    g.n_tiles = int64_t(g.n_mt) * g.n_kt * g.n_lt;
    g.max_split = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(kGMaxSplit, kGSplitItems / g.n_tiles)));
    g.part_bytes = g.max_split > 1 ? align256(int64_t(g.max_split) * nx * ny * nz * 4) : 0;
    g.a_bytes = align256(int64_t(g.n_mt) * g.nc * kGPair);
    if (g.form) {
        g.y_bytes = align256(int64_t(g.nc) * ny * kGRowBytes);
        g.w_bytes = align256(int64_t(g.nc) * nz * kGRowBytes);
    } else {
        g.b_bytes = align256(int64_t(g.n_kt) * g.nc * kGPair);
    }
    return g;
}

}  // namespace

size_t grid_ws_bytes(int32_t nx, int32_t ny, int32_t nz, int64_t n_pad) {
    const GridPlan g = grid_plan(nx, ny, nz, n_pad);
    return static_cast<size_t>(g.a_bytes + g.y_bytes + g.w_bytes + g.b_bytes + g.part_bytes);
}

int launch_synth_grid(const void* table, int64_t n_modes, int32_t dim, const GridGeom& gg, const MapDev& map,
                      void* ws, int32_t fc, int32_t* status, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const unsigned char* tb = static_cast<const unsigned char*>(table);
    const TableLayout TL = table_layout(n_modes);
    if (g_num_sms == 0) {
        int dev = 0, sms = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(grid_mma_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGSmemMax);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(grid_mma_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGSmemMax);
        if (e != cudaSuccess) return e;
        g_num_sms = sms;
    }
    const GridPlan gp = grid_plan(gg.nx, gg.ny, gg.nz, TL.n_pad);
    unsigned char* w = static_cast<unsigned char*>(ws);
    GridPrep p{};
    p.thdr = reinterpret_cast<const TableHeader*>(tb);
    p.hot = reinterpret_cast<const float4*>(tb + TL.off_hot);
    p.cold = reinterpret_cast<const float4*>(tb + TL.off_cold);
    p.X = gg.X;
    p.Y = gg.Y;
    p.Z = gg.Z;
    p.nx = gg.nx;
    p.ny = gg.ny;
    p.nz = gg.nz;
    p.n_pad = static_cast<int32_t>(TL.n_pad);
    p.nc = gp.nc;
    p.n_mt = gp.n_mt;
    p.n_kt = gp.n_kt;
    p.dim = dim;
    p.form = gp.form ? 1 : 0;
    p.atab = w;
    if (gp.form) {
        p.ytab = reinterpret_cast<float2*>(w + gp.a_bytes);
        p.wztab = reinterpret_cast<float2*>(w + gp.a_bytes + gp.y_bytes);
    } else {
        p.btab = w + gp.a_bytes;
    }
    const int64_t items = int64_t(gp.n_mt) * gp.nc * kGM * 8 +
                          (gp.form ? (int64_t(gg.ny) + gg.nz) * TL.n_pad : int64_t(gp.n_kt) * gp.nc * kGN * 8);
    const int pb = 256;
    const int64_t pg = std::min<int64_t>((items + pb - 1) / pb, int64_t(g_num_sms) * 16);
    grid_prep_kernel<<<static_cast<unsigned>(pg), pb, 0, st>>>(p);
    count_launches(1);

    GridDesc d{};
    d.atab = p.atab;
    d.btab = p.btab;
    d.ytab = p.ytab;
    d.wztab = p.wztab;
    d.thdr = p.thdr;
    d.nx = gg.nx;
    d.ny = gg.ny;
    d.nz = gg.nz;
    d.n_pad = p.n_pad;
    d.nc = gp.nc;
    d.fc = fc;
    while (d.fc > 1 && gp.nc % d.fc != 0) d.fc >>= 1;  // whole fold intervals per tile
    d.n_mt = gp.n_mt;
    d.n_kt = gp.n_kt;
    d.n_lt = gp.n_lt;
    d.pk_log2 = gp.pk_log2;
    d.n_tiles = gp.n_tiles;
    d.n_split = std::min(gp.max_split, gp.nc / d.fc);  // whole fold intervals per split
    d.n_items = d.n_tiles * d.n_split;
    d.part = d.n_split > 1 ? reinterpret_cast<float*>(w + gp.a_bytes + gp.y_bytes + gp.w_bytes + gp.b_bytes)
                           : nullptr;
    d.form = p.form;
    d.sa = gp.sa;
    d.a_stage = gp.a_stage;
    d.off_b = gp.off_b;
    d.off_bar = gp.off_bar;
    d.map = map;
    const int64_t grid = std::min<int64_t>(d.n_items, g_num_sms);
    if (d.n_split > 1)
        grid_mma_kernel<true><<<static_cast<unsigned>(grid), kGThreads, gp.smem, st>>>(d, status);
    else
        grid_mma_kernel<false><<<static_cast<unsigned>(grid), kGThreads, gp.smem, st>>>(d, status);
    count_launches(1);
    const int64_t n = int64_t(gg.nx) * gg.ny * gg.nz;
    const int64_t fin_blocks = (n + 255) / 256;
    if (d.n_split > 1) {
        grid_split_finalize<<<static_cast<unsigned>(fin_blocks), 256, 0, st>>>(d.part, d.n_split, n, map);
        count_launches(1);
    }
    if (map.bits & kMapMismatch) {
        const int e = launch_loss_sum(map.lpart, d.n_split > 1 ? fin_blocks : d.n_tiles * kGEpiWarps, map.inv_n_mean,
                                      map.loss, st);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

int64_t grid_loss_partials(int32_t nx, int32_t ny, int32_t nz) {
    // at most: one per (tile, warp) without a split, one per finalize block with one
    const GridPlan g = grid_plan(nx, ny, nz, kGModes * 4);
    return std::max<int64_t>(g.n_tiles * kGEpiWarps, (int64_t(nx) * ny * nz + 255) / 256);
}

int64_t grid_tiles(int32_t nx, int32_t ny, int32_t nz) { return grid_plan(nx, ny, nz, kGModes * 4).n_tiles; }

int take_grid_tiles(unsigned long long* tiles) {
    unsigned long long v = 0ull;
    const unsigned long long zero = 0ull;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_grid_tiles, sizeof(v));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_grid_tiles, &zero, sizeof(zero));
    if (e != cudaSuccess) return e;
    *tiles = v;
    return cudaSuccess;
}

int launch_mma_probe(const uint16_t* A, const uint16_t* B, int32_t k_chunks, float* D, int32_t* status,
                     void* stream) {
    mma_probe_kernel<<<1, 128, 0, static_cast<cudaStream_t>(stream)>>>(A, B, k_chunks, D, status);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace grf
