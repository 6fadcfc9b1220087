// Adjoint of the spectral field sum on Cartesian grids with the
// fifth-generation tensor cores (derivative of Eq. DiscreteFT, Sec. 4.1).
//
// Per mode j the adjoint needs, with theta_ij = 2 pi (a_j . x_i + psi_j),
//     E_j = sum_i g_i e^{i theta_ij}        (S_cos = Re E_j, S_sin = Im E_j),
//     S_c[j] = sum_i g_i x_ic sin theta_ij  (c = x, y, z).
// On the grid cell (i, k, l) the phasor factorises,
//     e^{i theta} = Xp_j(X_i) Yp_j(Y_k) Zp_j(Z_l),  Zp carrying psi_j,
// so E_j = sum_{k,l} Yp_j(Y_k) Zp_j(Z_l) D_j(k, l) with
//     D_j(k, l) = sum_i Xp_j(X_i) g(i, k, l),
// a real matrix product over the x cells: rows = 128 modes (TMEM lanes),
// columns = 64 (y, z) cells of a patch and the same 64 cells weighted by
// (X_i - X_0), K = 64 x cells.  A unit (one mode tile, one x chunk, one
// patch) fills two accumulators, the products with cos(2 pi a_jx X_i) and
// with sin(2 pi a_jx X_i).  The epilogue (one thread per mode) contracts the
// unit's 64 columns with Yp and Zp on the CUDA cores; the y and z weights
// enter there, so only x needs weighted columns.
//
// Precision as in the forward grid kernel: both operands are split into FP16
// hi + lo (g scaled by a power of two to |g| < 1, the x weights likewise),
// three products hi.hi + hi.lo + lo.hi per term, FP32 accumulation over the
// 64 x cells of a unit.  The epilogue's FP32 sums of a unit are folded into
// compensated (two-float) running sums, written as FP64 partials per (group,
// mode) and reduced in a fixed order by the CUDA-core adjoint's own
// reduction, which also applies the chain rule.
//
// Work: CTA c owns mode tile c mod T (T = n_pad / 128) and group c / T, a
// contiguous range of the (x chunk, y block, z block) units.  The mode
// tile's A tiles for the current x chunk and the phasor rows of the current
// y block stay in shared memory for a run of units; the B tiles stream
// through a ring of three stages, read by the T CTAs of a group at about the
// same time (L2).  Roles: warps 0-15 epilogue (warp w: TMEM lanes
// 32 (w mod 4) .., columns 16 (w / 4) ..), warp 16 issues the MMAs (one
// thread), warp 17 issues the bulk copies and owns TMEM.  TMEM (512 columns):
// two unit buffers of 256 (cos: plain, weighted; sin: plain, weighted).
// Every mbarrier wait is bounded and reports through the status word.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "device_common.cuh"
#include "grid_common.cuh"
#include "tcgen05.cuh"

namespace grf {

// Units computed by the grid adjoint since the last grf_take_grid_adjoint_units.
static __device__ unsigned long long g_grid_adj_units;

namespace {

using gridc::gwait;
using gridc::psi_z_turns;
using gridc::tile_off;

constexpr int kAM = 128;                          // modes per tile (TMEM lanes)
constexpr int kAYZ = 64;                          // (y, z) cells per unit
constexpr int kAX = gridc::kK;                    // x cells per unit (K)
constexpr int kAEpi = 16;                         // epilogue warps
constexpr int kAThreads = 32 * (kAEpi + 2);
constexpr int kACols = kAYZ / (kAEpi / 4);        // columns of a unit per epilogue warp
constexpr int kABStages = 3;
constexpr int kAStageA = 4 * gridc::kTileBytes;   // cos hi, cos lo, sin hi, sin lo
constexpr int kAStageB = 2 * gridc::kTileBytes;   // hi, lo (rows: 64 cells, 64 weighted cells)
constexpr int kAYRow = kAM * 8;                   // one staged y row: 128 modes x (cos, sin)
constexpr int kAOffB = kAStageA;
constexpr int kAOffY = kAOffB + kABStages * kAStageB;
constexpr int kAOffYw = kAOffY + kAYZ * kAYRow;   // y weights of the run's rows (patches of 64 x 1 cells)
constexpr int kAOffBar = kAOffYw + kAYZ * 4;
constexpr int kABarBytes = 256;
constexpr int kASmem = kAOffBar + kABarBytes + 1024;  // + room to align the stages to 1024 bytes
constexpr uint32_t kATmemCols = 512;
constexpr int kAScanBlocks = 256;                 // partial sums of g (fixed: a fixed summation order)
constexpr int kAMaxCtas = 256;                    // bound on (groups x mode tiles) when T <= 256
static_assert(kASmem <= gridc::kSmemMax, "shared memory of the grid adjoint");
static_assert(kACols == 16 && kAYZ == 64 && kAM == 128, "epilogue layout");
static_assert(4 * kAM * 5 * 8 <= kAStageA, "final combine fits in the A stage");

struct AdjDesc {
    const unsigned char* atab;  // [T][n_kc] x kAStageA
    const unsigned char* btab;  // [units] x kAStageB
    const float2* ytab;         // [ny][n_pad] (cos, sin) 2 pi a_jy Y_k
    const float2* ztab;         // [nz][n_pad] (cos, sin) 2 pi (a_jz Z_l + psi_j)
    const float* yw;            // [ny] Y_k - Y_0
    const float* zw;            // [nz] Z_l - Z_0 (0 without a z axis)
    const float* scal;          // [2] g scale, x-weight scale (written by the prep kernel)
    const float* X;
    const float* Y;
    const float* Z;             // nullptr without a z axis
    double* part;               // [groups][n_pad][5]
    int32_t ny, nz, n_pad, n_kc, n_yb, n_lt, py_log2, n_mt, groups;
    int32_t units;              // per mode tile: n_kc n_yb n_lt
};

// Walks a CTA's units u0 .. u1 - 1 in order: z block lt fastest, then y
// block yb, then x chunk kc (no divisions in the loops).
struct UnitIter {
    int32_t lt, yb, kc;
    __device__ __forceinline__ UnitIter(int32_t u, const AdjDesc& d) {
        lt = u % d.n_lt;
        const int32_t combo = u / d.n_lt;
        yb = combo % d.n_yb;
        kc = combo / d.n_yb;
    }
    __device__ __forceinline__ void next(const AdjDesc& d) {
        if (++lt == d.n_lt) {
            lt = 0;
            if (++yb == d.n_yb) {
                yb = 0;
                ++kc;
            }
        }
    }
};

struct AdjPrep {
    const TableHeader* thdr;
    const float4* cold;
    const float* X;
    const float* Y;
    const float* Z;
    const float* gY;
    const float* gmax;  // [kAScanBlocks]
    const float* xmax;  // [kAScanBlocks]
    unsigned char* atab;
    unsigned char* btab;
    float2* ytab;
    float2* ztab;
    float* yw;
    float* zw;
    float* scal;
    int32_t nx, ny, nz, n_pad, n_kc, n_yb, n_lt, py_log2, n_mt;
    int64_t units;
};

// Block-wide reduction in a fixed order (warp butterflies, then the warp
// results in warp order); the result is valid in thread 0.
template <class T, class Op>
__device__ __forceinline__ T block_reduce(T v, Op op, T* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, off));
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < static_cast<int>(blockDim.x >> 5); ++w) v = op(v, sh[w]);
    __syncthreads();
    return v;
}

// Per block: max |g|, the sum of g (compensated per thread, FP64 across the
// block) and max |X_i - X_0|.
__global__ void __launch_bounds__(256) adj_scan_kernel(const float* g, int64_t n, const float* X, int32_t nx,
                                                        float* gmax, double* gsum, float* xmax) {
    __shared__ float shf[8];
    __shared__ double shd[8];
    float mx = 0.0f, sh = 0.0f, sl = 0.0f, xm = 0.0f;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float v = __ldg(g + i);
        mx = fmaxf(mx, fabsf(v));
        two_sum_acc(sh, sl, v);
    }
    const float x0 = __ldg(X);
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < nx; i += stride)
        xm = fmaxf(xm, fabsf(__ldg(X + i) - x0));
    const auto fmax_op = [](float a, float b) { return fmaxf(a, b); };
    const auto add_op = [](double a, double b) { return a + b; };
    mx = block_reduce(mx, fmax_op, shf);
    xm = block_reduce(xm, fmax_op, shf);
    const double s = block_reduce(static_cast<double>(sh) + static_cast<double>(sl), add_op, shd);
    if (threadIdx.x == 0) {
        gmax[blockIdx.x] = mx;
        xmax[blockIdx.x] = xm;
        gsum[blockIdx.x] = s;
    }
}

// Tables of one adjoint call (workspace).  Work items, flattened:
//   A : (mode tile, x chunk, row, 8-cell segment) -> cos and sin of
//       2 pi a_jx X_i as hi and lo tiles (x beyond nx: 0);
//   Y : (k, slot) -> (cos, sin) 2 pi a_jy Y_k;
//   Z : (l, slot) -> (cos, sin) 2 pi (a_jz Z_l + psi_j);
//   B : (unit, patch cell, 8-cell segment) -> s g and s g (X_i - X_0) t as hi
//       and lo tiles (rows 0-63 and 64-127; cells outside the grid: 0);
//   W : Y_k - Y_0 and Z_l - Z_0.
// s and t are the powers of two that bring max |g| and max |X_i - X_0|
// below 1 (from the scan's per-block maxima; every block derives the same).
__global__ void __launch_bounds__(256) adj_prep_kernel(AdjPrep p) {
    __shared__ float shf[8];
    float gm = 0.0f, xm = 0.0f;
    for (int b = threadIdx.x; b < kAScanBlocks; b += blockDim.x) {
        gm = fmaxf(gm, p.gmax[b]);
        xm = fmaxf(xm, p.xmax[b]);
    }
    const auto fmax_op = [](float a, float b) { return fmaxf(a, b); };
    gm = block_reduce(gm, fmax_op, shf);
    xm = block_reduce(xm, fmax_op, shf);
    __shared__ float sc[2];
    if (threadIdx.x == 0) {
        sc[0] = gridc::pow2_scale_below_one(gm);
        sc[1] = gridc::pow2_scale_below_one(xm);
        if (blockIdx.x == 0) {
            p.scal[0] = sc[0];
            p.scal[1] = sc[1];
        }
    }
    __syncthreads();
    const float gs = sc[0], xs = sc[1];
    const bool has_z = p.Z != nullptr;
    const float x0 = __ldg(p.X);
    const int py = 1 << p.py_log2;
    const int64_t nA = static_cast<int64_t>(p.n_mt) * p.n_kc * kAM * 8;
    const int64_t nY = static_cast<int64_t>(p.ny) * p.n_pad;
    const int64_t nZ = static_cast<int64_t>(p.nz) * p.n_pad;
    const int64_t nB = p.units * kAYZ * 8;
    const int64_t nW = static_cast<int64_t>(p.ny) + p.nz;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; idx < nA + nY + nZ + nB + nW;
         idx += stride) {
        if (idx < nA) {
            const int kk8 = static_cast<int>(idx & 7);
            const int r = static_cast<int>((idx >> 3) & (kAM - 1));
            const int64_t rest = idx >> 10;  // mode tile * n_kc + x chunk
            const int kc = static_cast<int>(rest % p.n_kc);
            const int m = static_cast<int>(rest / p.n_kc) * kAM + r;
            const float4 c0 = __ldg(p.cold + 2 * m);
            float cs[8], sn[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int x = kc * kAX + kk8 * 8 + e;
                cs[e] = 0.0f;
                sn[e] = 0.0f;
                if (x < p.nx) sincospif(2.0f * turns_axis(c0.x, c0.y, __ldg(p.X + x)), &sn[e], &cs[e]);
            }
            uint4 CH, CL, SH, SL;
            tc::split_f16x2(cs[0], cs[1], CH.x, CL.x);
            tc::split_f16x2(cs[2], cs[3], CH.y, CL.y);
            tc::split_f16x2(cs[4], cs[5], CH.z, CL.z);
            tc::split_f16x2(cs[6], cs[7], CH.w, CL.w);
            tc::split_f16x2(sn[0], sn[1], SH.x, SL.x);
            tc::split_f16x2(sn[2], sn[3], SH.y, SL.y);
            tc::split_f16x2(sn[4], sn[5], SH.z, SL.z);
            tc::split_f16x2(sn[6], sn[7], SH.w, SL.w);
            unsigned char* o = p.atab + rest * kAStageA + tile_off(r, kk8);
            *reinterpret_cast<uint4*>(o) = CH;
            *reinterpret_cast<uint4*>(o + gridc::kTileBytes) = CL;
            *reinterpret_cast<uint4*>(o + 2 * gridc::kTileBytes) = SH;
            *reinterpret_cast<uint4*>(o + 3 * gridc::kTileBytes) = SL;
        } else if (idx < nA + nY) {
            const int64_t u = idx - nA;
            const int m = static_cast<int>(u % p.n_pad);
            const int64_t k = u / p.n_pad;
            const float4 c0 = __ldg(p.cold + 2 * m);
            float cs, sn;
            sincospif(2.0f * turns_axis(c0.z, c0.w, __ldg(p.Y + k)), &sn, &cs);
            p.ytab[u] = make_float2(cs, sn);
        } else if (idx < nA + nY + nZ) {
            const int64_t u = idx - nA - nY;
            const int m = static_cast<int>(u % p.n_pad);
            const int64_t l = u / p.n_pad;
            const float4 c1 = __ldg(p.cold + 2 * m + 1);
            float cs, sn;
            sincospif(2.0f * psi_z_turns(c1, has_z ? __ldg(p.Z + l) : 0.0f, has_z), &sn, &cs);
            p.ztab[u] = make_float2(cs, sn);
        } else if (idx < nA + nY + nZ + nB) {
            const int64_t v = idx - nA - nY - nZ;
            const int kk8 = static_cast<int>(v & 7);
            const int r = static_cast<int>((v >> 3) & (kAYZ - 1));
            const int64_t u = v >> 9;  // unit
            const int64_t combo = u / p.n_lt;
            const int lt = static_cast<int>(u % p.n_lt);
            const int yb = static_cast<int>(combo % p.n_yb);
            const int kc = static_cast<int>(combo / p.n_yb);
            const int k = yb * py + (r & (py - 1));
            const int l = lt * (kAYZ >> p.py_log2) + (r >> p.py_log2);
            const bool valid = k < p.ny && l < p.nz;
            const int64_t row = valid ? static_cast<int64_t>(p.nx) * (k + static_cast<int64_t>(p.ny) * l) : 0;
            float gv[8], wv[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int x = kc * kAX + kk8 * 8 + e;
                gv[e] = 0.0f;
                wv[e] = 0.0f;
                if (valid && x < p.nx) {
                    gv[e] = __ldg(p.gY + row + x) * gs;
                    wv[e] = gv[e] * ((__ldg(p.X + x) - x0) * xs);
                }
            }
            uint4 GH, GL, WH, WL;
            tc::split_f16x2(gv[0], gv[1], GH.x, GL.x);
            tc::split_f16x2(gv[2], gv[3], GH.y, GL.y);
            tc::split_f16x2(gv[4], gv[5], GH.z, GL.z);
            tc::split_f16x2(gv[6], gv[7], GH.w, GL.w);
            tc::split_f16x2(wv[0], wv[1], WH.x, WL.x);
            tc::split_f16x2(wv[2], wv[3], WH.y, WL.y);
            tc::split_f16x2(wv[4], wv[5], WH.z, WL.z);
            tc::split_f16x2(wv[6], wv[7], WH.w, WL.w);
            unsigned char* o = p.btab + u * kAStageB;
            *reinterpret_cast<uint4*>(o + tile_off(r, kk8)) = GH;
            *reinterpret_cast<uint4*>(o + gridc::kTileBytes + tile_off(r, kk8)) = GL;
            *reinterpret_cast<uint4*>(o + tile_off(kAYZ + r, kk8)) = WH;
            *reinterpret_cast<uint4*>(o + gridc::kTileBytes + tile_off(kAYZ + r, kk8)) = WL;
        } else {
            const int64_t w = idx - nA - nY - nZ - nB;
            if (w < p.ny) {
                p.yw[w] = __ldg(p.Y + w) - __ldg(p.Y);
            } else {
                const int64_t l = w - p.ny;
                p.zw[l] = has_z ? __ldg(p.Z + l) - __ldg(p.Z) : 0.0f;
            }
        }
    }
}

__global__ void __launch_bounds__(kAThreads, 1) grid_adj_kernel(AdjDesc d, int32_t* status) {
    extern __shared__ __align__(1024) unsigned char asm_raw[];
    // stages on a 1024-byte boundary of the shared window (swizzle atoms)
    unsigned char* gsm = asm_raw + ((1024u - (smem_u32(asm_raw) & 1023u)) & 1023u);
    uint64_t* bars = reinterpret_cast<uint64_t*>(gsm + kAOffBar);
    uint64_t* afull = bars;                // A tiles and y rows of a run landed (transaction bytes)
    uint64_t* afree = bars + 1;            // the run's MMAs completed
    uint64_t* yfree = bars + 2;            // the run's y rows read (one arrival per epilogue warp)
    uint64_t* bfull = bars + 3;            // [kABStages] B stage landed
    uint64_t* bfree = bfull + kABStages;   // [kABStages] B stage's MMAs completed
    uint64_t* accfull = bfree + kABStages; // [2] unit's MMAs completed
    uint64_t* accfree = accfull + 2;       // [2] accumulators read by every epilogue warp
    uint64_t* done = accfree + 2;          // all MMAs of this CTA completed
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int32_t* abort = reinterpret_cast<volatile int32_t*>(done + 2);
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int mt = static_cast<int>(blockIdx.x % d.n_mt);
    const int grp = static_cast<int>(blockIdx.x / d.n_mt);
    const int32_t u0 = static_cast<int32_t>(static_cast<int64_t>(d.units) * grp / d.groups);
    const int32_t u1 = static_cast<int32_t>(static_cast<int64_t>(d.units) * (grp + 1) / d.groups);
    const int py = 1 << d.py_log2;

    if (threadIdx.x == 0) {
        mbar_init(afull, 1);
        mbar_init(afree, 1);
        mbar_init(yfree, kAEpi);
        for (int s = 0; s < kABStages; ++s) {
            mbar_init(bfull + s, 1);
            mbar_init(bfree + s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accfull + b, 1);
            mbar_init(accfree + b, kAEpi);
        }
        mbar_init(done, 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == kAEpi + 1) tc::alloc(tslot, kATmemCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = *tslot;

    if (warp < kAEpi) {
        // ---- epilogue: contract the unit's columns with the y and z phasors --------
        const int q = warp & 3;   // TMEM lane quarter: modes 32 q .. 32 q + 31 of the tile
        const int h = warp >> 2;  // columns kACols h .. of the unit
        const int ml = 32 * q + lane;
        const int m = mt * kAM + ml;
        const uint32_t lane_off = static_cast<uint32_t>(32 * q) << 16;
        const float2* ys = reinterpret_cast<const float2*>(gsm + kAOffY) + ml;
        const float* yws = reinterpret_cast<const float*>(gsm + kAOffYw);
        const bool run64 = d.py_log2 == 6;
        float ah[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f}, al[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        bool ok = true;
        uint32_t run = 0;
        UnitIter it(u0, d);
        for (int32_t u = u0; u < u1; ++u, it.next(d)) {
            const uint32_t ui = static_cast<uint32_t>(u - u0);
            const int lt = it.lt;
            const int yb = it.yb;
            if (u == u0 || lt == 0) {
                // a new run: the previous run's y rows are no longer read
                if (u != u0) {
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(yfree);
                }
                if (!__all_sync(0xffffffffu, gwait(afull, run & 1u, abort, status))) {
                    ok = false;
                    break;
                }
                ++run;
            }
            const uint32_t b = ui & 1u;
            if (!__all_sync(0xffffffffu, gwait(accfull + b, (ui >> 1) & 1u, abort, status))) {
                ok = false;
                break;
            }
            tc::fence_after();
            float uc = 0.0f, us = 0.0f, ux = 0.0f, uy = 0.0f, uz = 0.0f;
            if (run64) {
                // patches of 64 y-cells x 1 z-cell: the warp's 16 columns are
                // consecutive y cells of z cell lt
                const int c0 = kACols * h;
                const int nv = min(kACols, d.ny - yb * kAYZ - c0);  // valid columns (warp-uniform)
                const float2 zv = __ldg(d.ztab + static_cast<int64_t>(lt) * d.n_pad + m);
                const float zwl = __ldg(d.zw + lt);
                // four groups of 4 columns; the next group's TMEM loads are in
                // flight while the current group is contracted
                float qr = 0.0f, qi = 0.0f, qxr = 0.0f, qxi = 0.0f, qyr = 0.0f, qyi = 0.0f;
                const uint32_t col = tbase + lane_off + b * 256u + static_cast<uint32_t>(c0);
                uint32_t dv[2][4][4];  // [buffer][cos, cos weighted, sin, sin weighted][column]
                tc::ld4(col, dv[0][0]);
                tc::ld4(col + 64, dv[0][1]);
                tc::ld4(col + 128, dv[0][2]);
                tc::ld4(col + 192, dv[0][3]);
                tc::wait_ld();
                const float2* yr = ys + c0 * kAM;
                const float4* ywr = reinterpret_cast<const float4*>(yws + c0);  // 4 columns per broadcast load
#pragma unroll
                for (int gq = 0; gq < 4; ++gq) {
                    const int cur = gq & 1;
                    const float4 w4 = ywr[gq];
                    const float wq[4] = {w4.x, w4.y, w4.z, w4.w};
                    if (gq < 3) {
                        const uint32_t cn = col + 4u * static_cast<uint32_t>(gq + 1);
                        tc::ld4(cn, dv[cur ^ 1][0]);
                        tc::ld4(cn + 64, dv[cur ^ 1][1]);
                        tc::ld4(cn + 128, dv[cur ^ 1][2]);
                        tc::ld4(cn + 192, dv[cur ^ 1][3]);
                    }
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int cc = 4 * gq + c;
                        if (nv == kACols || cc < nv) {
                            const float2 y = yr[cc * kAM];
                            const float w = wq[c];
                            const float cv = __uint_as_float(dv[cur][0][c]), sv = __uint_as_float(dv[cur][2][c]);
                            const float xcv = __uint_as_float(dv[cur][1][c]), xsv = __uint_as_float(dv[cur][3][c]);
                            const float pr = fmaf(cv, y.x, -sv * y.y), pi = fmaf(cv, y.y, sv * y.x);
                            qr += pr;
                            qi += pi;
                            qyr = fmaf(w, pr, qyr);
                            qyi = fmaf(w, pi, qyi);
                            qxr = fmaf(xcv, y.x, qxr);
                            qxr = fmaf(-xsv, y.y, qxr);
                            qxi = fmaf(xcv, y.y, qxi);
                            qxi = fmaf(xsv, y.x, qxi);
                        }
                    }
                    if (gq < 3) tc::wait_ld();
                    if (gq == 2) {
                        // every column of the unit is in registers: release the accumulators
                        tc::fence_before();
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(accfree + b);
                    }
                }
                const float ei = fmaf(qr, zv.y, qi * zv.x);
                uc = fmaf(qr, zv.x, -qi * zv.y);
                us = ei;
                ux = fmaf(qxr, zv.y, qxi * zv.x);
                uy = fmaf(qyr, zv.y, qyi * zv.x);
                uz = zwl * ei;
            } else {
            float qr = 0.0f, qi = 0.0f, qxr = 0.0f, qxi = 0.0f, qyr = 0.0f, qyi = 0.0f;
#pragma unroll 1
            for (int half = 0; half < 2; ++half) {
                const uint32_t col = tbase + lane_off + b * 256u + static_cast<uint32_t>(kACols * h + 8 * half);
                uint32_t dc[8], dxc[8], ds[8], dxs[8];
                tc::ld8(col, dc);
                tc::ld8(col + 64, dxc);
                tc::ld8(col + 128, ds);
                tc::ld8(col + 192, dxs);
                tc::wait_ld();
                if (half == 1) {
                    tc::fence_before();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(accfree + b);
                }
#pragma unroll
                for (int cc = 0; cc < 8; ++cc) {
                    const int r = kACols * h + 8 * half + cc;  // patch cell (warp-uniform)
                    const int kl = r & (py - 1);
                    const int k = yb * py + kl;
                    const int l = lt * (kAYZ >> d.py_log2) + (r >> d.py_log2);
                    if (k < d.ny && l < d.nz) {
                        const float2 y = ys[kl * kAM];
                        const float c = __uint_as_float(dc[cc]), s = __uint_as_float(ds[cc]);
                        const float xc = __uint_as_float(dxc[cc]), xsn = __uint_as_float(dxs[cc]);
                        const float pr = fmaf(c, y.x, -s * y.y), pi = fmaf(c, y.y, s * y.x);
                        const float w = __ldg(d.yw + k);
                        qr += pr;
                        qi += pi;
                        qyr = fmaf(w, pr, qyr);
                        qyi = fmaf(w, pi, qyi);
                        qxr += fmaf(xc, y.x, -xsn * y.y);
                        qxi += fmaf(xc, y.y, xsn * y.x);
                    }
                    // end of a run of one z cell: multiply by its z phasor
                    if (kl == py - 1 || (half == 1 && cc == 7)) {
                        if (l < d.nz) {
                            const float2 z = __ldg(d.ztab + static_cast<int64_t>(l) * d.n_pad + m);
                            const float er = fmaf(qr, z.x, -qi * z.y), ei = fmaf(qr, z.y, qi * z.x);
                            uc += er;
                            us += ei;
                            ux += fmaf(qxr, z.y, qxi * z.x);
                            uy += fmaf(qyr, z.y, qyi * z.x);
                            uz = fmaf(__ldg(d.zw + l), ei, uz);
                        }
                        qr = qi = qxr = qxi = qyr = qyi = 0.0f;
                    }
                }
            }
            }
            two_sum_acc(ah[0], al[0], uc);
            two_sum_acc(ah[1], al[1], us);
            two_sum_acc(ah[2], al[2], ux);
            two_sum_acc(ah[3], al[3], uy);
            two_sum_acc(ah[4], al[4], uz);
        }
        // the four column blocks of a mode, added in block order; the last
        // accumulator wait also covered every MMA, so the A stage is free
        double* red = reinterpret_cast<double*>(gsm);
#pragma unroll
        for (int i = 0; i < 5; ++i)
            red[(h * kAM + ml) * 5 + i] = static_cast<double>(ah[i]) + static_cast<double>(al[i]);
        asm volatile("bar.sync 1, %0;" ::"r"(32 * kAEpi) : "memory");
        if (h == 0 && ok && !*abort) {
            double v[5];
#pragma unroll
            for (int i = 0; i < 5; ++i)
                v[i] = ((red[ml * 5 + i] + red[(kAM + ml) * 5 + i]) + red[(2 * kAM + ml) * 5 + i]) +
                       red[(3 * kAM + ml) * 5 + i];
            const double gs = static_cast<double>(d.scal[0]), xs = static_cast<double>(d.scal[1]);
            const double ssin = v[1] / gs;
            double* o = d.part + (static_cast<int64_t>(grp) * d.n_pad + m) * 5;
            o[0] = v[0] / gs;
            o[1] = ssin;
            o[2] = v[2] / (gs * xs) + static_cast<double>(__ldg(d.X)) * ssin;
            o[3] = v[3] / gs + static_cast<double>(__ldg(d.Y)) * ssin;
            o[4] = v[4] / gs + (d.Z != nullptr ? static_cast<double>(__ldg(d.Z)) * ssin : 0.0);
        }
    } else if (warp == kAEpi) {
        // ---- MMA issue ------------------------------------------------------------
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_f16_f32(kAM, 2 * kAYZ);
            constexpr uint32_t dhi = tc::smem_desc_sw128_hi(gridc::kSbo);
            constexpr uint32_t tstep = gridc::kTileBytes >> 4;  // one operand tile in descriptor units
            const uint32_t alo = tc::smem_desc_sw128_lo(smem_u32(gsm));
            const uint32_t blo0 = tc::smem_desc_sw128_lo(smem_u32(gsm + kAOffB));
            bool ok = true;
            uint32_t run = 0;
            UnitIter it(u0, d);
            for (int32_t u = u0; u < u1 && ok; ++u, it.next(d)) {
                const uint32_t ui = static_cast<uint32_t>(u - u0);
                const int lt = it.lt;
                if ((u == u0 || lt == 0) && !gwait(afull, (run++) & 1u, abort, status)) {
                    ok = false;
                    break;
                }
                const uint32_t b = ui & 1u;
                const uint32_t s = ui % kABStages;
                if ((ui >= 2 && !gwait(accfree + b, ((ui >> 1) - 1u) & 1u, abort, status)) ||
                    !gwait(bfull + s, (ui / kABStages) & 1u, abort, status)) {
                    ok = false;
                    break;
                }
                tc::fence_after();
                const uint32_t blo = blo0 + s * (kAStageB >> 4);
                const uint32_t dcos = tbase + b * 256u, dsin = dcos + 128u;
#pragma unroll
                for (int ks = 0; ks < kAX / 16; ++ks) {
                    const uint32_t ko = static_cast<uint32_t>(ks) * (gridc::kKStep >> 4);  // 16 K elements
                    const uint64_t ch = tc::desc_of(alo + ko, dhi);
                    const uint64_t cl = tc::desc_of(alo + tstep + ko, dhi);
                    const uint64_t sh = tc::desc_of(alo + 2 * tstep + ko, dhi);
                    const uint64_t sl = tc::desc_of(alo + 3 * tstep + ko, dhi);
                    const uint64_t bh = tc::desc_of(blo + ko, dhi);
                    const uint64_t bl = tc::desc_of(blo + tstep + ko, dhi);
                    tc::mma_f16(dcos, ch, bh, idesc, ks != 0 ? 1u : 0u);
                    tc::mma_f16(dcos, ch, bl, idesc, 1u);
                    tc::mma_f16(dcos, cl, bh, idesc, 1u);
                    tc::mma_f16(dsin, sh, bh, idesc, ks != 0 ? 1u : 0u);
                    tc::mma_f16(dsin, sh, bl, idesc, 1u);
                    tc::mma_f16(dsin, sl, bh, idesc, 1u);
                }
                tc::commit(bfree + s);
                tc::commit(accfull + b);
                if (u + 1 == u1 || lt + 1 == d.n_lt) tc::commit(afree);  // last unit of the run
            }
            if (ok) atomicAdd(&g_grid_adj_units, static_cast<unsigned long long>(u1 - u0));
            // every MMA this CTA issued has completed before TMEM is released
            tc::commit(done);
            mbar_wait_bounded(done, 0);
        }
        __syncwarp();
    } else {
        // ---- bulk copies: per run the A tiles and y rows, per unit the B tiles ---------
        if (lane == 0) {
            uint32_t run = 0, issued_b = 0;
            UnitIter it(u0, d);
            for (int32_t u = u0; u < u1; ++u, it.next(d)) {
                const uint32_t ui = static_cast<uint32_t>(u - u0);
                if (u == u0 || it.lt == 0) {
                    if (run > 0 && (!gwait(afree, (run - 1u) & 1u, abort, status) ||
                                    !gwait(yfree, (run - 1u) & 1u, abort, status)))
                        break;
                    const int yb = it.yb;
                    const int kc = it.kc;
                    const int pkv = min(py, d.ny - yb * py);
                    // y weights of the rows (64 x 1 patches): whole 16-byte
                    // groups; the section is padded to 256 bytes
                    const uint32_t ywb = py == kAYZ ? static_cast<uint32_t>((pkv + 3) / 4 * 16) : 0u;
                    mbar_arrive_expect_tx(afull, kAStageA + pkv * kAYRow + ywb);
                    if (ywb) bulk_g2s(gsm + kAOffYw, d.yw + yb * py, ywb, afull);
                    const unsigned char* asrc = d.atab + (static_cast<int64_t>(mt) * d.n_kc + kc) * kAStageA;
                    for (int t = 0; t < 4; ++t)
                        bulk_g2s(gsm + t * gridc::kTileBytes, asrc + t * gridc::kTileBytes, gridc::kTileBytes, afull);
                    for (int r = 0; r < pkv; ++r)
                        bulk_g2s(gsm + kAOffY + r * kAYRow,
                                 d.ytab + (static_cast<int64_t>(yb * py + r) * d.n_pad + mt * kAM), kAYRow, afull);
                    ++run;
                }
                const uint32_t s = ui % kABStages;
                if (ui >= kABStages && !gwait(bfree + s, ((ui / kABStages) - 1u) & 1u, abort, status)) break;
                mbar_arrive_expect_tx(bfull + s, kAStageB);
                bulk_g2s(gsm + kAOffB + s * kAStageB, d.btab + static_cast<int64_t>(u) * kAStageB, kAStageB,
                         bfull + s);
                ++issued_b;
            }
            // copies still in flight land before the CTA's shared memory goes away
            if (run > 0) mbar_wait_bounded(afull, (run - 1u) & 1u);
            for (uint32_t t = issued_b > kABStages ? issued_b - kABStages : 0u; t < issued_b; ++t)
                mbar_wait_bounded(bfull + t % kABStages, (t / kABStages) & 1u);
        }
        __syncwarp();
    }
    tc::fence_before();
    __syncthreads();
    if (warp == kAEpi + 1) {
        tc::fence_after();
        tc::dealloc(tbase, kATmemCols);
    }
}

int g_adj_sms = 0;

// Layout of one grid adjoint: patch, units, groups and workspace sections.
struct AdjPlan {
    int py_log2, n_mt, n_kc, n_yb, n_lt, groups;
    int64_t units;
    int64_t off_part, off_gpart, off_gmax, off_xmax, off_scal, off_contrib, off_a, off_y, off_z, off_yw, off_zw,
        off_b, total;
};

AdjPlan adj_plan(int32_t nx, int32_t ny, int32_t nz, int64_t n_pad, int sms) {
    AdjPlan a{};
    // patch of 2^p y-cells by 64 / 2^p z-cells: fewest wasted columns, then
    // the longest runs of one z cell
    double best = 1e300;
    for (int p = 0; p <= 6; ++p) {
        const int64_t PY = int64_t(1) << p, PZ = kAYZ / PY;
        const double cols = double((ny + PY - 1) / PY * PY) * double((nz + PZ - 1) / PZ * PZ);
        const double w = cols / (double(ny) * double(nz)) - 1e-4 * double(p);
        if (w < best) {
            best = w;
            a.py_log2 = p;
        }
    }
    const int PY = 1 << a.py_log2, PZ = kAYZ >> a.py_log2;
    a.n_mt = static_cast<int>(n_pad / kAM);
    a.n_kc = (nx + kAX - 1) / kAX;
    a.n_yb = (ny + PY - 1) / PY;
    a.n_lt = (nz + PZ - 1) / PZ;
    a.units = int64_t(a.n_kc) * a.n_yb * a.n_lt;
    // groups: as many as fit one CTA per SM (mode tiles x groups <= SMs)
    int64_t g = sms > 0 ? sms / a.n_mt : 1;
    g = std::max<int64_t>(1, std::min<int64_t>(g, a.units));
    g = std::min<int64_t>(g, std::max<int64_t>(1, kAMaxCtas / a.n_mt));
    a.groups = static_cast<int>(g);
    int64_t off = 0;
    auto take = [&](int64_t bytes) {
        const int64_t o = off;
        off += align256(bytes);
        return o;
    };
    a.off_part = take(std::max<int64_t>(int64_t(kAMaxCtas) * kAM, n_pad) * 5 * 8);
    a.off_gpart = take(int64_t(kAScanBlocks) * 8);
    a.off_gmax = take(int64_t(kAScanBlocks) * 4);
    a.off_xmax = take(int64_t(kAScanBlocks) * 4);
    a.off_scal = take(16);
    a.off_contrib = take(n_pad * kBwdContrib * 8);
    a.off_a = take(int64_t(a.n_mt) * a.n_kc * kAStageA);
    a.off_y = take(int64_t(ny) * n_pad * 8);
    a.off_z = take(int64_t(nz) * n_pad * 8);
    a.off_yw = take(int64_t(ny) * 4);
    a.off_zw = take(int64_t(nz) * 4);
    a.off_b = take(a.units * kAStageB);
    a.total = off;
    return a;
}

}  // namespace

size_t bwd_grid_ws_bytes(int32_t nx, int32_t ny, int32_t nz, int64_t n_pad) {
    // the layout's sizes do not depend on the SM count
    return static_cast<size_t>(adj_plan(nx, ny, nz, n_pad, 1).total);
}

int launch_synth_bwd_grid(const void* table, int64_t n_modes, int32_t dim, const GridGeom& gg, const float* gY,
                          double sigma, const double* ell, const double* rot, int32_t periodic_mask,
                          const grf_grads& g, void* ws, int32_t* status, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (g_adj_sms == 0) {
        int dev = 0, sms = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(grid_adj_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kASmem);
        if (e != cudaSuccess) return e;
        g_adj_sms = sms;
    }
    const TableLayout TL = table_layout(n_modes);
    const unsigned char* tb = static_cast<const unsigned char*>(table);
    const AdjPlan ap = adj_plan(gg.nx, gg.ny, gg.nz, TL.n_pad, g_adj_sms);
    if (ap.units > INT32_MAX) return cudaErrorInvalidValue;
    unsigned char* w = static_cast<unsigned char*>(ws);
    const int64_t n = int64_t(gg.nx) * gg.ny * gg.nz;
    const float* Z = dim > 2 ? gg.Z : nullptr;

    AdjPrep p{};
    p.thdr = reinterpret_cast<const TableHeader*>(tb);
    p.cold = reinterpret_cast<const float4*>(tb + TL.off_cold);
    p.X = gg.X;
    p.Y = gg.Y;
    p.Z = Z;
    p.gY = gY;
    p.gmax = reinterpret_cast<const float*>(w + ap.off_gmax);
    p.xmax = reinterpret_cast<const float*>(w + ap.off_xmax);
    p.atab = w + ap.off_a;
    p.btab = w + ap.off_b;
    p.ytab = reinterpret_cast<float2*>(w + ap.off_y);
    p.ztab = reinterpret_cast<float2*>(w + ap.off_z);
    p.yw = reinterpret_cast<float*>(w + ap.off_yw);
    p.zw = reinterpret_cast<float*>(w + ap.off_zw);
    p.scal = reinterpret_cast<float*>(w + ap.off_scal);
    p.nx = gg.nx;
    p.ny = gg.ny;
    p.nz = gg.nz;
    p.n_pad = static_cast<int32_t>(TL.n_pad);
    p.n_kc = ap.n_kc;
    p.n_yb = ap.n_yb;
    p.n_lt = ap.n_lt;
    p.py_log2 = ap.py_log2;
    p.n_mt = ap.n_mt;
    p.units = ap.units;

    adj_scan_kernel<<<kAScanBlocks, 256, 0, st>>>(gY, n, gg.X, gg.nx, reinterpret_cast<float*>(w + ap.off_gmax),
                                                  reinterpret_cast<double*>(w + ap.off_gpart),
                                                  reinterpret_cast<float*>(w + ap.off_xmax));
    const int64_t items = int64_t(ap.n_mt) * ap.n_kc * kAM * 8 + (int64_t(gg.ny) + gg.nz) * TL.n_pad +
                          ap.units * kAYZ * 8 + gg.ny + gg.nz;
    const int64_t pg = std::min<int64_t>((items + 255) / 256, int64_t(g_adj_sms) * 16);
    adj_prep_kernel<<<static_cast<unsigned>(pg), 256, 0, st>>>(p);
    count_launches(2);

    AdjDesc d{};
    d.atab = p.atab;
    d.btab = p.btab;
    d.ytab = p.ytab;
    d.ztab = p.ztab;
    d.yw = p.yw;
    d.zw = p.zw;
    d.scal = p.scal;
    d.X = gg.X;
    d.Y = gg.Y;
    d.Z = Z;
    d.part = reinterpret_cast<double*>(w + ap.off_part);
    d.ny = gg.ny;
    d.nz = gg.nz;
    d.n_pad = p.n_pad;
    d.n_kc = ap.n_kc;
    d.n_yb = ap.n_yb;
    d.n_lt = ap.n_lt;
    d.py_log2 = ap.py_log2;
    d.n_mt = ap.n_mt;
    d.groups = ap.groups;
    d.units = static_cast<int32_t>(ap.units);
    grid_adj_kernel<<<static_cast<unsigned>(ap.groups * ap.n_mt), kAThreads, kASmem, st>>>(d, status);
    count_launches(1);
    return launch_bwd_reduce(table, n_modes, dim, sigma, ell, rot, periodic_mask, g, d.part, ap.groups,
                             reinterpret_cast<double*>(w + ap.off_gpart), kAScanBlocks,
                             reinterpret_cast<double*>(w + ap.off_contrib), stream);
}

int take_grid_adj_units(unsigned long long* units) {
    unsigned long long v = 0ull;
    const unsigned long long zero = 0ull;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_grid_adj_units, sizeof(v));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_grid_adj_units, &zero, sizeof(zero));
    if (e != cudaSuccess) return e;
    *units = v;
    return cudaSuccess;
}

}  // namespace grf
