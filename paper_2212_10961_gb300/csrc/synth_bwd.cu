// Adjoint of the spectral field sum (derivative of Eq. DiscreteFT, Sec. 4.1,
// with the reparameterisation A = sigma rho, a = R^T kappa / (2 pi l) and
// periodic axes rounded to multiples of 1/L).
//
// Given g_i = dL/dY_i, per mode j (theta_ij = 2 pi (a_j . x_i + psi_j)):
//     S_cos[j] = sum_i g_i cos theta_ij,  S_sin[j] = sum_i g_i sin theta_ij,
//     S_x[j,c] = sum_i g_i sin theta_ij x_ic
// and then dA = S_cos, dpsi = -2 pi A S_sin, da = -2 pi A S_x,
// drho = sigma dA, dsigma = sum_j (A_j / sigma) dA_j, with e = da with the
// periodic components zeroed and u = kappa / (2 pi l): dkappa_c =
// (R e)_c / (2 pi l_c), dl_c = -sum_j (u_jc / l_c) (R e_j)_c,
// dR_cd = sum_j u_jc e_jd, dmu = sum_i g_i.
//
// Kernel 1 (mode-stationary): a block owns kBwdThreads * MPT consecutive
// modes (MPT per thread, registers) and a contiguous range of spatially
// sorted cell tiles of kBwdTile cells.  Each tile is staged in shared memory
// with its bounding-box origin x0; phases are split exactly as in the
// forward kernel (per (tile, mode) compensated origin phase, FP32 offsets;
// exact per-cell path for the modes whose span over the tile is large).
// sin and cos are recomputed with the hardware MUFU (never stored).  Tile
// sums are FP32, folded into TwoSum-compensated accumulators, and written as
// FP64 partials per (split, mode).
// Kernel 2 sums the partials over splits in a fixed order (deterministic)
// and applies the chain rule per mode; kernel 3 reduces the scalar
// gradients (sigma, l, mu) in a fixed order.
#include <cuda_runtime.h>

#include "device_common.cuh"

namespace grf {

// Warp tiles of the adjoint that took the general path [0] and the lattice
// path [1] since the last grf_take_adjoint_path_counts (diagnostics).
static __device__ unsigned long long g_bwd_path_tiles[2];

namespace {

constexpr int kBwdThreads = 128;
constexpr int kBwdTile = 256;
constexpr int kBwdMaxSplits = 256;

// Most cell splits the workspace holds for a table of n_pad slots: 256, but
// no more than keep splits x mode blocks at 65536 (with that many mode blocks
// the GPU is full without splits), so the FP64 partials stay O(65536 x 512 x
// 40 bytes) whatever N.
__host__ __device__ constexpr int64_t bwd_max_splits(int64_t n_pad) {
    return n_pad / 512 >= 256 ? (65536 / (n_pad / 512) > 1 ? 65536 / (n_pad / 512) : 1) : kBwdMaxSplits;
}
constexpr int kMPT = 4;  // modes per thread
constexpr int kContrib = kBwdContrib;  // per-mode terms of the scalar gradients
constexpr double kTwoPi = 6.283185307179586476925286766559;

struct BwdArgs {
    const float4* hot;
    const float4* cold;
    const int32_t* order;
    const int32_t* kpref;
    int32_t n_modes;
    int32_t n_pad;
    int32_t dim;
    int32_t splits;
    double sigma;
    double ell[3];
    double rot[9];    // row-major transform R of the anisotropy axes (identity: none)
    double rot_it[9]; // R^-T, which maps a back to u = kappa / (2 pi l) (R itself for a rotation)
    int32_t periodic; // bit c: axis c is periodic (its dL/da reaches neither kappa, l nor R)
    const double* kap;      // table's kappa section [n_pad][3] (sorted slots)
    const int32_t* has_kap; // table header flag: 1 when kap holds the modes' kappa
    const float* xs;
    const float* ys;
    const float* zs;
    const int32_t* perm;
    int64_t perm_base;
    int64_t n_cells;
    const float* gY;
    double* part;     // [splits][n_pad][5]
    double* gpart;    // [n_gpart]: partial sums of g
    int32_t n_gpart;
    double* contrib;  // [kContrib][n_pad / 32]: per reduction block, the sums over its 32 modes
                      // of (A/sigma) dA, the dl terms (3) and the dR terms (9)
    double inv_sigma;
    double inv_ell[3];
    double inv_2pi_ell[3];
    grf_grads g;
};

__device__ __forceinline__ int bucket_of_bwd(float E) {
    if (!(E > 0.0f)) return 0;
    int b = static_cast<int>(ceilf(4.0f * __log2f(E))) + kBucketBias + 1;
    return b < 0 ? 0 : b;
}

// Phase a v in turns, reduced to [-1/2, 1/2], of a = ah + al (FP32 pair) at a
// point v of one axis (the product split exactly by an FMA).
__device__ __forceinline__ float axis_turns_bwd(float ah, float al, float v) {
    const float pr = ah * v;
    const float e = fmaf(ah, v, -pr);
    return frac_turn(frac_turn(pr) + fmaf(al, v, e));
}

struct DF {  // double-float accumulator
    float hi, lo;
    __device__ __forceinline__ void add(float v) { two_sum_acc(hi, lo, v); }
    __device__ __forceinline__ double value() const {
        return static_cast<double>(hi) + static_cast<double>(lo);
    }
};

// Per-warp shared memory: the warp's current cell tile and the compensated
// running sums of its modes (hi, lo pairs; kept here to free registers).
template <int MPT>
struct BwdWarpSmem {
    float4 cd[kBwdTile];           // (x - x0, y - y0, z - z0, g)
    float4 gd[kBwdTile];           // g (x - x0, y - y0, z - z0), 0: one FFMA per sum below
    float2 acc[32 * MPT][5];       // per mode: cos, sin, sin*x, sin*y, sin*z
};

// Per-mode sums over a lattice tile (see the check in bwd_partial_kernel): for
// brick b with corner c_b, e^{i theta} of cell (i, j, k) is
//     R_jk X^i,   R_jk = E_b Y^j Z^k,   E_b = e^{i theta(c_b)},
//     X = e^{2 pi i a_x hx},  Y = e^{2 pi i a_y hy},  Z = e^{2 pi i a_z hz},
// so a row's terms are R_jk H with H = sum_i g_i X^i evaluated from the
// powers X, X^2, X^3 (formed once per tile), and with the gradients g and
// i g staged per cell:
//     sum g cos, sum g sin            = Re, Im of sum g R X^i,
//     sum g sin (x - x0)              = (c_bx - x0) sum g sin + hx sum i g sin,
//     sum g sin (y - y0), (z - z0)    likewise with the weights j, k.
// No sine or cosine per cell: per (tile, mode) the exact step phasors
// (exactly reduced phases, hardware sine/cosine) and per (brick, mode) the
// corner phasor (warp-origin phase plus offset for light modes, the exact
// compensated phase for the first k_heavy modes).  Adds to sc, ss, sx.
template <int MPT, class SM>
__device__ __forceinline__ void bwd_lattice_tile(const BwdArgs& args, const SM& sm, const float4 (&hot)[MPT],
                                                 const int (&mm)[MPT], int m_base, int k_heavy, const float (&x0)[3],
                                                 const float (&cbk)[4][3], const float (&hl)[3],
                                                 const float (&t0)[MPT], float (&sc)[MPT], float (&ss)[MPT],
                                                 float (&sx)[MPT][3]) {
    constexpr int G = 2;  // modes per pass (the per-mode state of all MPT modes does not fit in registers)
    static_assert(MPT % G == 0, "mode groups");
    const float* gs = reinterpret_cast<const float*>(sm.cd);
    const float* gi = gs + kBwdTile;
#pragma unroll
    for (int kg = 0; kg < MPT; kg += G) {
        float X1r[G], X1i[G], X2r[G], X2i[G], X3r[G], X3i[G], Yr[G], Yi[G], Zr[G], Zi[G];
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const float4 c0 = __ldg(args.cold + 2 * mm[kg + k]);
            const float4 c1 = __ldg(args.cold + 2 * mm[kg + k] + 1);
            const float tx = kTwoPiF * axis_turns_bwd(c0.x, c0.y, hl[0]);
            const float tx2 = kTwoPiF * axis_turns_bwd(c0.x, c0.y, 2.0f * hl[0]);
            const float tx3 = kTwoPiF * axis_turns_bwd(c0.x, c0.y, 3.0f * hl[0]);
            const float ty = kTwoPiF * axis_turns_bwd(c0.z, c0.w, hl[1]);
            const float tz = kTwoPiF * axis_turns_bwd(c1.x, c1.y, hl[2]);
            X1r[k] = hw_cos(tx);
            X1i[k] = hw_sin(tx);
            X2r[k] = hw_cos(tx2);
            X2i[k] = hw_sin(tx2);
            X3r[k] = hw_cos(tx3);
            X3i[k] = hw_sin(tx3);
            Yr[k] = hw_cos(ty);
            Yi[k] = hw_sin(ty);
            Zr[k] = hw_cos(tz);
            Zi[k] = hw_sin(tz);
        }
#pragma unroll 1
        for (int b = 0; b < 4; ++b) {
            float Qr[G], Qi[G];  // plane phasor E_b Z^k
            float Sr[G], Si[G], Sp[G], Sj[G], Sk[G];
            const float dxb[3] = {cbk[b][0] - x0[0], cbk[b][1] - x0[1], cbk[b][2] - x0[2]};
#pragma unroll
            for (int k = 0; k < G; ++k) {
                float th;
                if (m_base + kg + k < k_heavy) {
                    th = kTwoPiF * phase_exact_turns<3>(cbk[b], __ldg(args.cold + 2 * mm[kg + k]),
                                                        __ldg(args.cold + 2 * mm[kg + k] + 1));
                } else {
                    th = fmaf(hot[kg + k].x, dxb[0], t0[kg + k]);
                    th = fmaf(hot[kg + k].y, dxb[1], th);
                    th = fmaf(hot[kg + k].z, dxb[2], th);
                }
                Qr[k] = hw_cos(th);
                Qi[k] = hw_sin(th);
                Sr[k] = Si[k] = Sp[k] = Sj[k] = Sk[k] = 0.f;
            }
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                float Rr[G], Ri[G], Tk[G];
#pragma unroll
                for (int k = 0; k < G; ++k) {
                    if (kk > 0) {
                        const float qr = fmaf(Qr[k], Zr[k], -Qi[k] * Zi[k]);
                        Qi[k] = fmaf(Qr[k], Zi[k], Qi[k] * Zr[k]);
                        Qr[k] = qr;
                    }
                    Rr[k] = Qr[k];
                    Ri[k] = Qi[k];
                    Tk[k] = 0.f;
                }
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const int base = 64 * b + 16 * kk + 4 * jj;
                    const float4 g4 = *reinterpret_cast<const float4*>(gs + base);
                    const float4 c4 = *reinterpret_cast<const float4*>(gi + base);
#pragma unroll
                    for (int k = 0; k < G; ++k) {
                        if (jj > 0) {
                            const float rr = fmaf(Rr[k], Yr[k], -Ri[k] * Yi[k]);
                            Ri[k] = fmaf(Rr[k], Yi[k], Ri[k] * Yr[k]);
                            Rr[k] = rr;
                        }
                        // the row's sums H = sum_i g_i X^i and H' = sum_i i g_i X^i
                        // from the precomputed powers (short, independent chains),
                        // then R H and Im(R H')
                        const float hr = fmaf(g4.w, X3r[k], fmaf(g4.z, X2r[k], fmaf(g4.y, X1r[k], g4.x)));
                        const float hi = fmaf(g4.w, X3i[k], fmaf(g4.z, X2i[k], g4.y * X1i[k]));
                        const float pr = fmaf(c4.w, X3r[k], fmaf(c4.z, X2r[k], c4.y * X1r[k]));
                        const float pi = fmaf(c4.w, X3i[k], fmaf(c4.z, X2i[k], c4.y * X1i[k]));
                        const float re = fmaf(Rr[k], hr, -Ri[k] * hi);
                        const float im = fmaf(Rr[k], hi, Ri[k] * hr);
                        Sr[k] += re;
                        Si[k] += im;
                        Sp[k] = fmaf(Rr[k], pi, fmaf(Ri[k], pr, Sp[k]));
                        if (jj > 0) Sj[k] = fmaf(static_cast<float>(jj), im, Sj[k]);
                        Tk[k] += im;
                    }
                }
#pragma unroll
                for (int k = 0; k < G; ++k)
                    if (kk > 0) Sk[k] = fmaf(static_cast<float>(kk), Tk[k], Sk[k]);
            }
#pragma unroll
            for (int k = 0; k < G; ++k) {
                sc[kg + k] += Sr[k];
                ss[kg + k] += Si[k];
                sx[kg + k][0] += fmaf(dxb[0], Si[k], hl[0] * Sp[k]);
                sx[kg + k][1] += fmaf(dxb[1], Si[k], hl[1] * Sj[k]);
                sx[kg + k][2] += fmaf(dxb[2], Si[k], hl[2] * Sk[k]);
            }
        }
    }
}

// Every warp works on its own: it owns 32 * MPT consecutive modes (MPT per
// lane, registers) and walks the block's range of cell tiles, staging each
// tile in its own shared memory (no block-wide barrier).  The next tile's
// coordinates and gradients are loaded into registers while the current
// tile is being summed.
constexpr int kBwdSmemBytes = static_cast<int>((kBwdThreads / 32) * sizeof(BwdWarpSmem<kMPT>));

template <int DIM, int MPT>
__global__ void __launch_bounds__(kBwdThreads, 4) bwd_partial_kernel(BwdArgs args, int32_t* status) {
    extern __shared__ __align__(16) unsigned char bwd_raw[];
    BwdWarpSmem<MPT>* wsm = reinterpret_cast<BwdWarpSmem<MPT>*>(bwd_raw);
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    BwdWarpSmem<MPT>& sm = wsm[warp];
    const int m_base = (blockIdx.x * (kBwdThreads / 32) + warp) * (32 * MPT) + lane * MPT;
    if ((blockIdx.x * (kBwdThreads / 32) + warp) * (32 * MPT) >= args.n_pad) return;  // whole warp idle

    // mode parameters (slots past n_pad are skipped; padding modes have A = 0);
    // the hi/lo pairs (cold records) are re-read from L1 once per tile
    float4 hot[MPT];
    int mm[MPT];
    bool live[MPT];
#pragma unroll
    for (int k = 0; k < MPT; ++k) {
        const int m = m_base + k;
        live[k] = m < args.n_pad;
        mm[k] = live[k] ? m : 0;
        hot[k] = __ldg(args.hot + mm[k]);
#pragma unroll
        for (int q = 0; q < 5; ++q) sm.acc[lane * MPT + k][q] = make_float2(0.f, 0.f);
    }
    DF gsum{0.f, 0.f};  // compensated FP32 pair instead of FP64 adds (slow pipe on this GPU)
    const bool count_g = blockIdx.x == 0 && warp == 0;  // one warp per split sums g

    const int64_t n = args.n_cells;
    const int64_t n_tiles = (n + kBwdTile - 1) / kBwdTile;
    const int64_t per_split = (n_tiles + args.splits - 1) / args.splits;
    const int64_t t_begin = blockIdx.y * per_split;
    const int64_t t_end = t_begin + per_split < n_tiles ? t_begin + per_split : n_tiles;
    constexpr int kPer = kBwdTile / 32;  // cells per lane per tile

    // registers holding the next tile (cells lane + 32 q)
    float xv[kPer][3];
    float gv[kPer];
    auto load_tile = [&](int64_t t) {
        const int64_t tb = t * kBwdTile;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int64_t i = tb + q * 32 + lane;
            const bool in = i < n;
            const int64_t ii = in ? i : tb;
            xv[q][0] = __ldg(args.xs + ii);
            xv[q][1] = DIM > 1 ? __ldg(args.ys + ii) : 0.f;
            xv[q][2] = DIM > 2 ? __ldg(args.zs + ii) : 0.f;
            const int64_t o = in ? static_cast<int64_t>(__ldg(args.perm + i)) - args.perm_base : 0;
            gv[q] = in && index_ok(o, n) ? __ldg(args.gY + o) : 0.f;
        }
    };
    if (t_begin < t_end) load_tile(t_begin);

    for (int64_t t = t_begin; t < t_end; ++t) {
        // ---- bounding box and origin of the tile (warp-wide) -----------------
        float x0[3] = {0.f, 0.f, 0.f};
        float E = 0.f;
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
            float mn = xv[0][c], mx = xv[0][c];
#pragma unroll
            for (int q = 1; q < kPer; ++q) {
                mn = fminf(mn, xv[q][c]);
                mx = fmaxf(mx, xv[q][c]);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, off));
                mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
            }
            x0[c] = 0.5f * mn + 0.5f * mx;
            E = fmaxf(E, fmaxf(mx - x0[c], x0[c] - mn));
        }
        const int bk = bucket_of_bwd(E);
        const int k_heavy = bk >= kBuckets ? args.n_pad : __ldg(args.kpref + bk);

        // ---- lattice tile (3-D): four 4 x 4 x 4 bricks of one grid spacing -----
        // Cell idx = 64 b + 16 k + 4 j + i of the tile lies at the corner of its
        // brick b (cell 64 b) plus (i hx, j hy, k hz), exactly in FP32 -- a
        // Cartesian grid handed over x-fastest, as the plan keeps it.  Lane l's
        // cell q (idx = 32 q + l) has b = q / 2, i = l % 4, j = (l / 4) % 4,
        // k = 2 (q % 2) + l / 16.  Every lane takes part in every shuffle.
        bool lat = false;
        float cbk[4][3] = {};
        float hl[3] = {0.f, 0.f, 0.f};
        if constexpr (DIM == 3) {
#pragma unroll
            for (int b = 0; b < 4; ++b)
#pragma unroll
                for (int c = 0; c < 3; ++c) cbk[b][c] = __shfl_sync(0xffffffffu, xv[2 * b][c], 0);
            hl[0] = __shfl_sync(0xffffffffu, xv[0][0], 1) - cbk[0][0];
            hl[1] = __shfl_sync(0xffffffffu, xv[0][1], 4) - cbk[0][1];
            hl[2] = __shfl_sync(0xffffffffu, xv[0][2], 16) - cbk[0][2];
            bool okl = t * kBwdTile + kBwdTile <= n && hl[0] > 0.f && hl[1] > 0.f && hl[2] > 0.f;
            const float oi = static_cast<float>(lane & 3) * hl[0];
            const float oj = static_cast<float>((lane >> 2) & 3) * hl[1];
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                const int b = q >> 1;
                const float ok_ = static_cast<float>(2 * (q & 1) + (lane >> 4)) * hl[2];
                okl = okl && (xv[q][0] - cbk[b][0] == oi) && (cbk[b][0] + oi == xv[q][0]) &&
                      (xv[q][1] - cbk[b][1] == oj) && (cbk[b][1] + oj == xv[q][1]) &&
                      (xv[q][2] - cbk[b][2] == ok_) && (cbk[b][2] + ok_ == xv[q][2]);
            }
            lat = __all_sync(0xffffffffu, okl);
            if (lane == 0) atomicAdd(&g_bwd_path_tiles[lat ? 1 : 0], 1ull);
        }
        __syncwarp();  // the previous tile's shared data is no longer read
        if (lat) {
            // g and i g per cell (i the cell's x index in its brick)
            float* gs = reinterpret_cast<float*>(sm.cd);
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                const int idx = q * 32 + lane;
                gs[idx] = gv[q];
                gs[kBwdTile + idx] = static_cast<float>(lane & 3) * gv[q];
            }
        } else {
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                const int idx = q * 32 + lane;
                const float dx = xv[q][0] - x0[0], dy = xv[q][1] - x0[1], dz = xv[q][2] - x0[2];
                sm.cd[idx] = make_float4(dx, dy, dz, gv[q]);
                sm.gd[idx] = make_float4(gv[q] * dx, gv[q] * dy, gv[q] * dz, 0.f);
            }
        }
        if (count_g) {
#pragma unroll
            for (int q = 0; q < kPer; ++q) gsum.add(gv[q]);  // cascaded sum: TwoSum per value
        }
        __syncwarp();
        // overlaps with the sums below (a lattice tile loads it after its sums:
        // its per-mode state needs the registers)
        if (!lat && t + 1 < t_end) load_tile(t + 1);

        // ---- per-mode sums over the tile ------------------------------------------
        const bool any_heavy = m_base < k_heavy;
        float sc[MPT], ss[MPT], sx[MPT][3];
        float t0[MPT];
#pragma unroll
        for (int k = 0; k < MPT; ++k) {
            sc[k] = 0.f;
            ss[k] = 0.f;
            sx[k][0] = sx[k][1] = sx[k][2] = 0.f;
            t0[k] = kTwoPiF * phase_exact_turns<DIM>(x0, __ldg(args.cold + 2 * mm[k]),
                                                      __ldg(args.cold + 2 * mm[k] + 1));
        }
        if (lat) {
            if constexpr (DIM == 3) bwd_lattice_tile<MPT>(args, sm, hot, mm, m_base, k_heavy, x0, cbk, hl, t0, sc, ss, sx);
            if (t + 1 < t_end) load_tile(t + 1);
        } else if (!__any_sync(0xffffffffu, any_heavy)) {
#pragma unroll 8
            for (int i = 0; i < kBwdTile; ++i) {
                const float4 c = sm.cd[i];
                const float4 gq = sm.gd[i];
#pragma unroll
                for (int k = 0; k < MPT; ++k) {
                    float th = fmaf(hot[k].x, c.x, t0[k]);
                    if (DIM > 1) th = fmaf(hot[k].y, c.y, th);
                    if (DIM > 2) th = fmaf(hot[k].z, c.z, th);
                    const float cs = hw_cos(th);
                    const float sn = hw_sin(th);
                    sc[k] = fmaf(c.w, cs, sc[k]);
                    ss[k] = fmaf(c.w, sn, ss[k]);
                    sx[k][0] = fmaf(gq.x, sn, sx[k][0]);
                    if (DIM > 1) sx[k][1] = fmaf(gq.y, sn, sx[k][1]);
                    if (DIM > 2) sx[k][2] = fmaf(gq.z, sn, sx[k][2]);
                }
            }
        } else {
            const int64_t tb = t * kBwdTile;
#pragma unroll
            for (int k = 0; k < MPT; ++k) {
                const bool heavy = (m_base + k) < k_heavy;
                const float4 c0 = __ldg(args.cold + 2 * mm[k]);
                const float4 c1 = __ldg(args.cold + 2 * mm[k] + 1);
                for (int i = 0; i < kBwdTile; ++i) {
                    const float4 c = sm.cd[i];
                    float th;
                    if (heavy) {
                        // exact coordinates re-read (the staged offsets are rounded)
                        const int64_t ii = tb + i < n ? tb + i : tb;
                        const float xa[3] = {__ldg(args.xs + ii), DIM > 1 ? __ldg(args.ys + ii) : 0.f,
                                             DIM > 2 ? __ldg(args.zs + ii) : 0.f};
                        th = kTwoPiF * phase_exact_turns<DIM>(xa, c0, c1);
                    } else {
                        th = fmaf(hot[k].x, c.x, t0[k]);
                        if (DIM > 1) th = fmaf(hot[k].y, c.y, th);
                        if (DIM > 2) th = fmaf(hot[k].z, c.z, th);
                    }
                    const float cs = hw_cos(th);
                    const float sn = hw_sin(th);
                    const float gs = c.w * sn;
                    sc[k] = fmaf(c.w, cs, sc[k]);
                    ss[k] += gs;
                    sx[k][0] = fmaf(gs, c.x, sx[k][0]);
                    if (DIM > 1) sx[k][1] = fmaf(gs, c.y, sx[k][1]);
                    if (DIM > 2) sx[k][2] = fmaf(gs, c.z, sx[k][2]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < MPT; ++k) {
            float2* a = sm.acc[lane * MPT + k];
            const float v[5] = {sc[k], ss[k], sx[k][0], sx[k][1], sx[k][2]};
#pragma unroll
            for (int q = 0; q < 2 + DIM; ++q) {
                float2 r = a[q];
                two_sum_acc(r.x, r.y, v[q]);
                if (q >= 2) two_sum_acc(r.x, r.y, x0[q - 2] * ss[k]);
                a[q] = r;
            }
        }
    }

    // ---- write FP64 partials ---------------------------------------------------------
#pragma unroll
    for (int k = 0; k < MPT; ++k) {
        if (!live[k]) continue;
        const int m = m_base + k;
        double* o = args.part + (static_cast<int64_t>(blockIdx.y) * args.n_pad + m) * 5;
        const float2* a = sm.acc[lane * MPT + k];
#pragma unroll
        for (int q = 0; q < 5; ++q)
            o[q] = q < 2 + DIM ? static_cast<double>(a[q].x) + static_cast<double>(a[q].y) : 0.0;
    }
    if (count_g) {
        double gs = gsum.value();
        for (int off = 16; off > 0; off >>= 1) gs += __shfl_xor_sync(0xffffffffu, gs, off);
        if (lane == 0) args.gpart[blockIdx.y] = gs;
    }
    (void)status;
}

// Kernel 2: per mode, fixed-order sum over splits, chain rule, scatter to the
// original mode index.  A block owns 32 modes (one per lane); warp w sums
// the splits w, w + 8, w + 16, ... in increasing order (coalesced rows of the
// partials, many loads in flight), and warp 0 adds the 8 warp sums in warp
// order, applies the chain rule (reciprocals of sigma and l precomputed: few
// FP64 operations, which are slow on this part) and writes the block's sums
// of the 13 scalar-gradient terms over its 32 modes, in mode order: a fixed
// order throughout, so the result does not depend on timing.
constexpr int kRedWarps = 8;

__global__ void __launch_bounds__(32 * kRedWarps) bwd_reduce_kernel(BwdArgs args) {
    __shared__ double red[kRedWarps][32][5];
    __shared__ double cts[kContrib][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int m = blockIdx.x * 32 + lane;  // n_pad is a multiple of 128
    {
        double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll 4
        for (int s = warp; s < args.splits; s += kRedWarps) {
            const double* p = args.part + (static_cast<int64_t>(s) * args.n_pad + m) * 5;
#pragma unroll
            for (int q = 0; q < 5; ++q) v[q] += p[q];
        }
#pragma unroll
        for (int q = 0; q < 5; ++q) red[warp][lane][q] = v[q];
    }
    __syncthreads();
    if (warp == 0) {
        double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int w = 0; w < kRedWarps; ++w)
#pragma unroll
            for (int q = 0; q < 5; ++q) v[q] += red[w][lane][q];
        double ct[kContrib];
#pragma unroll
        for (int q = 0; q < kContrib; ++q) ct[q] = 0.0;
        const int j = args.order[m];
        if (j >= 0) {
            const float4 h = args.hot[m];
            const float4 q0 = args.cold[2 * m];
            const float4 q1 = args.cold[2 * m + 1];
            const double A = static_cast<double>(h.w);
            const double a[3] = {static_cast<double>(q0.x) + static_cast<double>(q0.y),
                                 static_cast<double>(q0.z) + static_cast<double>(q0.w),
                                 static_cast<double>(q1.x) + static_cast<double>(q1.y)};
            const double gs = args.g.gscale != nullptr ? *args.g.gscale : 1.0;
            // the table holds the mode as (-A, psi + 1/2) at odd positions, where the
            // cosine sum v[0] has the opposite sign; A * v[1] and A * v[2..] do not
            const double dA = mode_flipped(m) ? -v[0] : v[0];
            args.g.dA[j] = gs * dA;
            args.g.dpsi[j] = gs * (-kTwoPi * A * v[1]);
            if (args.g.drho != nullptr) args.g.drho[j] = gs * (args.sigma * dA);
            ct[0] = (A * args.inv_sigma) * v[0];
            const int d = args.dim;
            double e[3] = {0.0, 0.0, 0.0};  // da with the periodic components zeroed
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (c >= d) break;
                const double da = -kTwoPi * A * v[2 + c];
                e[c] = (args.periodic >> c) & 1 ? 0.0 : da;
                args.g.da[static_cast<int64_t>(j) * d + c] = gs * da;
            }
            // u = kappa / (2 pi l) from the table when it holds kappa, else R^-T a
            // (the frequencies before the transform, a = R^T u); dL/du = R e
            const bool from_kappa = *args.has_kap != 0;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (c >= d) break;
                double u = 0.0, du = 0.0;
                if (from_kappa) u = args.kap[static_cast<int64_t>(m) * 3 + c] * args.inv_2pi_ell[c];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    if (k >= d) break;
                    if (!from_kappa) u += args.rot_it[c * 3 + k] * a[k];
                    du += args.rot[c * 3 + k] * e[k];
                }
                if (args.g.dkappa != nullptr) args.g.dkappa[static_cast<int64_t>(j) * d + c] = gs * (du * args.inv_2pi_ell[c]);
                ct[1 + c] = -(u * args.inv_ell[c]) * du;
#pragma unroll
                for (int q = 0; q < 3; ++q) ct[4 + c * 3 + q] = q < d ? u * e[q] : 0.0;
            }
        }
#pragma unroll
        for (int q = 0; q < kContrib; ++q) cts[q][lane] = ct[q];
        __syncwarp();
        // the block's sum of each term over its 32 modes, in mode order
        if (lane < kContrib) {
            double t = 0.0;
            for (int l = 0; l < 32; ++l) t += cts[lane][l];
            args.contrib[static_cast<int64_t>(lane) * gridDim.x + blockIdx.x] = t;
        }
    }
}

// Kernel 3: scalar gradients, one block of one warp per row: warp q sums row
// q (the reduction blocks' partials of term q, or the partial sums of g for
// dmu) with a lane stride, then adds the lanes by butterflies: a fixed order.
constexpr int kScalarRows = kContrib + 1;  // + the sum of g (dmu)

__global__ void __launch_bounds__(32 * kScalarRows) bwd_scalar_kernel(BwdArgs args, int32_t n_blocks) {
    const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
    double t = 0.0;
    if (q < kContrib) {
        const double* row = args.contrib + static_cast<int64_t>(q) * n_blocks;
        for (int k = lane; k < n_blocks; k += 32) t += row[k];
    } else {
        for (int k = lane; k < args.n_gpart; k += 32) t += args.gpart[k];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if (lane != 0) return;
    const double gs = args.g.gscale != nullptr ? *args.g.gscale : 1.0;
    if (q == 0) {
        args.g.dsigma[0] = gs * t;
        if (args.g.dsigma2 != nullptr) args.g.dsigma2[0] = gs * (t / (2.0 * args.sigma));
    } else if (q < 4) {
        if (q - 1 < args.dim) args.g.dell[q - 1] = gs * t;
    } else if (q < kContrib) {
        if (args.g.drot != nullptr) {
            const int c = (q - 4) / 3, e = (q - 4) % 3;
            if (c < args.dim && e < args.dim) args.g.drot[c * args.dim + e] = gs * t;
        }
    } else {
        args.g.dmu[0] = gs * t;
    }
}

// Cell splits: the grid (mode_blocks x splits) should be a whole number of
// waves of resident blocks, so that no SM idles in a partial last wave.
// The per-warp tiles need more than the default 48 KB of shared memory per block.
int bwd_allow_smem(int dim) {
    cudaError_t e;
    switch (dim) {
        case 1: e = cudaFuncSetAttribute(bwd_partial_kernel<1, kMPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBwdSmemBytes); break;
        case 2: e = cudaFuncSetAttribute(bwd_partial_kernel<2, kMPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBwdSmemBytes); break;
        default: e = cudaFuncSetAttribute(bwd_partial_kernel<3, kMPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBwdSmemBytes); break;
    }
    return e;
}

template <int DIM>
int choose_splits(int64_t n_cells, int mode_blocks, int64_t max_splits) {
    int dev = 0, sms = 148, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bwd_partial_kernel<DIM, kMPT>, kBwdThreads,
                                                  kBwdSmemBytes);
    if (per_sm < 1) per_sm = 1;
    const int64_t resident = static_cast<int64_t>(sms) * per_sm;
    const int64_t tiles = (n_cells + kBwdTile - 1) / kBwdTile;
    int64_t best = 1;
    double best_eff = -1.0;
    for (int64_t s = 1; s <= max_splits && s <= tiles; ++s) {
        const int64_t blocks = s * mode_blocks;
        const int64_t waves = (blocks + resident - 1) / resident;
        const double fill = static_cast<double>(blocks) / static_cast<double>(waves * resident);
        // per-block work is ceil(tiles / s) tiles; penalise the imbalance too
        const double per = static_cast<double>((tiles + s - 1) / s);
        const double bal = static_cast<double>(tiles) / (per * s);
        const double eff = fill * bal - 0.002 * static_cast<double>(waves);
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = s;
        }
    }
    return static_cast<int>(best);
}

}  // namespace

size_t bwd_workspace_bytes(int64_t n_cells, int64_t n_modes, int32_t dim) {
    (void)n_cells;
    (void)dim;
    const int64_t n_pad = pad_modes(n_modes);
    const int64_t part = bwd_max_splits(n_pad) * n_pad * 5 * 8;
    const int64_t gpart = bwd_max_splits(n_pad) * 8;
    const int64_t contrib = n_pad * kContrib * 8;
    return static_cast<size_t>(align256(part) + align256(gpart) + align256(contrib));
}

namespace {

// The table, parameter and transform fields of the adjoint's arguments.
void bwd_common_args(BwdArgs& a, const void* table, int64_t n_modes, int32_t dim, double sigma, const double* ell,
                     const double* rot, int32_t periodic_mask, const grf_grads& g) {
    const TableLayout TL = table_layout(n_modes);
    const unsigned char* tb = static_cast<const unsigned char*>(table);
    a.hot = reinterpret_cast<const float4*>(tb + TL.off_hot);
    a.cold = reinterpret_cast<const float4*>(tb + TL.off_cold);
    a.order = reinterpret_cast<const int32_t*>(tb + TL.off_order);
    a.kpref = reinterpret_cast<const int32_t*>(tb + TL.off_kpref);
    a.kap = reinterpret_cast<const double*>(tb + TL.off_kappa);
    a.has_kap = &reinterpret_cast<const TableHeader*>(tb)->has_kappa;
    a.periodic = periodic_mask;
    a.n_modes = static_cast<int32_t>(n_modes);
    a.n_pad = static_cast<int32_t>(TL.n_pad);
    a.dim = dim;
    a.sigma = sigma;
    for (int c = 0; c < 3; ++c) a.ell[c] = c < dim ? ell[c] : 1.0;
    a.inv_sigma = 1.0 / sigma;
    for (int c = 0; c < 3; ++c) {
        a.inv_ell[c] = 1.0 / a.ell[c];
        a.inv_2pi_ell[c] = 1.0 / (kTwoPi * a.ell[c]);
    }
    for (int k = 0; k < 9; ++k) a.rot[k] = rot[k];
    // inverse transpose of the leading dim x dim block (adjugate / determinant;
    // the host checks that the block is invertible)
    {
        double m[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        for (int i = 0; i < dim; ++i)
            for (int k = 0; k < dim; ++k) m[i][k] = rot[i * 3 + k];
        const double c00 = m[1][1] * m[2][2] - m[1][2] * m[2][1];
        const double c01 = m[1][2] * m[2][0] - m[1][0] * m[2][2];
        const double c02 = m[1][0] * m[2][1] - m[1][1] * m[2][0];
        const double c10 = m[0][2] * m[2][1] - m[0][1] * m[2][2];
        const double c11 = m[0][0] * m[2][2] - m[0][2] * m[2][0];
        const double c12 = m[0][1] * m[2][0] - m[0][0] * m[2][1];
        const double c20 = m[0][1] * m[1][2] - m[0][2] * m[1][1];
        const double c21 = m[0][2] * m[1][0] - m[0][0] * m[1][2];
        const double c22 = m[0][0] * m[1][1] - m[0][1] * m[1][0];
        const double det = m[0][0] * c00 + m[0][1] * c01 + m[0][2] * c02;
        // (R^-1)^T = cofactor matrix / det
        const double cof[3][3] = {{c00, c01, c02}, {c10, c11, c12}, {c20, c21, c22}};
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) a.rot_it[i * 3 + k] = cof[i][k] / det;
    }
    a.g = g;
}

}  // namespace

int launch_bwd_reduce(const void* table, int64_t n_modes, int32_t dim, double sigma, const double* ell,
                      const double* rot, int32_t periodic_mask, const grf_grads& g, double* part, int32_t splits,
                      double* gpart, int32_t n_gpart, double* contrib, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    BwdArgs a{};
    bwd_common_args(a, table, n_modes, dim, sigma, ell, rot, periodic_mask, g);
    a.part = part;
    a.splits = splits;
    a.gpart = gpart;
    a.n_gpart = n_gpart;
    a.contrib = contrib;
    bwd_reduce_kernel<<<static_cast<unsigned>(a.n_pad / 32), 32 * kRedWarps, 0, st>>>(a);
    bwd_scalar_kernel<<<1, 32 * kScalarRows, 0, st>>>(a, a.n_pad / 32);
    count_launches(2);
    return cudaGetLastError();
}

int launch_synth_bwd(const void* table, int64_t n_modes, int32_t dim, double sigma,
                     const double* ell, const double* rot, int32_t periodic_mask, const float* xs,
                     const float* ys, const float* zs,
                     const int32_t* perm, int64_t perm_base, int64_t n_cells, const float* gY,
                     const grf_grads& g, void* workspace, int32_t* status, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (const int e = bwd_allow_smem(dim)) return e;
    const TableLayout TL = table_layout(n_modes);
    BwdArgs a{};
    bwd_common_args(a, table, n_modes, dim, sigma, ell, rot, periodic_mask, g);
    a.xs = xs;
    a.ys = ys;
    a.zs = zs;
    a.perm = perm;
    a.perm_base = perm_base;
    a.n_cells = n_cells;
    a.gY = gY;
    const int mode_blocks = static_cast<int>((TL.n_pad + kBwdThreads * kMPT - 1) / (kBwdThreads * kMPT));
    a.splits = 1;
    if (n_cells > 0) {
        switch (dim) {
            case 1: a.splits = choose_splits<1>(n_cells, mode_blocks, bwd_max_splits(TL.n_pad)); break;
            case 2: a.splits = choose_splits<2>(n_cells, mode_blocks, bwd_max_splits(TL.n_pad)); break;
            default: a.splits = choose_splits<3>(n_cells, mode_blocks, bwd_max_splits(TL.n_pad)); break;
        }
    }
    const int64_t n_pad = TL.n_pad;
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    a.part = reinterpret_cast<double*>(ws);
    a.gpart = reinterpret_cast<double*>(ws + align256(bwd_max_splits(n_pad) * n_pad * 5 * 8));
    a.contrib = reinterpret_cast<double*>(ws + align256(bwd_max_splits(n_pad) * n_pad * 5 * 8) +
                                          align256(bwd_max_splits(n_pad) * 8));
    if (n_cells == 0) {
        // no cells: all gradients are zero
        cudaError_t e = cudaMemsetAsync(a.part, 0, sizeof(double) * n_pad * 5, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(a.gpart, 0, sizeof(double), st);
        if (e != cudaSuccess) return e;
        a.splits = 1;
    } else {
        dim3 grid(mode_blocks, a.splits);
        switch (dim) {
            case 1: bwd_partial_kernel<1, kMPT><<<grid, kBwdThreads, kBwdSmemBytes, st>>>(a, status); break;
            case 2: bwd_partial_kernel<2, kMPT><<<grid, kBwdThreads, kBwdSmemBytes, st>>>(a, status); break;
            case 3: bwd_partial_kernel<3, kMPT><<<grid, kBwdThreads, kBwdSmemBytes, st>>>(a, status); break;
            default: return cudaErrorInvalidValue;
        }
        count_launches(1);
    }
    a.n_gpart = a.splits;
    bwd_reduce_kernel<<<static_cast<unsigned>(n_pad / 32), 32 * kRedWarps, 0, st>>>(a);
    bwd_scalar_kernel<<<1, 32 * kScalarRows, 0, st>>>(a, static_cast<int32_t>(n_pad / 32));
    count_launches(2);
    return cudaGetLastError();
}

unsigned long long take_index_faults_bwd() { return take_tu_index_faults(); }

int take_bwd_path_counts(unsigned long long* general, unsigned long long* lattice) {
    unsigned long long v[2] = {0ull, 0ull};
    const unsigned long long zero[2] = {0ull, 0ull};
    cudaError_t e = cudaMemcpyFromSymbol(v, g_bwd_path_tiles, sizeof(v));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_bwd_path_tiles, zero, sizeof(zero));
    *general = v[0];
    *lattice = v[1];
    return e;
}

}  // namespace grf
