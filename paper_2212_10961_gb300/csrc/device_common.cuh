// Device helpers shared by the CUDA kernels: hardware cosine/sine, the
// compensated phase of one mode at one point, compensated accumulation, and
// the mbarrier / bulk-copy primitives used to stage mode chunks.
#pragma once

#include <cstdint>

#include "grf_internal.h"

namespace grf {

constexpr float kTwoPiF = 6.28318530717958647692f;
// (v + 1.5*2^23) - 1.5*2^23 rounds v to the nearest integer for |v| < 2^22.
constexpr float kRoundMagic = 12582912.0f;  // 1.5 * 2^23

// Hardware approximate cosine / sine (PTX cos.approx / sin.approx), radians.
__device__ __forceinline__ float hw_cos(float x) {
    float y;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float hw_sin(float x) {
    float y;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// cos(2 pi f) for |f| <= 1/2 (turns) on the FMA pipe: polynomial of degree 6
// in s = f^2, Horner in FP32, max abs error 4.0e-7.  Coefficients: FP64
// least-squares fit on Chebyshev nodes of [0, 1/4] rounded to FP32
// (gen_cos_poly.py in this directory prints them and the error).
__device__ __forceinline__ float cos_turns_poly(float f) {
    const float s = f * f;
    float r = 6.528658390e+00f;
    r = fmaf(r, s, -2.596759987e+01f);
    r = fmaf(r, s, 6.016762924e+01f);
    r = fmaf(r, s, -8.545014191e+01f);
    r = fmaf(r, s, 6.493911743e+01f);
    r = fmaf(r, s, -1.973920441e+01f);
    return fmaf(r, s, 1.000000000e+00f);
}

// Remove an integer from v exactly with FP32 adds only (no conversion unit):
// r = v - ((v + 1.5*2^23) - 1.5*2^23).  For |v| < 2^22 the subtracted value is
// rint(v) and |r| <= 1/2; for 2^22 <= |v| < 2^46 it is an integer within one
// of v (|r| <= 1, r == v mod 1).  Exact in every case.
__device__ __forceinline__ float frac_turn(float v) {
    return v - ((v + kRoundMagic) - kRoundMagic);
}

// Exact reduced phase of one mode at point x, in turns, |result| <= 1/2:
//   t = a . x + psi  with a = ah + al, psi = psi_h + psi_l (FP32 pairs).
// For each axis ah*x is split exactly into p + e (FMA), the integer part of
// p is removed exactly, and the remainders are summed with the high part kept
// in [-1/2, 1/2] after every addition (error <= 2^-24 turn per addition).
// c0 = (ah_x, al_x, ah_y, al_y), c1 = (ah_z, al_z, psi_h, psi_l).  Valid for
// |ah * x| < 2^46.
template <int DIM>
__device__ __forceinline__ float phase_exact_turns(const float* x, float4 c0, float4 c1) {
    float hi = c1.z;
    float lo = c1.w;
    const float ah[3] = {c0.x, c0.z, c1.x};
    const float al[3] = {c0.y, c0.w, c1.y};
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        const float p = ah[c] * x[c];
        const float e = fmaf(ah[c], x[c], -p);
        hi = frac_turn(hi + frac_turn(p));
        lo += fmaf(al[c], x[c], e);
    }
    return frac_turn(hi + frac_turn(lo));
}

// Phase a v in turns, reduced to [-1/2, 1/2], of a = ah + al (FP32 pair) at a
// point v of one axis: the product ah v split exactly by an FMA, integer
// parts removed exactly (as phase_exact_turns, for one axis and no psi).
__device__ __forceinline__ float turns_axis(float ah, float al, float v) {
    const float pr = ah * v;
    const float e = fmaf(ah, v, -pr);
    return frac_turn(frac_turn(pr) + fmaf(al, v, e));
}

// Accumulate partial sum p into (s, e) with an exact TwoSum error term.
__device__ __forceinline__ void two_sum_acc(float& s, float& e, float p) {
    float t = s + p;
    float bp = t - s;
    float err = (s - (t - bp)) + (p - bp);
    s = t;
    e += err;
}

// ---------------------------------------------------------------------------
// mbarrier and bulk copy (global -> shared), PTX.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait: returns false if the phase did not complete within
// `limit_ns` (two seconds by default, checked on the global timer every 256
// polls) or within 2^24 polls, whichever comes first, so the wait ends even
// if the timer does not advance.
constexpr uint64_t kWaitLimitNs = 2000000000ull;
constexpr uint32_t kWaitMaxRounds = 1u << 16;  // x 256 polls
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t limit_ns = kWaitLimitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t round = 0; round < kWaitMaxRounds; ++round) {
        for (int i = 0; i < 256; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// 1-D bulk copy global -> shared, completion reported to `bar` as tx bytes.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes,
                                         uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
        "[%3];" ::"r"(smem_u32(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Hint: bring the 128-byte line holding `p` into L1 (no register, no wait).
__device__ __forceinline__ void prefetch_l1(const void* p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Orders this thread's generic-proxy shared-memory accesses before later
// async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---- checked builds --------------------------------------------------------
// Compiled with -DGRF_CHECKED=1 (libgrf_checked.so), every index that a kernel
// reads from device memory before using it as an address (a permutation
// entry, a scatter position) is tested first: an index out of range is
// counted in this translation unit's g_index_faults and its access skipped,
// instead of reading or writing out of bounds.  The release build compiles
// the tests out (GRF_CHECKED is set in grf_internal.h).
#if GRF_CHECKED
static __device__ unsigned long long g_index_faults;
#endif

__device__ __forceinline__ bool index_ok(int64_t i, int64_t n) {
#if GRF_CHECKED
    if (i >= 0 && i < n) return true;
    atomicAdd(&g_index_faults, 1ull);
    return false;
#else
    (void)i;
    (void)n;
    return true;
#endif
}

// Host side: this translation unit's count since the last call, then reset
// (synchronous; 0 without a checked build).
static inline unsigned long long take_tu_index_faults() {
#if GRF_CHECKED
    unsigned long long v = 0ull;
    const unsigned long long zero = 0ull;
    if (cudaMemcpyFromSymbol(&v, g_index_faults, sizeof(v)) != cudaSuccess) return ~0ull;
    if (cudaMemcpyToSymbol(g_index_faults, &zero, sizeof(zero)) != cudaSuccess) return ~0ull;
    return v;
#else
    return 0ull;
#endif
}

// Mismatch epilogue of one cell (kMapMismatch): K = exp(Y), gY = 2 (K - T) K
// / n_mean with the same FP32 operations as the standalone loss kernel, and
// the squared difference returned for the loss sum (FP64).
__device__ __forceinline__ double mismatch_store(const MapDev& m, int64_t o, float y) {
    const float k = expf(y);
    const float d = k - __ldg(m.T + o);
    m.G[o] = m.g_scale * d * k;
    return static_cast<double>(d) * static_cast<double>(d);
}

// Map epilogue of one cell (Sec. 3.1 truncation rule, Sec. 4.1 lognormal).
__device__ __forceinline__ void map_store(const MapDev& m, int64_t o, float y) {
    const int bits = m.bits;
    if (bits & GRF_MAP_Y) m.Y[o] = y;
    if (bits & GRF_MAP_LOGNORMAL) m.K[o] = m.k_ref * expf(y);
    if (bits & (GRF_MAP_FACIES | GRF_MAP_VALUES)) {
        int lab = 0;
        for (int t = 0; t < m.n_thr; ++t) lab += (y > m.thr[t]) ? 1 : 0;
        if (bits & GRF_MAP_FACIES) m.F[o] = static_cast<uint8_t>(lab);
        if (bits & GRF_MAP_VALUES) m.P[o] = m.values[lab];
    }
    if (bits & GRF_MAP_POROSITY) {
        float p = fmaf(m.phi1, (y - m.mu) * m.sigma_inv, m.phi0);
        m.P[o] = fminf(fmaxf(p, m.phi_min), m.phi_max);
    }
}

}  // namespace grf
