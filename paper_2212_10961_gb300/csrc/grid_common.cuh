// Pieces shared by the tensor-core grid kernels (forward synthesis and
// adjoint): the shared-memory layout of one FP16 operand tile and the
// bounded mbarrier wait of their warp-specialised pipelines.
#pragma once

#include <cstdint>

#include "device_common.cuh"

namespace grf {
namespace gridc {

constexpr int kRows = 128;                 // rows of an operand tile (M or N)
constexpr int kK = 64;                     // K elements of a tile row (128 bytes of FP16)
constexpr int kTileBytes = kRows * kK * 2; // 16 KB
constexpr uint32_t kSbo = 1024;            // 8-row groups: one 128-byte-swizzle atom apart
constexpr uint32_t kKStep = 32;            // bytes of 16 K elements inside an atom row
constexpr int kSmemMax = 232448;           // dynamic shared memory per CTA (227 KB)

// Byte offset of the 16-byte row segment (row r, K elements 8 kk8 .. 8 kk8 + 7)
// in a 128 x 64 K-major FP16 tile in the 128-byte swizzled layout: row r at
// (r / 8) * 1024 + (r % 8) * 128, its 16-byte chunk kk8 at position
// kk8 ^ (r % 8) of the row (so 8 consecutive rows' chunks kk8 fall in 8
// different bank groups).
__host__ __device__ __forceinline__ uint32_t tile_off(int r, int kk8) {
    return static_cast<uint32_t>(r >> 3) * kSbo + static_cast<uint32_t>(r & 7) * 128u +
           (static_cast<uint32_t>(kk8 ^ (r & 7)) << 4);
}

// Bounded wait that also gives up once another role has set the abort flag
// (then status bit 2 is set).
__device__ __forceinline__ bool gwait(uint64_t* bar, uint32_t parity, volatile int32_t* abort, int32_t* status) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t round = 0; round < kWaitMaxRounds; ++round) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (*abort) return false;
        if (global_ns() - t0 > kWaitLimitNs) break;
    }
    *abort = 1;
    atomicOr(status, 2);
    return false;
}

// (z + psi) phase of a mode in turns, exactly reduced: c1 = (a_z hi, a_z lo,
// psi hi, psi lo) of the table's cold record at the z coordinate (psi alone
// without a z axis).
__device__ __forceinline__ float psi_z_turns(const float4 c1, float z, bool has_z) {
    float t = has_z ? turns_axis(c1.x, c1.y, z) : 0.0f;
    t = frac_turn(t + c1.z);
    return frac_turn(t + c1.w);
}

// The power of two s with |v| s < 1 for every |v| <= m (1 when m is 0 or not
// finite).
__device__ __forceinline__ float pow2_scale_below_one(float m) {
    if (!(m > 0.0f) || !(m < 3.0e38f)) return 1.0f;
    int e;
    frexpf(m, &e);  // m = f 2^e, f in [1/2, 1)
    return ldexpf(1.0f, -e);
}

}  // namespace gridc
}  // namespace grf
