// Fifth-generation tensor core (tcgen05) helpers for sm_103a, inline PTX:
// tensor-memory (TMEM) allocation, shared-memory matrix descriptors, MMA
// issue, completion tracking on an mbarrier, TMEM <-> register moves and the
// fences that order them against thread synchronisation.
#pragma once

#include <cstdint>

#include "device_common.cuh"

namespace grf {
namespace tc {

// Shared-memory matrix descriptor of a K-major operand in the 128-byte
// swizzled layout: atoms of 8 rows x 128 bytes (64 FP16 elements of K per
// row), the 16-byte chunk c of row r stored at chunk c ^ (r mod 8) of its
// row, atoms of consecutive 8-row groups `sbo` bytes apart.  The atoms start
// on 1024-byte boundaries; a K step of 16 elements advances the start
// address by 32 bytes inside the atom.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr, uint32_t sbo) {
    uint64_t d = static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
    d |= 1ull << 16;  // leading-dimension offset (unused by swizzled K-major layouts), 16 bytes
    d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;  // descriptor version of the tcgen05 family; base offset 0
    d |= 2ull << 61;  // 128-byte swizzle
    return d;
}

// The same descriptor as two 32-bit words: lo (start address field and the
// unused leading-dimension offset) and hi (stride offset, version, swizzle).
// A start address advanced by k bytes (k a multiple of 16, the result below
// 256 KB) is lo + k / 16: the field cannot carry into the next one, so the
// issuing thread adds K steps and tile offsets with one 32-bit add.
__device__ __forceinline__ uint32_t smem_desc_sw128_lo(uint32_t saddr) {
    return ((saddr & 0x3FFFFu) >> 4) | (1u << 16);
}
__host__ __device__ constexpr uint32_t smem_desc_sw128_hi(uint32_t sbo) {
    return ((sbo >> 4) & 0x3FFFu) | (1u << 14) | (2u << 29);
}
__device__ __forceinline__ uint64_t desc_of(uint32_t lo, uint32_t hi) {
    return (static_cast<uint64_t>(hi) << 32) | lo;
}

// Instruction descriptor of kind::f16: FP16 A and B, FP32 accumulator, both
// operands K-major, no negation, dense; shape M x N.
__host__ __device__ constexpr uint32_t idesc_f16_f32(int M, int N) {
    return (1u << 4)                                  // D: FP32
           | (0u << 7) | (0u << 10)                   // A, B: FP16
           | (static_cast<uint32_t>(N >> 3) << 17)    // N / 8
           | (static_cast<uint32_t>(M >> 4) << 24);   // M / 16
}

// D[tmem] (+)= A[smem] * B[smem]^T, one CTA, issued by a single thread.
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                        uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// The mbarrier receives one arrival once every tcgen05 operation this thread
// issued before has completed.
__device__ __forceinline__ void commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// Warp-wide: allocate `ncols` TMEM columns (power of two >= 32), address
// written to *slot (shared memory).
__device__ __forceinline__ void alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
// Warp-wide.
__device__ __forceinline__ void dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

#define GRF_R8(i) "=r"(r[i]), "=r"(r[i + 1]), "=r"(r[i + 2]), "=r"(r[i + 3]), "=r"(r[i + 4]), "=r"(r[i + 5]), \
                  "=r"(r[i + 6]), "=r"(r[i + 7])
#define GRF_W8(i) "r"(r[i]), "r"(r[i + 1]), "r"(r[i + 2]), "r"(r[i + 3]), "r"(r[i + 4]), "r"(r[i + 5]), \
                  "r"(r[i + 6]), "r"(r[i + 7])

// Warp-wide: lane t of the warp reads TMEM lane (lane field of taddr) + t,
// 32 consecutive 32-bit columns starting at the column field of taddr.  The
// warp may touch only its own quarter of the lanes (32 (warp id mod 4) ...).
__device__ __forceinline__ void ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : GRF_R8(0), GRF_R8(8), GRF_R8(16), GRF_R8(24)
        : "r"(taddr)
        : "memory");
}

// As ld32 with 4 columns.
__device__ __forceinline__ void ld4(uint32_t taddr, uint32_t (&r)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr)
                 : "memory");
}

// As ld32 with 8 columns.
__device__ __forceinline__ void ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : GRF_R8(0)
                 : "r"(taddr)
                 : "memory");
}

// As ld32 with 16 columns.
__device__ __forceinline__ void ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : GRF_R8(0), GRF_R8(8)
        : "r"(taddr)
        : "memory");
}

// Warp-wide store of 16 columns (layout as ld16).
__device__ __forceinline__ void st16(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        GRF_W8(0), GRF_W8(8)
        : "memory");
}

// Warp-wide store of 32 columns (layout as ld32).
__device__ __forceinline__ void st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        GRF_W8(0), GRF_W8(8), GRF_W8(16), GRF_W8(24)
        : "memory");
}

// As ld32 with 64 columns.
__device__ __forceinline__ void ld64(uint32_t taddr, uint32_t (&r)[64]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
        "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
        "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
        : GRF_R8(0), GRF_R8(8), GRF_R8(16), GRF_R8(24), GRF_R8(32), GRF_R8(40), GRF_R8(48), GRF_R8(56)
        : "r"(taddr)
        : "memory");
}

// Warp-wide store of 64 columns (layout as ld64).
__device__ __forceinline__ void st64(uint32_t taddr, const uint32_t (&r)[64]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x64.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,"
        "%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,"
        "%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63,%64};" ::"r"(taddr),
        GRF_W8(0), GRF_W8(8), GRF_W8(16), GRF_W8(24), GRF_W8(32), GRF_W8(40), GRF_W8(48), GRF_W8(56)
        : "memory");
}
#undef GRF_R8
#undef GRF_W8

// Plain mbarrier arrival (count 1).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Two FP32 values rounded to FP16 (round to nearest even) and packed, `lo`
// in the low half (the lower address in memory).
__device__ __forceinline__ uint32_t pack_f16x2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}
// The two FP16 halves of a packed word as FP32 (exact).
__device__ __forceinline__ void unpack_f16x2(uint32_t v, float& lo, float& hi) {
    asm("{\n\t.reg .b16 l, h;\n\t"
        "mov.b32 {l, h}, %2;\n\t"
        "cvt.f32.f16 %0, l;\n\t"
        "cvt.f32.f16 %1, h;\n\t}"
        : "=f"(lo), "=f"(hi)
        : "r"(v));
}

// x = hi + lo with hi = fp16(x) and lo = fp16(x - hi), for a pair of values:
// |x - hi - lo| <= 2^-24 for |x| <= 1 (lo's own rounding; hi's error is
// carried exactly by x - hi in FP32).
__device__ __forceinline__ void split_f16x2(float a, float b, uint32_t& hi, uint32_t& lo) {
    hi = pack_f16x2(a, b);
    float ah, bh;
    unpack_f16x2(hi, ah, bh);
    lo = pack_f16x2(a - ah, b - bh);
}

}  // namespace tc
}  // namespace grf
