// Fifth-generation tensor-core primitives (tcgen05, sm_103a) shared by the
// contractions of the mixed-precision path: shared-memory and instruction
// descriptors for K-major TF32 operands staged by TMA with the 128-byte
// swizzle, the MMA issue and commit, tensor-memory loads, and the TF32 split
// of an fp32 value.
#pragma once

#include "tma.cuh"

namespace pichol {
namespace tc5 {

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand tile written by TMA with
// the 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);   // start address >> 4
    d |= (uint64_t)1 << 16;                     // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset: 8 rows x 128 bytes
    d |= (uint64_t)1 << 46;                     // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                     // 128-byte swizzle
    return d;
}

// Instruction descriptor: kind::tf32, fp32 accumulator, both operands K-major,
// M rows, N columns (M = 128; N a multiple of 16 up to 256).
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N)
{
    return (1u << 4)            // D format: f32
         | (2u << 7)            // A format: tf32
         | (2u << 10)           // B format: tf32
         | ((uint32_t)(N >> 3) << 17)
         | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// One K block (32 TF32 values per row: four MMAs of K = 8) of a split-TF32
// product into one accumulator: lo*hi, then hi*hi, then hi*lo, each over the
// four K steps.  The tensor pipe then switches operand buffers once for A and
// once for B per block; measured on GB300, 128 x 128 x 8 MMAs take 78 cycles
// each in this order against 109 when the three products alternate at every K
// step (64 with no switch at all).  `overwrite`: the first MMA replaces the
// accumulator instead of adding to it.  ah / al / bh / bl: shared-memory
// addresses of 1024-byte aligned 128-byte-swizzled operand tiles.
__device__ __forceinline__ void mma_split3_k32(uint32_t acc, uint32_t ah, uint32_t al, uint32_t bh, uint32_t bl,
                                               uint32_t idesc, bool overwrite)
{
    // advancing 32 bytes along K adds 2 to the descriptor's start-address field
    const uint64_t dah = sw128_desc(ah), dal = sw128_desc(al), dbh = sw128_desc(bh), dbl = sw128_desc(bl);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) mma_tf32(acc, dal + 2 * kk, dbh + 2 * kk, idesc, (overwrite && kk == 0) ? 0u : 1u);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) mma_tf32(acc, dah + 2 * kk, dbh + 2 * kk, idesc, 1u);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) mma_tf32(acc, dah + 2 * kk, dbl + 2 * kk, idesc, 1u);
}

// Arrives on `bar` once every MMA this thread issued before has completed.
__device__ __forceinline__ void commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive fp32 columns of the warp's 32 tensor-memory lanes.
__device__ __forceinline__ void ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// The same load without its wait: several loads are issued back to back, then
// wait_ld() and, for each destination, regs_ready() (the values may be used only
// through regs_ready's outputs, which the compiler cannot move above the wait).
__device__ __forceinline__ void ld16_issue(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

__device__ __forceinline__ void regs_ready(uint32_t (&r)[16])
{
    asm volatile(""
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}

// Allocation of `cols` tensor-memory columns by one whole warp; the address
// lands in *slot (shared memory).
__device__ __forceinline__ void alloc(uint32_t* slot, uint32_t cols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(slot)),
                 "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void dealloc(uint32_t tmem, uint32_t cols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(cols) : "memory");
}

// x rounded to the nearest TF32 value (10 mantissa bits); x - tf32_round(x)
// is exact in fp32.
__device__ __forceinline__ float tf32_round(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

}  // namespace tc5
}  // namespace pichol
