// Inline-PTX helpers for the fifth-generation tensor cores (tcgen05) on
// sm_100 and later, here sm_103a.
//
// Products take their operands from shared memory in the canonical K-major
// layout without swizzle: core matrices of 8 rows x 16 bytes (128 contiguous
// bytes each); LBO is the byte step between core matrices along K, SBO the
// byte step between 8-row groups.  The FP32 accumulator lives in tensor
// memory (TMEM, 128 lanes = rows); one thread issues tcgen05.mma, completion
// is signalled by tcgen05.commit on an mbarrier, and tcgen05.ld brings rows
// back to registers.
#pragma once

#include <stdint.h>

#include "bvf_tma.cuh"

namespace tc {

__device__ __forceinline__ uint64_t smem_desc(const void *p, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((bvf::tma::saddr(p) >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;                      // descriptor version; no swizzle
    return d;
}

// kind::tf32 instruction descriptor: D FP32, A and B TF32, both K-major
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// kind::f16 instruction descriptor with BF16 operands: D FP32, A and B BF16,
// both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     bvf::tma::saddr(dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
// D (TMEM) = A B (acc = 0) or D + A B (acc = 1), TF32 operands
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, int acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
                 : "memory");
}
// the same with 16-bit operands (kind::f16: FP16 or BF16 per the descriptor)
__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, int acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
                 : "memory");
}
__device__ __forceinline__ void commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     bvf::tma::saddr(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 32 consecutive columns of this warp's 32 lanes: thread i of the warp gets
// row (lane base + i), columns col .. col+31
__device__ __forceinline__ void ld32(uint32_t taddr, float (&r)[32])
{
    uint32_t u[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]),
                   "=r"(u[6]), "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]),
                   "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]), "=r"(u[16]), "=r"(u[17]),
                   "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]),
                   "=r"(u[24]), "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]),
                   "=r"(u[30]), "=r"(u[31])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 32; ++i) r[i] = __uint_as_float(u[i]);
}

// 8 consecutive columns of this warp's 32 lanes (the narrow form of ld32)
__device__ __forceinline__ void ld8(uint32_t taddr, float (&r)[8])
{
    uint32_t u[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]),
                   "=r"(u[6]), "=r"(u[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) r[i] = __uint_as_float(u[i]);
}

// byte offset of element (row, k) in a K-major TF32 operand with K columns
__host__ __device__ __forceinline__ uint32_t kmaj_off(int row, int k, int K)
{
    return (uint32_t)((((row >> 3) * (K >> 2) + (k >> 2)) << 7) + ((row & 7) << 4) + ((k & 3) << 2));
}
// byte offset of the 16-byte core-matrix row holding elements (row, k8 .. k8+7)
// of a K-major 16-bit operand with K columns (k8 a multiple of 8)
__host__ __device__ __forceinline__ uint32_t kmaj_off16(int row, int k8, int K)
{
    return (uint32_t)((((row >> 3) * (K >> 3) + (k8 >> 3)) << 7) + ((row & 7) << 4));
}

}  // namespace tc
