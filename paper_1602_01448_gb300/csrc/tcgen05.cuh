// Fifth-generation tensor core (tcgen05) and tensor memory (TMEM) primitives
// for sm_100-class GPUs (written for sm_103a), as inline PTX.
//
// Only what the DFT-contraction frame kernels need:
//  - TMEM allocation by one warp, release at the end of the block;
//  - tcgen05.mma.cta_group::1.kind::f16 (FP16 or BF16 operands, FP32
//    accumulators in TMEM) with both operands in shared memory, described by
//    64-bit matrix descriptors in the canonical K-major layout without
//    swizzle: 8-row x 16-byte core matrices stored as contiguous 128-byte
//    blocks; SBO = byte distance between core matrices adjacent in the M/N
//    direction, LBO = byte distance between core matrices adjacent in K;
//  - tcgen05.commit to an mbarrier (completion of the issued MMAs);
//  - tcgen05.ld / tcgen05.st of 32 lanes x 16 columns (32x32b shape): warp w
//    of the block reaches TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31.
#pragma once

#include <stdint.h>

#include "tma.cuh"

namespace sharp {

// ---------------------------------------------------------------- TMEM
// Allocate `ncols` TMEM columns (a power of two >= 32); the base address is
// written to *dst.  Executed by all 32 lanes of one warp.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
// Release; the same warp that allocated, after every access has completed.
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Ordering of tcgen05 operations across a thread barrier.
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// TMEM address: lane in the upper 16 bits, column in the lower 16.
__device__ __forceinline__ uint32_t taddr_of(uint32_t base, uint32_t lane, uint32_t col) {
    return base + (lane << 16) + col;
}

// Two 16-column loads (e.g. real and imaginary planes) of this warp's 32
// lanes, completed before the asm ends, so the registers are valid on return.
__device__ __forceinline__ void tmem_ld16x2(uint32_t ta, uint32_t tb, float (&a)[16], float (&b)[16]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%32];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, "
        "[%33];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(ta), "r"(tb)
        : "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        a[j] = __uint_as_float(r[j]);
        b[j] = __uint_as_float(r[16 + j]);
    }
}

// Two 8-column stores of this warp's 32 lanes (not waited for: call
// tmem_wait_st before the values are read back or used by an MMA).
__device__ __forceinline__ void tmem_st8x2(uint32_t ta, uint32_t tb, const float (&a)[8], const float (&b)[8]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%2,%3,%4,%5,%6,%7,%8,%9};\n\t"
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%1], {%10,%11,%12,%13,%14,%15,%16,%17};" ::"r"(ta),
        "r"(tb), "r"(__float_as_uint(a[0])), "r"(__float_as_uint(a[1])), "r"(__float_as_uint(a[2])),
        "r"(__float_as_uint(a[3])), "r"(__float_as_uint(a[4])), "r"(__float_as_uint(a[5])),
        "r"(__float_as_uint(a[6])), "r"(__float_as_uint(a[7])), "r"(__float_as_uint(b[0])),
        "r"(__float_as_uint(b[1])), "r"(__float_as_uint(b[2])), "r"(__float_as_uint(b[3])),
        "r"(__float_as_uint(b[4])), "r"(__float_as_uint(b[5])), "r"(__float_as_uint(b[6])),
        "r"(__float_as_uint(b[7]))
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// N = 4 or 8 consecutive columns of this warp's 32 lanes, one value per
// column: a store (wait with tmem_wait_st before reading back) and a load
// completed before the asm ends.
template <int N>
__device__ __forceinline__ void tmem_st_cols(uint32_t ta, const float (&v)[N]) {
    static_assert(N == 4 || N == 8, "4 or 8 columns");
    if constexpr (N == 4) {
        asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(ta),
                     "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                     "r"(__float_as_uint(v[3]))
                     : "memory");
    } else {
        asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(ta),
                     "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                     "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                     "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                     : "memory");
    }
}
// Two loads of N columns (at ta and tb), waited for.
template <int N>
__device__ __forceinline__ void tmem_ld_cols2(uint32_t ta, uint32_t tb, float (&a)[N], float (&b)[N]) {
    static_assert(N == 4 || N == 8, "4 or 8 columns");
    uint32_t r[2 * N];
    if constexpr (N == 4) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%8];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4,%5,%6,%7}, [%9];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
            : "r"(ta), "r"(tb)
            : "memory");
    } else {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%16];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%17];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(ta), "r"(tb)
            : "memory");
    }
#pragma unroll
    for (int j = 0; j < N; ++j) {
        a[j] = __uint_as_float(r[j]);
        b[j] = __uint_as_float(r[N + j]);
    }
}

// ---------------------------------------------------------------- MMA
// Shared-memory matrix descriptor: canonical K-major layout, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo_bytes, uint32_t sbo_bytes) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo_bytes >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo_bytes >> 4) & 0x3FFFu) << 32) | (1ull << 46);   // bits 46-47: descriptor version 1
}

// Instruction descriptor of kind::f16 with FP32 accumulation, both operands
// K-major: bf16 = 0 for FP16 operands, 1 for BF16; neg_a negates A.
__host__ __device__ constexpr uint32_t idesc_f16(int bf16, int neg_a, int M, int N) {
    return (1u << 4)                         // D format: F32
           | ((uint32_t)bf16 << 7)           // A format
           | ((uint32_t)bf16 << 10)          // B format
           | ((uint32_t)neg_a << 13)         // negate A
           | ((uint32_t)(N >> 3) << 17)      // N / 8
           | ((uint32_t)(M >> 4) << 24);     // M / 16
}

// D[tmem] (+)= A[smem] . B[smem]^T  (M x N x 16); accumulate when acc != 0.
// Issued by one thread.
__device__ __forceinline__ void mma_f16_ss(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

// Arrive once on `bar` when every MMA this thread issued before has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

}  // namespace sharp
