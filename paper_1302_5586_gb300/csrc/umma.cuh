// umma.cuh -- building blocks of the 5th-generation tensor core (tcgen05) on
// sm_103a: shared-memory matrix descriptors, the instruction descriptor of
// kind::f16 with FP32 accumulation, tensor-memory (TMEM) allocation, the MMA
// itself, its commit to an mbarrier and the TMEM -> register load.
//
// Operand layout used here: K-major without swizzle.  A matrix of R rows and
// K columns is stored as "core matrices" of 8 rows x 16 bytes (8 binary16
// values per row, rows 16 bytes apart, 128 contiguous bytes); LBO is the byte
// distance between core matrices adjacent along K, SBO between core matrices
// adjacent along the rows.  D (M x N, FP32) lives in TMEM: row m in lane m,
// column n in column n of the allocation.  One MMA computes
// D = A * B^T (+ D), A M x K and B N x K, both K-major.
#pragma once

#include <stdint.h>

#include "tma.cuh"

namespace pencil {
namespace umma {

// Descriptor of a K-major operand without swizzle at shared address saddr
// (16-byte aligned): bits 0-13 address >> 4, 16-29 LBO >> 4, 32-45 SBO >> 4,
// 46-47 the descriptor version of this architecture family (1); base offset,
// LBO mode and swizzle (bits 49-52, 61-63) zero.
__device__ __forceinline__ uint64_t smem_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B
// binary16 (bits 7-9, 10-12 = 0), no negation, both K-major (bits 15, 16 =
// 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_f16_f32(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Allocate ncols TMEM columns (a power of two >= 32) for this CTA; the base
// address is written to *dst.  Executed by all 32 threads of one warp, which
// must also free it.
__device__ __forceinline__ void tmem_alloc(unsigned *dst, unsigned ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     tma::smem_addr(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_free(unsigned taddr, unsigned ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}

// D (+)= A * B^T; issued by one thread.  accumulate = false overwrites D.
__device__ __forceinline__ void mma_f16(unsigned d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                        bool accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"((int)accumulate)
        : "memory");
}

// `bar` receives one arrival once every MMA this thread issued before has
// completed (and its reads of shared memory are done).
__device__ __forceinline__ void commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     tma::smem_addr(bar))
                 : "memory");
}

// One plain arrival on an mbarrier (no transaction count).
__device__ __forceinline__ void arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(tma::smem_addr(bar)) : "memory");
}

// Order this thread's generic-proxy shared-memory writes before later
// async-proxy reads (the tensor core reads its operands through the async
// proxy).
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// 16 consecutive FP32 columns of the TMEM lane of each thread of the warp:
// warp w (of a warpgroup) reads lanes 32 (w % 4) .. + 31; taddr carries the
// lane in bits 16-31 and the column in bits 0-15.
__device__ __forceinline__ void ld16(unsigned taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// 32 consecutive FP32 columns (as raw bits) of the warp's TMEM lanes, not
// yet waited for: call wait_ld() before using r.
__device__ __forceinline__ void ld32_async(unsigned taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

}  // namespace umma
}  // namespace pencil
