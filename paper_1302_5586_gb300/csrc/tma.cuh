// tma.cuh -- tensor-memory-accelerator (TMA) tile loads for sm_103a: one
// thread of a CTA issues a cp.async.bulk.tensor copy of a whole halo tile
// into shared memory and the CTA waits on an mbarrier whose transaction count
// the copy completes.  Every wait is bounded: a wait that runs out records a
// timeout in a device counter and the kernel skips its tile instead of
// spinning forever.
#pragma once

#include <cuda.h>

#include "internal.cuh"

namespace pencil {
namespace tma {

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// mbarrier with `count` expected arrivals, visible to the async proxy.
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// Arrive once and expect `bytes` more of transaction count in this phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// One poll of the phase with the given parity (the hardware may suspend the
// thread for a short, bounded time inside the poll).
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

// Wait for the phase with the given parity for at most `limit_ns`
// nanoseconds of the GPU's global timer; false if it has not completed.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}

// Copy the box of the 3-D tensor map at element coordinates (x, y, z) into
// shared memory at dst, completing `bar`'s transaction count.  x * element
// size must be a multiple of 16 bytes; dst 128-byte aligned.  Coordinates
// outside the tensor read zeros.
__device__ __forceinline__ void load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
        "%4}], [%5];\n" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// Copy the box of the 1-D tensor map starting at element x into shared
// memory at dst, completing `bar`'s transaction count.  Same rules as
// load_3d: x * element size a multiple of 16 bytes, dst 128-byte aligned,
// elements outside the tensor read as zeros.
__device__ __forceinline__ void load_1d(void *dst, const CUtensorMap *map, int x, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.1d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2}], "
        "[%3];\n" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(smem_addr(bar))
        : "memory");
}

// Bound of a wait on one tile load: far beyond any load's latency (a few
// microseconds), short enough that a lost completion ends the kernel.
constexpr uint64_t kLoadWaitNs = 1000000000ull;

}  // namespace tma
}  // namespace pencil
