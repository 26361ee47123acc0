// bulk.cuh -- staging through shared memory with the bulk-copy engine: mbarrier objects and
// one-dimensional cp.async.bulk copies from global to shared memory whose completion is counted in
// bytes on an mbarrier (PTX ISA: mbarrier, cp.async.bulk; sm_90 and later).
#pragma once
#include <cstdint>

namespace tl {

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes the initialised barriers visible to the bulk-copy engine before the first copy names them.
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// One arrival that also announces `bytes` of copies still to land on this phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Copy `bytes` (a multiple of 16; both addresses 16-byte aligned) from global to shared memory; the
// bytes count against the current phase of `bar` when they land.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// One poll; the thread may be suspended for up to about `suspend_ns` while the phase is incomplete.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity, uint32_t suspend_ns)
{
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done)
                 : "r"(smem_addr(bar)), "r"(parity), "r"(suspend_ns)
                 : "memory");
    return done != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of `bar` with the given parity to complete.  Bounded twice over: at most `polls`
// polls of at most ~1 us each, and at most `limit_ns` of wall-clock time; false when either runs out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t polls, uint64_t limit_ns)
{
    if (mbar_try_wait(bar, parity, 1000))
        return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 1; i < polls; ++i) {
        if (mbar_try_wait(bar, parity, 1000))
            return true;
        if (global_ns() - t0 > limit_ns)
            return false;
    }
    return false;
}

}  // namespace tl
