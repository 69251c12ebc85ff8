// clbm_sync.cuh -- mbarrier helpers of the TMA-staged kernels: init, arrive
// (with a transaction count), and the bounded wait that every spin on a
// barrier goes through (a time-out returns false; callers record an error
// code and stop, so a barrier that never completes cannot hang a kernel).
#pragma once

#include <stdint.h>

namespace clbm {
namespace {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Bounded wait for phase `parity` of the barrier, at most `polls` polls;
// false on time-out.
__device__ __forceinline__ bool mbar_wait_n(uint64_t* bar, uint32_t parity, int polls) {
    const uint32_t a = smem_addr(bar);
    for (int it = 0; it < polls; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// The waits of the pipelined kernels: 2^18 polls.  A poll of a barrier
// that has not completed suspends for about 3.8 us on a GB300 (measured by
// clbm_selftest_bounded_wait), so the limit is about one second -- far
// beyond any load's latency: a time-out means the barrier will not
// complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    return mbar_wait_n(bar, parity, 1 << 18);
}

}  // namespace
}  // namespace clbm
