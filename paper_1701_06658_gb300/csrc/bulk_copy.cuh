// Bulk copies global -> shared memory (cp.async.bulk, the TMA's untiled form)
// completing on mbarriers, and bounded waits on those barriers.
//
// A copy moves `bytes` (a multiple of 16) from a 16-byte aligned global
// address to a 16-byte aligned shared address and signals the barrier's
// transaction count.  Waits poll mbarrier.try_wait a bounded number of times
// (kWaitIters) and report failure instead of spinning forever.
#pragma once

#include <cstdint>

namespace lsgg {

__device__ __forceinline__ uint32_t sa(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
        : "=r"(r)
        : "r"(sa(b)), "r"(parity)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     sa(dst)),
                 "l"(src), "r"(bytes), "r"(sa(b))
                 : "memory");
}
constexpr int kWaitIters = 1 << 22;
// At most `limit` polls (the step's own waits take the context's limit, which
// a test hook can lower; the drains after a failed wait keep kWaitIters).
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int limit = kWaitIters) {
    for (int i = 0; i < limit; ++i)
        if (mbar_test(b, parity)) return true;
    return false;
}

}  // namespace lsgg
