// mbarrier and bulk-copy (TMA) helpers in inline PTX, shared by the staged kernels (sm_103a).
#pragma once

#include <stdint.h>

namespace msda {

constexpr long long kSpinLimit = 1ll << 26;  // bounded mbarrier wait (~seconds)

// Poll limit of the first wait of a staging step in the translation unit that includes this header: kSpinLimit
// unless msda_debug_set_wait_limit lowered it (0: give up at once).  The wait that drains the copies after a
// give-up always keeps kSpinLimit, so no copy is in flight when a block leaves.
static __device__ long long g_first_wait_limit = kSpinLimit;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// Plain arrival (no transaction bytes): completes the phase of a barrier initialised with count 1.
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// First wait of a staging step: true when the phase completed within the limit.
__device__ __forceinline__ bool mbar_wait_first(uint64_t* bar, uint32_t parity) {
    const long long lim = g_first_wait_limit;
    if (lim <= 0) return false;
    long long spins = 0;
    while (!mbar_try_wait(bar, parity))
        if (++spins > lim) return false;
    return true;
}

// Drain wait after a first wait gave up: the full limit, so the copies in flight land before the block goes on.
__device__ __forceinline__ bool mbar_wait_drain(uint64_t* bar, uint32_t parity) {
    long long spins = 0;
    while (!mbar_try_wait(bar, parity))
        if (++spins > kSpinLimit) return false;
    return true;
}

// 1D bulk copy global -> shared (both addresses 16-byte aligned, bytes a multiple of 16), completing on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

}  // namespace msda
