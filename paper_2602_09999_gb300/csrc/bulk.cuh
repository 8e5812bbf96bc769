// bulk.cuh -- bulk asynchronous copies from global to shared memory with
// mbarrier completion (sm_90 and later, here sm_103a), in hand-written PTX.
//
// One elected thread arms a barrier with the number of bytes it expects
// (mbarrier.arrive.expect_tx) and issues cp.async.bulk copies whose
// completion counts those bytes down; the consumers wait on the barrier's
// phase.  Source and destination must be 16-byte aligned and every size a
// multiple of 16 bytes: the callers check this before taking this path.
//
// Every wait is bounded: bulk_wait gives up after kBulkWaitLimit polls and
// returns false, so a kernel can set an error flag and return instead of
// hanging.
#pragma once

#include <stdint.h>

namespace fgs {

// Polls of mbarrier.try_wait before a wait gives up.  Each poll may suspend
// the thread for a while on its own, so this bounds the wait far above any
// copy's latency (microseconds) while keeping a lost arrival finite.
constexpr uint32_t kBulkWaitLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Initialises a barrier for one arrival per phase (the arming thread's).
__device__ __forceinline__ void bulk_bar_init(uint64_t* bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}

// Makes barrier initialisations visible to the asynchronous proxy (the
// copy engine) before the first copy that signals them.
__device__ __forceinline__ void bulk_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier shared-memory accesses (through the CTA
// barrier that preceded it, every thread's) before later asynchronous
// copies into the same memory.
__device__ __forceinline__ void bulk_fence_proxy()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// The arming thread: expect `bytes` more bytes in the barrier's current phase
// and arrive.
__device__ __forceinline__ void bulk_expect(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Copies `bytes` from global `src` to shared `dst`; completion is counted
// on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Waits until the barrier's phase with the given parity has completed.
// Returns false when kBulkWaitLimit polls did not see it.
__device__ __forceinline__ bool bulk_wait(uint64_t* bar, uint32_t parity)
{
    const uint32_t a = smem_addr(bar);
    for (uint32_t i = 0; i < kBulkWaitLimit; ++i) {
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

}  // namespace fgs
