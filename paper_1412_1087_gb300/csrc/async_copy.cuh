// Copies by the tensor-memory-access engine into shared memory, completed on
// shared-memory mbarriers, and the time-limited waits on them.
#pragma once

#include <stdint.h>

namespace mhdpic {

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ long long timer_ns()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// one arrival per phase (the thread that posts the expected bytes)
__device__ __forceinline__ void mbar_init(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// true when the phase completed within limit_ns
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, long long limit_ns)
{
    const long long t0 = timer_ns();
    while (!mbar_try_wait(bar, parity))
        if (timer_ns() - t0 > limit_ns)
            return false;
    return true;
}

// Orders this thread's earlier generic accesses to shared memory before the
// copies it issues next (a buffer being refilled), and makes mbarrier
// initialisations visible to the copy engine.
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Contiguous copy of `bytes` (a multiple of 16) from global src to shared
// dst, both 16-byte aligned, completing on bar.
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// The default wait limit of a copy, and the limit of the wait that drains the
// copies still in flight before a block that gave up returns (so none lands
// in shared memory after the block has gone).
constexpr long long COPY_LIMIT_NS = 1000000000ll;   // one second

}  // namespace mhdpic
