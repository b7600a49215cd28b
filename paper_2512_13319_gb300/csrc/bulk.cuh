// Bulk copies on the tensor memory accelerator (TMA): global -> shared
// completing on an mbarrier in shared memory, with a bounded wait (a tile's
// contiguous per-step inputs staged with one instruction instead of per-thread
// strided loads), and shared -> global in bulk groups (a tile's outputs written
// with one instruction).
//
// Requirements (checked by the callers): source and destination 16-byte
// aligned, size a multiple of 16 bytes and below 2^20 (the transaction count
// of one mbarrier phase).
#pragma once
#include <cuda_runtime.h>

namespace mapk {

__device__ __forceinline__ unsigned smem_addr(const void* p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    // make the initialised barrier visible to the async (TMA) proxy
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one arrival that also announces `bytes` of transactions for this phase
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity)
{
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for phase `parity` of the barrier, giving up after `limit` polls (each
// poll may itself suspend the thread for a bounded time).  Returns whether
// the phase completed.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity, int limit)
{
    for (int i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

constexpr int MBAR_POLLS = 1 << 22;

// Bulk shared -> global copy (bulk-group completion).  The generic-proxy
// writes of the source must be made visible to the async proxy first
// (fence_proxy_async_smem by the issuing thread after a block barrier).
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void bulk_copy_s2g(void* dst, const void* src, unsigned bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
                 "r"(bytes)
                 : "memory");
}

// commit the issued bulk copies as one group and wait until all of them have
// completed (source read and destination written)
__device__ __forceinline__ void bulk_commit_and_wait()
{
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// start bringing the bytes at src into L2 (the range widened to whole 16-byte
// words: the caller's allocation must hold them); nothing waits for it, later
// loads of the range hit L2
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, unsigned bytes)
{
    const unsigned long long a = reinterpret_cast<unsigned long long>(src);
    const unsigned long long lo = a & ~15ull, hi = (a + bytes + 15ull) & ~15ull;
    if (hi > lo)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"((unsigned)(hi - lo)) : "memory");
}

}  // namespace mapk
