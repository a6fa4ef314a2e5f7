// PTX helpers shared by the force kernels: mbarrier initialisation and
// phase waits, bulk global -> shared copies on the TMA engine, and a
// globaltimer-bounded wait so that no kernel can spin forever on a copy.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nb {

// ---------------------------------------------------------------------------
// PTX helpers: mbarrier + bulk copies (TMA engine), all waits bounded.
// ---------------------------------------------------------------------------

static constexpr unsigned long long WAIT_LIMIT_NS = 4000000000ull;  // 4 s

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Global -> shared bulk copy, completion signalled on bar (bytes % 16 == 0,
// both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of bar; gives up after limit_ns (WAIT_LIMIT_NS).
static __device__ __noinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                       unsigned long long limit_ns = WAIT_LIMIT_NS)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (;;) {
        for (int k = 0; k < 32; ++k)
            if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer() - t0 > limit_ns) return false;
    }
}

// After a wait gave up at tile kt, let the copies already issued (tiles kt ..
// kt + NS - 1 of n_tiles, ring position seq0 + tile) land before the CTA stops
// using its shared memory: one more bounded wait on each. Thread 0 only.
template <int NS>
__device__ __noinline__ void drain_ring(uint64_t *full, unsigned seq0, int kt, int n_tiles)
{
    for (int q = kt; q < n_tiles && q < kt + NS; ++q) {
        const unsigned sq = seq0 + (unsigned)q;
        mbar_wait(&full[sq % NS], (sq / NS) & 1u);
    }
}

}  // namespace nb
