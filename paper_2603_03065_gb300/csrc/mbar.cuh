// Shared-memory barriers (mbarrier) and the copy engine's bulk and tiled
// loads, as inline PTX for sm_103a.  A copy adds its bytes to a barrier's
// transaction count; the phase completes once the expected bytes have landed
// and the expected arrivals have been made.  Waits are bounded in time (the
// global nanosecond timer), so a copy that never lands ends in an error the
// caller reports, not in a hang.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "gl.cuh"

namespace v3c {

using gl::u32;
using gl::u64;

__device__ __forceinline__ u64 global_timer_ns()
{
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ u32 smem_addr(const void* p) { return (u32)__cvta_generic_to_shared(p); }

// Barrier with `count` expected arrivals per phase.  Call from one thread,
// then mbar_init_fence, then a CTA barrier before any use.
__device__ __forceinline__ void mbar_init(u64* bar, u32 count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes initialised barriers visible to the copy engine.
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Orders this thread's earlier shared-memory accesses before copies it
// issues next into the same memory.
__device__ __forceinline__ void proxy_async_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(u64* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// One arrival plus `bytes` more expected from copies.
__device__ __forceinline__ void mbar_expect_tx(u64* bar, u32 bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(u64* bar, u32 parity)
{
    u32 done;
    asm volatile(
        "{\n\t"
        ".reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t"
        "}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Waits for the phase of `bar` with the given parity; false after limit_ns.
__device__ __forceinline__ bool mbar_wait(u64* bar, u32 parity, u64 limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const u64 t0 = global_timer_ns();
    for (u32 i = 1;; i++) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63) == 0 && global_timer_ns() - t0 > limit_ns) return false;
    }
}

// `bytes` contiguous bytes from global src to shared dst (both 16-byte
// aligned, bytes a multiple of 16), completing `bar`'s transaction count.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, u32 bytes, u64* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Tile (x, y) of a 2-D tensor map (x in elements, x times the element size a
// multiple of 16 bytes) into shared memory at dst, completing `bar`'s
// transaction count.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, u32 x, u32 y, u64* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<u64>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

}  // namespace v3c
