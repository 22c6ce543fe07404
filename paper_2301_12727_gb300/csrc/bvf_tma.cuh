// Inline-PTX helpers for the tensor-memory accelerator (TMA) and mbarriers
// used by the TMA-fed acoustic kernels (sm_90 and later, here sm_103a).
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace bvf {
namespace tma {

__device__ __forceinline__ unsigned saddr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}

// return an mbarrier's shared memory to plain use (before re-initialising it
// for the next tile of a persistent block)
__device__ __forceinline__ void mbar_inval(uint64_t *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(saddr(bar)) : "memory");
}

// make a tensor map that sits in global memory (written before the launch)
// visible to the tensor-map proxy before this thread's copies use it
__device__ __forceinline__ void tensormap_acquire(const void *map)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}

__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// arrive once and add `bytes` to the transaction count of the current phase
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n"
        " selp.u32 %0, 1, 0, P;\n}\n"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of the given parity: at most `limit` polls, then
// false (the phase has not completed).  The caller records the time-out and
// stops issuing copies; see the acoustic and projection kernels.
constexpr unsigned kWaitLimit = 1u << 22;
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, unsigned limit)
{
    for (unsigned it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// bring the 128-byte line holding p into L2 ahead of its use (no register
// result; the address lies inside an allocation)
__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// order this thread's generic-proxy shared-memory accesses before later
// async-proxy (TMA) accesses
__device__ __forceinline__ void fence_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// global -> shared tile load of a 3-D tensor map box at (x, y, z); completion
// is counted in bytes on `bar`.  Out-of-range elements are zero-filled.
__device__ __forceinline__ void load3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                       uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(saddr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(saddr(bar))
        : "memory");
}

// shared -> global tile store; out-of-range elements are not written
__device__ __forceinline__ void store3d(const CUtensorMap *map, int x, int y, int z, const void *src)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(map),
        "r"(x), "r"(y), "r"(z), "r"(saddr(src))
        : "memory");
}

__device__ __forceinline__ void bulk_commit()
{
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// wait until at most N committed store groups are still reading shared memory
template <int N>
__device__ __forceinline__ void bulk_wait_read()
{
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

// wait until at most N committed store groups are still in flight
template <int N>
__device__ __forceinline__ void bulk_wait()
{
    asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace tma
}  // namespace bvf
