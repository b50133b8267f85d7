// Asynchronous bulk copies from this GPU's global memory into the issuing
// block's own shared memory (cp.async.bulk, no tensor map, no multicast),
// completed through a shared-memory mbarrier that counts the bytes landed.
//
// Rules of the copy unit: both addresses 16-byte aligned, the size a
// multiple of 16 bytes.  Callers copy the 16-byte-aligned body of a range
// with one bulk copy and load the few elements outside it with plain loads.
// Every wait on a barrier is bounded: after kBulkPollLimit polls the waiter
// gives up and reports false, so a kernel always terminates.
#pragma once

#include <cstdint>

namespace ldni {

constexpr int kBulkPollLimit = 1 << 22;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// One thread initialises; a fence makes the barrier visible to the copy unit.
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t arrivals) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(arrivals) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// The calling thread arrives and announces `bytes` of copies to come.
__device__ __forceinline__ void mbar_arrive_expect(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// The calling thread arrives (no copies announced).
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// bytes (> 0, multiple of 16) from src (global, 16-byte aligned) to dst
// (shared, 16-byte aligned); completion counted on bar.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
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

// Wait for phase `parity` of bar to complete; false after kBulkPollLimit polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (int k = 0; k < kBulkPollLimit; ++k)
        if (mbar_test(bar, parity)) return true;
    return false;
}

// Issues the bulk part of copying elements [g0, g1) of a 4-byte array whose
// base is 16-byte aligned into dst, where dst[i - floor4(g0)] receives
// element i: the body [floor4(g0), floor4(g1)) by one bulk copy (returns its
// bytes, 0 when empty).  The tail [floor4(g1), g1) is the caller's, by plain
// loads (tail_load).  Nothing outside [floor4(g0), g1) is read.
__device__ __forceinline__ uint32_t bulk_range4(void *dst, const void *base, long long g0, long long g1,
                                                uint64_t *bar) {
    const long long s = g0 & ~3ll, e = g1 & ~3ll;
    if (e <= s) return 0;
    const uint32_t bytes = (uint32_t)((e - s) * 4);
    bulk_load(dst, static_cast<const char *>(base) + s * 4, bytes, bar);
    return bytes;
}

// Plain loads of the tail [max(floor4(g1), g0), g1) of the range, by threads
// t < 4 of the block.
__device__ __forceinline__ void tail_load(uint32_t *dst, const uint32_t *base, long long g0, long long g1) {
    const long long s = g0 & ~3ll, e = g1 & ~3ll;
    const long long i = e + (long long)threadIdx.x;
    if (threadIdx.x < 4 && i < g1 && i >= g0) dst[i - s] = base[i];
}

}  // namespace ldni
