// Bulk global -> shared copies completing on an mbarrier (no tensor map, no
// multicast), with bounded waits: a wait that gives up sets the caller's error
// flag and returns false instead of spinning on.
#pragma once

#include <cstdint>

namespace {

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}


// bulk global -> shared copy (no tensor map, no multicast); size multiple of 16
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// true when the phase completed; the thread may first be suspended for up
// to hint_ns while it has not
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

constexpr uint32_t kWaitLimit = 1u << 25;   // bounded spins of a non-suspending test (about a second)
constexpr uint32_t kSuspendLimit = 1u << 20;   // bounded suspending polls of at most 1 us each (about a second)

// bounded wait: true when the phase completed; false (error flag set) when the limit expired
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err) {
    for (uint32_t i = 0; i < kWaitLimit; ++i)
        if (mbar_test(bar, parity)) return true;
    atomicExch(err, 1);
    return false;
}


// bounded wait that lets the thread be suspended between polls (no issue
// slots spent spinning): true when the phase completed; false (error flag
// set) when the limit expired
__device__ __forceinline__ bool mbar_wait_suspend(uint64_t *bar, uint32_t parity, int *err) {
    for (uint32_t i = 0; i < kSuspendLimit; ++i)
        if (mbar_try(bar, parity, 1000u)) return true;
    atomicExch(err, 1);
    return false;
}

}  // namespace
