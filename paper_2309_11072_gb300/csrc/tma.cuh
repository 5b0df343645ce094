// Bulk asynchronous copies (TMA, cp.async.bulk) into shared memory with
// mbarrier completion, and a bounded wait.
//
// A wait that does not complete within kMaxSpins polls records an error code
// in a device status word (the caller's; the library's is read with
// slrme_device_status) and reports failure; kernels then stop issuing work
// and return, so a lost copy can never hang the GPU.
#pragma once

#include <stdint.h>

namespace slrme {

constexpr int kStatusWaitTimeout = 1;   // bit 0: an mbarrier wait gave up

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Makes barrier initialisation and earlier generic-proxy accesses of shared
// memory visible to the async proxy (the TMA unit).
__device__ __forceinline__ void fence_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// 1-D bulk copy global -> shared (dst, src and bytes multiples of 16).
__device__ __forceinline__ void tma_load_1d(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

constexpr int kMaxSpins = 1 << 22;

// Waits for phase `parity` of the barrier; false (and the status word set)
// if it did not complete within the bound.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* status, int max_spins = kMaxSpins) {
    for (int i = 0; i < max_spins; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    atomicOr(status, kStatusWaitTimeout);
    return false;
}

// The same wait for all 32 lanes of a warp together: the warp polls until
// every lane sees the phase complete, so the lanes return the same outcome.
__device__ __forceinline__ bool mbar_wait_warp(uint32_t bar, uint32_t parity, int* status,
                                               int max_spins = kMaxSpins) {
    for (int i = 0; i < max_spins; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (__all_sync(0xffffffffu, done != 0u)) return true;
    }
    if ((threadIdx.x & 31) == 0) atomicOr(status, kStatusWaitTimeout);
    return false;
}

}  // namespace slrme
