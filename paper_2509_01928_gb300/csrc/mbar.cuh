// Shared-memory mbarrier helpers with bounded waits (inline PTX, sm_100+).
//
// Every wait on an mbarrier phase gives up after a time limit measured with
// %globaltimer: it then sets DEV_ERR_TIMEOUT in the handle's device error word
// and raises the CTA's abort flag, so the kernel can drain its copies, free
// what it holds and return. The host maps the error word to ISING_ERR_TIMEOUT.
#pragma once

#include <stdint.h>

#include "internal.cuh"

namespace doch {

constexpr uint64_t kWaitNs = 1000000000ull;  // default limit of a bounded wait: 1 s

__device__ __forceinline__ uint32_t saddr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t gtime() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned long long *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait for a long phase (the accumulator): polls every ~0.5 us so the
// waiting warps leave the issue slots to the producer, MMA and converter threads
__device__ __forceinline__ bool mbar_wait_idle(unsigned long long *bar, uint32_t parity, int *err,
                                               volatile int *abort_flag, uint64_t limit_ns = kWaitNs) {
    const uint64_t t0 = gtime();
    while (!mbar_test(bar, parity)) {
        if (*abort_flag) return false;
        if (gtime() - t0 > limit_ns) {
            atomicOr(err, DEV_ERR_TIMEOUT);
            *abort_flag = 1;
            return false;
        }
        __nanosleep(500);
    }
    return true;
}

// bounded wait on a phase parity; false (and the error word set) on timeout
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity, int *err,
                                          volatile int *abort_flag, uint64_t limit_ns = kWaitNs) {
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = gtime();
    while (true) {
        if (mbar_test(bar, parity)) return true;
        if (*abort_flag) return false;
        if (gtime() - t0 > limit_ns) {
            atomicOr(err, DEV_ERR_TIMEOUT);
            *abort_flag = 1;
            return false;
        }
    }
}

}  // namespace doch
