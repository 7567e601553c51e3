// mbarrier helpers shared by the tensor-core GEMM and the wait diagnostic.
// Every wait is bounded by %globaltimer: on expiry it records DUST_ETIMEOUT
// in the caller's status word (and raises the CTA's abort flag) instead of
// spinning on, so a kernel whose producer never arrives still returns.
#pragma once
#include "dust_internal.cuh"

namespace dust {
namespace {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase with the given parity; false on timeout or abort.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          int *status, unsigned long long limit_ns = WAIT_NS) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 255) == 0) {
            if (*abort_flag) return false;
            if (globaltimer_ns() - t0 > limit_ns) {
                *abort_flag = 1;
                record_status(status, DUST_ETIMEOUT);
                return false;
            }
        }
    }
}
// Bounded wait that ignores the abort flag (used to drain asynchronous work
// before shared memory or tensor memory is released).
__device__ __forceinline__ void mbar_drain(uint64_t *bar, uint32_t parity, int *status) {
    const unsigned long long t0 = globaltimer_ns();
    while (!mbar_try(bar, parity)) {
        if (globaltimer_ns() - t0 > WAIT_NS) { record_status(status, DUST_ETIMEOUT); return; }
    }
}
}  // namespace
}  // namespace dust
