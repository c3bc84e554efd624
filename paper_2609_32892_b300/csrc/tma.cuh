// Bulk asynchronous copies global -> shared memory through the tensor memory
// accelerator (cp.async.bulk, completion counted on an mbarrier), for the
// streaming stencil passes.  Every wait is bounded: a kernel whose wait gives
// up sets kStatusTimeout in its DevState status word (lbm_sync then returns
// LBM_ERR_TIMEOUT) instead of spinning for ever.
#pragma once

#include <stdint.h>

#include "lbm_common.cuh"

namespace lbm {

constexpr unsigned kStatusTimeout = 4u;     // DevState::status bit: a bounded wait gave up
constexpr long long kWaitTries = 1LL << 22; // mbarrier try_wait attempts before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// mbarrier with `count` expected arrivals, made visible to the async proxy
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one arrival that also announces `bytes` of asynchronous copies to come
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// one arrival without transactions (completes the phase of a count-1 barrier)
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// `bytes` (a multiple of 16, both addresses 16-byte aligned) from global to shared
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for the phase with the given parity to complete; false if it did not
// within kWaitTries attempts.  Lanes that issue copies must all have issued
// them (__syncwarp) before any lane of their warp waits: a diverged warp does
// not interleave its two paths fairly, and waiting lanes can use up their
// attempts before the issuing lanes run.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (long long i = 0; i < kWaitTries; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// After a wait gave up: flag it, then wait once more (bounded) so that the
// block does not leave while its copies may still be landing.
__device__ __forceinline__ void mbar_give_up(uint64_t* bar, uint32_t parity, DevState* st) {
    atomicOr(&st->status, kStatusTimeout);  // every thread that gave up: none goes unreported
    mbar_wait(bar, parity);
}

}  // namespace lbm
