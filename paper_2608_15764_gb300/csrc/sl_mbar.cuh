// sl_mbar.cuh -- mbarrier, bulk-copy and bounded-wait helpers of the TMA
// rings (single-buffer and batched).
//
// Every wait is bounded: a wait that exceeds timeout_ns (by %globaltimer) or
// a hard iteration cap records an error code in *err, raises the CTA's abort
// flag and returns false; waiters that watch the abort flag give up when they
// see it.
#pragma once

#include "sl_device.cuh"

namespace sl {

constexpr uint32_t WAIT_ITER_CAP = 1u << 22;  // last-resort cap if %globaltimer were not to advance

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t tx) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(tx) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// Bounded wait for the phase of `bar` with the given parity to complete.
// Returns false on timeout (after recording `code`) or when the abort flag is
// seen (if watch_abort).
__device__ __forceinline__ bool bounded_wait(uint32_t bar, uint32_t parity, uint32_t* err, uint64_t timeout_ns,
                                             volatile int* abort_flag, bool watch_abort, uint32_t code) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t start = gtimer();
    for (uint32_t n = 0; n < WAIT_ITER_CAP; ++n) {
        if (mbar_try_wait(bar, parity)) return true;
        if (watch_abort && *abort_flag) return false;
        if (gtimer() - start > timeout_ns) break;
    }
    atomicCAS(err, 0u, code);
    *abort_flag = 1;
    return false;
}

// Initialise nst full barriers (count 1) and nst empty barriers (count
// `consumers`) and make them visible to the bulk-copy (async) proxy.
__device__ __forceinline__ void ring_init(uint32_t full0, uint32_t empty0, uint32_t nst, uint32_t consumers) {
    for (uint32_t s = 0; s < nst; ++s) {
        mbar_init(full0 + 8 * s, 1);
        mbar_init(empty0 + 8 * s, consumers);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace sl
