// k_cpasync.cuh -- the cp.async streaming kernel (instantiated in
// k_cpasync.cu for one copy per commit group, k_cpasync_g.cu for several).
//
// Paper §4.3 compares cp.async, which writes shared memory without a
// destination register, against plain loads at equal offered concurrency.
// Here each thread puts G 16-byte copies (cp.async.cg.shared.global) in each
// commit group and keeps D groups in flight in a D x G slot ring: it waits
// until at most D-1 groups are pending (so the oldest has landed), reads that
// group's G slots back with ld.shared and folds them, then refills the slots
// with the matching copies of its next tile and commits.  A thread reads only
// the slots it wrote itself, so no CTA barrier is needed.  G = 1 is the
// paper's cell: one copy, one commit and one wait per 16 bytes; G > 1 shares
// a commit and a wait among G copies at the same D*G*16 bytes in flight.
//
// The address sequence of a thread is the LDG kernel's at K = D*G: tile =
// cta*D*G vectors, CTA b walks tiles b, b+grid, ..., and copy j = k*G + g of a
// tile (group k, copy g) is vector tile*cta*D*G + j*cta + t.  Only the way the
// loads are kept in flight differs.
#pragma once
#include "sl_device.cuh"

namespace sl {

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* gptr) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(gptr) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int D, int G, int DT, bool COV = false>
__global__ void __launch_bounds__(D * G > 8 ? 512 : 1024) k_cpasync(const KArgs a) {
    // [D*G][cta]: slot j = k*G + g holds copy j of a tile.  128-byte aligned;
    // an experiment flag (SL_DEBUG_SMEM_SKEW) can shift it by 16-byte steps.
    extern __shared__ __align__(128) uint4 ring[];
    cta_start(a);
    const uint32_t cta = blockDim.x;
    const uint4* __restrict__ buf = static_cast<const uint4*>(a.buf);
    const uint32_t ntiles = static_cast<uint32_t>(a.ntiles);
    const uint32_t total = static_cast<uint32_t>(a.total);
    const uint64_t nvec = a.nvec;
    const uint64_t tile_vec = static_cast<uint64_t>(cta) * (D * G);
    const uint32_t skew = (static_cast<uint32_t>(a.debug) >> SL_DEBUG_SMEM_SKEW_SHIFT) & 7u;
    const uint32_t my0 = smem_addr(ring + skew + threadIdx.x), stride = cta * 16u;
    Acc<DT> acc;
    uint32_t full_tiles = 0;
    TileCursor c;
    c.start(ntiles);
    if (c.it < total) {
        // prologue: the D groups of the first tile, G copies each
        const uint64_t base = static_cast<uint64_t>(c.tile(a)) * tile_vec + threadIdx.x;
#pragma unroll
        for (int k = 0; k < D; ++k) {
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const uint32_t j = k * G + g;
                if (base + static_cast<uint64_t>(j) * cta < nvec) {
                    cp_async16(my0 + j * stride, buf + base + j * cta);
                    cov_count<COV>(a, base + static_cast<uint64_t>(j) * cta);
                }
            }
            cp_async_commit();
        }
    }
    const uint32_t nwhole = static_cast<uint32_t>(nvec / tile_vec);  // whole tiles of a pass: 0 .. nwhole-1
#pragma unroll 1
    while (c.it < total) {
        const uint32_t cur = c.tile(a);
        c.next(ntiles);
        const bool has_next = c.it < total;
        if (cur < nwhole && has_next && c.tile(a) < nwhole) {
            // The current and the next tile are both whole (every tile but the
            // last one or two of a pass): each group is folded and its slots
            // refilled with no range checks and no 64-bit bookkeeping.
            const uint4* np = buf + static_cast<uint64_t>(c.tile(a)) * tile_vec + threadIdx.x;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                cp_async_wait<D - 1>();
#pragma unroll
                for (int g = 0; g < G; ++g) acc.fold(lds16(my0 + (k * G + g) * stride));
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const uint32_t j = k * G + g;
                    cp_async16(my0 + j * stride, np + j * cta);
                    cov_count<COV>(a, (np + j * cta) - buf);
                }
                cp_async_commit();
            }
            ++full_tiles;
            continue;
        }
        const uint64_t cbase = static_cast<uint64_t>(cur) * tile_vec + threadIdx.x;
        const uint64_t nbase = has_next ? static_cast<uint64_t>(c.tile(a)) * tile_vec + threadIdx.x : nvec;
        // vectors left from this thread's first copy of the current / next
        // tile, clamped to 32 bits: copy j is in range iff j*cta < rem
        const uint32_t crem = cbase < nvec ? static_cast<uint32_t>(min(nvec - cbase, static_cast<uint64_t>(0xFFFFFFFFu))) : 0u;
        const uint32_t nrem = nbase < nvec ? static_cast<uint32_t>(min(nvec - nbase, static_cast<uint64_t>(0xFFFFFFFFu))) : 0u;
        const bool cfull = cur < nwhole;
        const uint4* np = buf + (has_next ? nbase : 0);
        // the last tiles: copies past the buffer's end are neither folded nor issued
#pragma unroll
        for (int k = 0; k < D; ++k) {
            // D groups are pending; wait until the oldest (group k of cur) has landed
            cp_async_wait<D - 1>();
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const uint32_t j = k * G + g;
                if (j * cta < crem) {
                    acc.fold(lds16(my0 + j * stride));
                    if (!cfull) acc.n += 1;
                }
            }
            // refill group k's slots with the next tile's copies (an empty group at the end)
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const uint32_t j = k * G + g;
                if (j * cta < nrem) {
                    cp_async16(my0 + j * stride, np + j * cta);
                    cov_count<COV>(a, (np + j * cta) - buf);
                }
            }
            cp_async_commit();
        }
        if (cfull) ++full_tiles;
    }
    cp_async_wait<0>();
    acc.n += full_tiles * (D * G);
    cta_finish<DT>(acc, true, threadIdx.x >> 5, cta >> 5, a);
}

template <int D, int G, int DT>
__host__ const void* cpasync_fn() {
    return reinterpret_cast<const void*>(&k_cpasync<D, G, DT>);
}

}  // namespace sl
