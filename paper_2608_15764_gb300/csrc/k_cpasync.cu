// k_cpasync.cu -- the cp.async streaming kernel.
//
// Paper §4.3 compares cp.async, which writes shared memory without a
// destination register, against plain loads at equal offered concurrency.
// Here each thread copies 16 bytes per commit group with
// cp.async.cg.shared.global into a D-slot ring and keeps D groups in flight:
// it waits until at most D-1 groups are pending (so the oldest has landed),
// reads that slot back with ld.shared and folds it, then refills the slot
// with the matching chunk of its next tile and commits.  A thread reads only
// the slot it wrote itself, so no CTA barrier is needed.
//
// The address sequence of a thread is the LDG kernel's at K = D: tile = cta*D
// vectors, CTA b walks tiles b, b+grid, ..., and chunk k of a tile is vector
// tile*cta*D + k*cta + t.  Only the way the loads are kept in flight differs.
#include "sl_device.cuh"

namespace sl {

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* gptr) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(gptr) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int D, int DT, bool COV = false>
__global__ void __launch_bounds__(D > 8 ? 512 : 1024) k_cpasync(const KArgs a) {
    // [D][cta]: slot k holds chunk k of a tile.  128-byte aligned; an
    // experiment flag (SL_DEBUG_SMEM_SKEW) can shift it by 16-byte steps.
    extern __shared__ __align__(128) uint4 ring[];
    cta_start(a);
    const uint32_t cta = blockDim.x;
    const uint4* __restrict__ buf = static_cast<const uint4*>(a.buf);
    const uint32_t ntiles = static_cast<uint32_t>(a.ntiles);
    const uint32_t total = static_cast<uint32_t>(a.total);
    const uint64_t nvec = a.nvec;
    const uint64_t tile_vec = static_cast<uint64_t>(cta) * D;
    const uint32_t skew = (static_cast<uint32_t>(a.debug) >> SL_DEBUG_SMEM_SKEW_SHIFT) & 7u;
    const uint32_t my0 = smem_addr(ring + skew + threadIdx.x), stride = cta * 16u;
    Acc<DT> acc;
    uint32_t full_tiles = 0;
    TileCursor c;
    c.start(ntiles);
    if (c.it < total) {
        // prologue: the D chunks of the first tile, one commit group each
        const uint64_t base = static_cast<uint64_t>(c.tile(a)) * tile_vec + threadIdx.x;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            if (base + static_cast<uint64_t>(k) * cta < nvec) {
                cp_async16(my0 + k * stride, buf + base + k * cta);
                cov_count<COV>(a, base + static_cast<uint64_t>(k) * cta);
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
            // last one or two of a pass): each chunk is folded and its slot
            // refilled with no range checks and no 64-bit bookkeeping.
            const uint4* np = buf + static_cast<uint64_t>(c.tile(a)) * tile_vec + threadIdx.x;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                cp_async_wait<D - 1>();
                acc.fold(lds16(my0 + k * stride));
                cp_async16(my0 + k * stride, np + static_cast<uint32_t>(k) * cta);
                cov_count<COV>(a, (np + static_cast<uint32_t>(k) * cta) - buf);
                cp_async_commit();
            }
            ++full_tiles;
            continue;
        }
        const uint64_t cbase = static_cast<uint64_t>(cur) * tile_vec + threadIdx.x;
        const uint64_t nbase = has_next ? static_cast<uint64_t>(c.tile(a)) * tile_vec + threadIdx.x : nvec;
        // vectors left from this thread's first chunk of the current / next
        // tile, clamped to 32 bits: chunk k is in range iff k*cta < rem
        const uint32_t crem = cbase < nvec ? static_cast<uint32_t>(min(nvec - cbase, static_cast<uint64_t>(0xFFFFFFFFu))) : 0u;
        const uint32_t nrem = nbase < nvec ? static_cast<uint32_t>(min(nvec - nbase, static_cast<uint64_t>(0xFFFFFFFFu))) : 0u;
        const bool cfull = cur < nwhole;
        const uint4* np = buf + (has_next ? nbase : 0);
        // the last tiles: chunks past the buffer's end are neither folded nor copied
        uint32_t off = 0;  // k * cta
#pragma unroll
        for (int k = 0; k < D; ++k) {
            // D groups are pending; wait until the oldest (chunk k of cur) has landed
            cp_async_wait<D - 1>();
            if (off < crem) {
                acc.fold(lds16(my0 + k * stride));
                if (!cfull) acc.n += 1;
            }
            // refill slot k with chunk k of the next tile (an empty group at the end)
            if (off < nrem) {
                cp_async16(my0 + k * stride, np + off);
                cov_count<COV>(a, (np + off) - buf);
            }
            cp_async_commit();
            off += cta;
        }
        if (cfull) ++full_tiles;
    }
    cp_async_wait<0>();
    acc.n += full_tiles * D;
    cta_finish<DT>(acc, true, threadIdx.x >> 5, cta >> 5, a);
}

template <int DT>
static const void* cpasync_for(int d) {
    switch (d) {
    case 1: return reinterpret_cast<const void*>(&k_cpasync<1, DT>);
    case 2: return reinterpret_cast<const void*>(&k_cpasync<2, DT>);
    case 3: return reinterpret_cast<const void*>(&k_cpasync<3, DT>);
    case 4: return reinterpret_cast<const void*>(&k_cpasync<4, DT>);
    case 5: return reinterpret_cast<const void*>(&k_cpasync<5, DT>);
    case 6: return reinterpret_cast<const void*>(&k_cpasync<6, DT>);
    case 7: return reinterpret_cast<const void*>(&k_cpasync<7, DT>);
    case 8: return reinterpret_cast<const void*>(&k_cpasync<8, DT>);
    case 9: return reinterpret_cast<const void*>(&k_cpasync<9, DT>);
    case 10: return reinterpret_cast<const void*>(&k_cpasync<10, DT>);
    case 11: return reinterpret_cast<const void*>(&k_cpasync<11, DT>);
    case 12: return reinterpret_cast<const void*>(&k_cpasync<12, DT>);
    case 13: return reinterpret_cast<const void*>(&k_cpasync<13, DT>);
    case 14: return reinterpret_cast<const void*>(&k_cpasync<14, DT>);
    case 15: return reinterpret_cast<const void*>(&k_cpasync<15, DT>);
    case 16: return reinterpret_cast<const void*>(&k_cpasync<16, DT>);
    default: return nullptr;
    }
}

const void* cpasync_cov_kernel(int d) {
    if (d == 1) return reinterpret_cast<const void*>(&k_cpasync<1, SL_U32, true>);
    if (d == 4) return reinterpret_cast<const void*>(&k_cpasync<4, SL_U32, true>);
    if (d == 16) return reinterpret_cast<const void*>(&k_cpasync<16, SL_U32, true>);
    return nullptr;
}

const void* cpasync_kernel(int dtype, int d) {
    switch (dtype) {
    case SL_U32: return cpasync_for<SL_U32>(d);
    case SL_F32: return cpasync_for<SL_F32>(d);
    case SL_BF16: return cpasync_for<SL_BF16>(d);
    case SL_FP8_E4M3: return cpasync_for<SL_FP8_E4M3>(d);
    default: return nullptr;
    }
}

}  // namespace sl
