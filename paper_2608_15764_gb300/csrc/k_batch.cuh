// k_batch.cuh -- persistent kernels of the batched form.
//
// A batch is cut into work items (a piece of at most 1 MiB of one buffer).
// Every class kernel runs a persistent grid; its CTAs claim the class's
// items one at a time from an atomic counter (dynamic balancing across
// uneven buffers), fold each item with the class's mechanism and write one
// partial per folding warp per item, at the item's own partial slots, so the
// result does not depend on which CTA took which item.  kb_combine then adds
// the partials of each buffer in slot order.
#pragma once

#include "sl_device.cuh"

namespace sl {

struct BatchItem {
    const uint4* ptr;  // first vector of the item
    uint32_t nvec;     // 16-byte vectors in the item (> 0)
    uint32_t part;     // first partial slot of the item (one per folding warp)
};
static_assert(sizeof(BatchItem) == 16, "BatchItem layout");

struct BufSeg {
    uint32_t pstart;  // first partial slot of the buffer
    uint32_t pcount;  // partial slots of the buffer (items x folding warps)
};

struct BArgs {
    const BatchItem* items;  // this class's items
    uint32_t nitems;
    uint32_t stage_bytes;    // TMA stage size
    uint32_t* next;          // item counter (zeroed before every launch)
    WarpPartial* parts;      // the batch's partial array
    uint32_t* err;           // device error word
    uint64_t timeout_ns;     // bound of any single device wait (TMA)
    int32_t nst;             // TMA stages
    int32_t reserved;
};

// Thread 0 claims the next item; every thread of the CTA gets its index.
__device__ __forceinline__ uint32_t claim_item(const BArgs& a, volatile uint32_t* slot) {
    if (threadIdx.x == 0) *slot = atomicAdd(a.next, 1u);
    __syncthreads();
    const uint32_t i = *slot;
    __syncthreads();  // everyone has read the slot before it is overwritten
    return i;
}

// Reduce a warp's accumulators and let lane 0 write the warp's item partial.
template <int DT>
__device__ __forceinline__ void warp_item_store(const Acc<DT>& acc, WarpPartial* dst) {
    uint32_t s = acc.s;
    uint64_t x = (static_cast<uint64_t>(acc.xh) << 32) | acc.xl, n = acc.n;
    float hi = 0.0f, lo = 0.0f;
    if constexpr (DT != SL_U32) acc.float_part(hi, lo);
    warp_merge<DT>(s, x, n, hi, lo);
    if ((threadIdx.x & 31) == 0) {
        WarpPartial p;
        p.sum = s;
        p.pad = 0;
        p.xr = x;
        p.issued = n;
        p.hi = hi;
        p.lo = lo;
        *dst = p;
    }
}

// LDG class kernel: per item, tiles of CTA*K vectors, K independent 16-byte
// loads per thread per tile (same fold and tile layout as k_ldg), guarded
// ragged tail.
template <int K, int CTA, int DT>
__global__ void __launch_bounds__(CTA, ldg_min_blocks<K, CTA, DT>()) kb_ldg(const BArgs a) {
    __shared__ uint32_t slot;
    constexpr uint32_t TILE = static_cast<uint32_t>(CTA) * K;
    for (;;) {
        const uint32_t item = claim_item(a, &slot);
        if (item >= a.nitems) break;
        const BatchItem it = a.items[item];
        Acc<DT> acc;
        const uint32_t nfull = it.nvec / TILE;
        const uint4* p = it.ptr + threadIdx.x;
#pragma unroll 1
        for (uint32_t t = 0; t < nfull; ++t, p += TILE) {
            uint4 v[K];
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = ldg16<SL_COP_CG>(p + k * CTA);
#pragma unroll
            for (int k = 0; k < K; ++k) acc.fold(v[k]);
        }
        acc.n = nfull * K;
        const uint32_t rem = it.nvec - nfull * TILE;
        if (rem) {
            uint4 v[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if (threadIdx.x + k * CTA < rem) v[k] = ldg16<SL_COP_CG>(p + k * CTA);
                else v[k] = make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if (threadIdx.x + k * CTA < rem) {
                    acc.fold(v[k]);
                    acc.n += 1;
                }
            }
        }
        warp_item_store<DT>(acc, a.parts + it.part + (threadIdx.x >> 5));
    }
}

}  // namespace sl
