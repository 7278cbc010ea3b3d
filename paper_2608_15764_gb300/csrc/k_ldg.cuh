// k_ldg.cuh -- the plain-load (LDG) streaming kernel.
//
// Paper §3 "The axis K": K is the number of independent ld.global
// instructions a thread issues per iteration before consuming them.  Paper §3
// "Fixed-work control": total issued logical loads are the same at every K;
// here exactly one 16-byte load per 16 bytes per pass (the last tile is
// guarded instead of rounding the iteration count).  Each warp instruction
// reads 32 consecutive 16-byte vectors (512 contiguous bytes), so every
// warp's access is contiguous and fully coalesced at every K.
//
// Tile = cta*K vectors.  CTA b walks tiles b, b+grid, b+2*grid, ... over all
// passes (tile index taken mod the tiles per pass; reversed for SL_DESC).
// Load k of thread t reads vector tile*cta*K + k*cta + t.
#pragma once

#include "sl_device.cuh"

namespace sl {

template <int K, int CTA, int DT, int COP, bool COV = false>
__global__ void __launch_bounds__(CTA, ldg_min_blocks<K, CTA, DT>()) k_ldg(const KArgs a) {
    // launch_bounds(CTA, 1) lets ptxas keep all K loaded vectors in registers
    // (4K registers) instead of interleaving loads with folds to save
    // registers (bfloat16 folds at K <= 8: see ldg_min_blocks); configurations
    // whose kernel would spill are rejected on the host (local memory > 0), as
    // the paper requires zero spills (§3).
    constexpr uint32_t TILE = static_cast<uint32_t>(CTA) * K;
    cta_start(a);
    const uint4* __restrict__ buf = static_cast<const uint4*>(a.buf);
    const uint32_t ntiles = static_cast<uint32_t>(a.ntiles);
    const uint32_t total = static_cast<uint32_t>(a.total);
    const bool last_full = (a.nvec == static_cast<uint64_t>(ntiles) * TILE);
    Acc<DT> acc;
    uint32_t full_iters = 0;
    TileCursor c;
    c.start(ntiles);
#pragma unroll 1
    for (; c.it < total; c.next(ntiles)) {
        const uint32_t tile = c.tile(a);
        const uint4* p = buf + static_cast<uint64_t>(tile) * TILE + threadIdx.x;
        uint4 v[K];
        if (last_full || tile + 1 < ntiles) {
            // K independent loads issued back to back, then consumed.
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = ldg16<COP>(p + k * CTA);
            if constexpr (COV) {
#pragma unroll
                for (int k = 0; k < K; ++k) cov_count<COV>(a, (p + k * CTA) - buf);
            }
#pragma unroll
            for (int k = 0; k < K; ++k) acc.fold(v[k]);
            ++full_iters;
        } else {
            // Ragged last tile: only vectors below nvec are loaded.
            const uint32_t rem = static_cast<uint32_t>(a.nvec - static_cast<uint64_t>(tile) * TILE);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if (threadIdx.x + k * CTA < rem) {
                    v[k] = ldg16<COP>(p + k * CTA);
                    cov_count<COV>(a, (p + k * CTA) - buf);
                } else {
                    v[k] = make_uint4(0u, 0u, 0u, 0u);
                }
            }
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if (threadIdx.x + k * CTA < rem) {
                    acc.fold(v[k]);
                    acc.n += 1;
                }
            }
        }
    }
    acc.n += full_iters * K;
    cta_finish<DT>(acc, true, threadIdx.x >> 5, CTA / 32, a);
}

// SL_DYN traversal: CTAs claim contiguous chunks of a.tile_vec vectors (a
// multiple of CTA*K, about 1 MiB) from the counter *a.next, so each CTA
// streams long contiguous runs and faster CTAs take more chunks.  Within a
// chunk the tiles and loads are those of k_ldg (K independent 16-byte loads
// per thread per tile, guarded ragged tail).  Thread 0 claims the following
// chunk while the CTA works on the current one (one CTA barrier per chunk).
// Integer results are exact; float sums are correct to the same bound but not
// bit-reproducible between runs, since a CTA's partial covers whichever
// chunks it claimed.
template <int K, int CTA, int DT, bool COV = false>
__global__ void __launch_bounds__(CTA, ldg_min_blocks<K, CTA, DT>()) k_ldg_dyn(const KArgs a) {
    constexpr uint32_t TILE = static_cast<uint32_t>(CTA) * K;
    __shared__ uint32_t slot[2];
    cta_start(a);
    const uint4* __restrict__ buf = static_cast<const uint4*>(a.buf);
    const uint32_t chunk_vec = a.tile_vec;
    const uint32_t nchunks = static_cast<uint32_t>(a.ntiles);
    const uint32_t total = static_cast<uint32_t>(a.total);
    Acc<DT> acc;
    uint32_t full_iters = 0;
    volatile uint32_t* vslot = slot;
    if (threadIdx.x == 0) vslot[0] = atomicAdd(a.next, 1u);
    __syncthreads();
    uint32_t cur = vslot[0];
#pragma unroll 1
    for (uint32_t j = 0; cur < total; ++j) {
        if (threadIdx.x == 0) vslot[(j + 1) & 1] = atomicAdd(a.next, 1u);
        const uint64_t base = static_cast<uint64_t>(cur % nchunks) * chunk_vec;
        const uint64_t left = a.nvec - base;
        const uint32_t len = left < chunk_vec ? static_cast<uint32_t>(left) : chunk_vec;
        const uint4* p = buf + base + threadIdx.x;
        const uint32_t nfull = len / TILE;
#pragma unroll 1
        for (uint32_t t = 0; t < nfull; ++t, p += TILE) {
            uint4 v[K];
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = ldg16<SL_COP_CG>(p + k * CTA);
            if constexpr (COV) {
#pragma unroll
                for (int k = 0; k < K; ++k) cov_count<COV>(a, (p + k * CTA) - buf);
            }
#pragma unroll
            for (int k = 0; k < K; ++k) acc.fold(v[k]);
        }
        full_iters += nfull;
        const uint32_t rem = len - nfull * TILE;
        if (rem) {
            uint4 v[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if (threadIdx.x + k * CTA < rem) {
                    v[k] = ldg16<SL_COP_CG>(p + k * CTA);
                    cov_count<COV>(a, (p + k * CTA) - buf);
                } else {
                    v[k] = make_uint4(0u, 0u, 0u, 0u);
                }
            }
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if (threadIdx.x + k * CTA < rem) {
                    acc.fold(v[k]);
                    acc.n += 1;
                }
            }
        }
        __syncthreads();  // the prefetched claim is visible; the slot read next is not rewritten until j+2
        cur = vslot[(j + 1) & 1];
    }
    acc.n += full_iters * K;
    cta_finish<DT>(acc, true, threadIdx.x >> 5, CTA / 32, a);
}

}  // namespace sl

// Table of instantiations K = 1..16 x CTA sizes x load flavours for one dtype.
#define SL_LDG_K_CASES(FN, ...)                                                        \
    switch (k) {                                                                       \
    case 1: return FN<1, __VA_ARGS__>();  case 2: return FN<2, __VA_ARGS__>();             \
    case 3: return FN<3, __VA_ARGS__>();  case 4: return FN<4, __VA_ARGS__>();             \
    case 5: return FN<5, __VA_ARGS__>();  case 6: return FN<6, __VA_ARGS__>();             \
    case 7: return FN<7, __VA_ARGS__>();  case 8: return FN<8, __VA_ARGS__>();             \
    case 9: return FN<9, __VA_ARGS__>();  case 10: return FN<10, __VA_ARGS__>();           \
    case 11: return FN<11, __VA_ARGS__>(); case 12: return FN<12, __VA_ARGS__>();          \
    case 13: return FN<13, __VA_ARGS__>(); case 14: return FN<14, __VA_ARGS__>();          \
    case 15: return FN<15, __VA_ARGS__>(); case 16: return FN<16, __VA_ARGS__>();          \
    default: return nullptr;                                                           \
    }

namespace sl {
template <int K, int CTA, int DT, int COP>
const void* ldg_ptr() { return reinterpret_cast<const void*>(&k_ldg<K, CTA, DT, COP>); }

template <int CTA, int DT, int COP>
const void* ldg_pick_k(int k) { SL_LDG_K_CASES(ldg_ptr, CTA, DT, COP) }
}  // namespace sl
