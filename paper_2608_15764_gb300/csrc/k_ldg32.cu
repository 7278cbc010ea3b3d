// k_ldg32.cu -- the 32-byte-width plain-load kernels (SL_LDG32).
//
// The paper sweeps load width as well as K (§3: 4- and 16-byte cells; its
// regime map is over warps x width).  sm_100-class GPUs add 256-bit global
// loads (ld.global.v8.u32), so the library adds a 32-byte width: K independent
// 32-byte loads per thread per iteration, issued before any is consumed; one
// warp instruction reads 1,024 contiguous bytes.
//
// Units are 32-byte vectors.  Tile = CTA*K units; load k of thread t reads
// unit tile*CTA*K + k*CTA + t.  A buffer whose size is an odd number of
// 16-byte vectors has a half unit at the end: the thread whose unit index is
// the first past the whole units loads that last 16-byte vector instead.
// The grid-stride kernel walks tiles like k_ldg; the SL_DYN kernel claims
// ~1 MiB chunks like k_ldg_dyn.  issued_loads counts loads: 32-byte loads plus
// the one 16-byte load of a half unit, per pass.
#include "sl_device.cuh"

namespace sl {

struct Oct {
    uint4 lo, hi;
};

// One 32-byte load (.cg: cached in L2 only); the address is 32-byte aligned.
__device__ __forceinline__ Oct ldg32(const Oct* p) {
    Oct v;
    asm volatile("ld.global.cg.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v.lo.x), "=r"(v.lo.y), "=r"(v.lo.z), "=r"(v.lo.w), "=r"(v.hi.x), "=r"(v.hi.y),
                   "=r"(v.hi.z), "=r"(v.hi.w)
                 : "l"(p));
    return v;
}

// Guarded tail of a tile or chunk: units below n32 load 32 bytes, the unit
// n32 itself (when the buffer ends in a half unit) loads the last 16 bytes.
template <int K, int CTA, int DT, bool COV>
__device__ __forceinline__ void ragged32(const KArgs& a, const Oct* buf, uint64_t first, uint64_t n32, bool half,
                                         Acc<DT>& acc) {
#pragma unroll 1
    for (int k = 0; k < K; ++k) {
        const uint64_t u = first + static_cast<uint64_t>(k) * CTA + threadIdx.x;
        if (u < n32) {
            const Oct v = ldg32(buf + u);
            cov_count<COV>(a, 2 * u);
            cov_count<COV>(a, 2 * u + 1);
            acc.fold(v.lo);
            acc.fold(v.hi);
            acc.n += 1;
        } else if (half && u == n32) {
            acc.fold(ldg16<SL_COP_CG>(reinterpret_cast<const uint4*>(buf + u)));
            cov_count<COV>(a, 2 * u);
            acc.n += 1;
        }
    }
}

template <int K, int CTA, int DT, bool COV = false>
__global__ void __launch_bounds__(CTA, 1) k_ldg32(const KArgs a) {
    constexpr uint32_t TILE = static_cast<uint32_t>(CTA) * K;
    cta_start(a);
    const Oct* __restrict__ buf = static_cast<const Oct*>(a.buf);
    const uint64_t n32 = a.nvec >> 1;
    const bool half = a.nvec & 1;
    const uint32_t ntiles = static_cast<uint32_t>(a.ntiles);
    const uint32_t total = static_cast<uint32_t>(a.total);
    const bool last_full = !half && n32 == static_cast<uint64_t>(ntiles) * TILE;
    Acc<DT> acc;
    uint32_t full_iters = 0;
    TileCursor c;
    c.start(ntiles);
#pragma unroll 1
    for (; c.it < total; c.next(ntiles)) {
        const uint32_t tile = c.tile(a);
        if (last_full || tile + 1 < ntiles) {
            const Oct* p = buf + static_cast<uint64_t>(tile) * TILE + threadIdx.x;
            Oct v[K];
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = ldg32(p + k * CTA);
            if constexpr (COV) {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    cov_count<COV>(a, 2 * static_cast<uint64_t>((p + k * CTA) - buf));
                    cov_count<COV>(a, 2 * static_cast<uint64_t>((p + k * CTA) - buf) + 1);
                }
            }
#pragma unroll
            for (int k = 0; k < K; ++k) {
                acc.fold(v[k].lo);
                acc.fold(v[k].hi);
            }
            ++full_iters;
        } else {
            ragged32<K, CTA, DT, COV>(a, buf, static_cast<uint64_t>(tile) * TILE, n32, half, acc);
        }
    }
    acc.n += full_iters * K;
    cta_finish<DT>(acc, true, threadIdx.x >> 5, CTA / 32, a);
}

// SL_DYN: chunks of a.tile_vec units claimed from *a.next (the next claim
// prefetched by thread 0; one CTA barrier per chunk).
template <int K, int CTA, int DT, bool COV = false>
__global__ void __launch_bounds__(CTA, 1) k_ldg32_dyn(const KArgs a) {
    constexpr uint32_t TILE = static_cast<uint32_t>(CTA) * K;
    __shared__ uint32_t slot[2];
    cta_start(a);
    const Oct* __restrict__ buf = static_cast<const Oct*>(a.buf);
    const uint64_t n32 = a.nvec >> 1;
    const bool half = a.nvec & 1;
    const uint64_t units = n32 + (half ? 1 : 0);
    const uint32_t chunk = a.tile_vec;
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
        const uint64_t base = static_cast<uint64_t>(cur % nchunks) * chunk;
        const uint64_t left = units - base;
        const uint32_t len = left < chunk ? static_cast<uint32_t>(left) : chunk;
        // whole tiles of whole units only: a chunk holding the half unit ends
        // in the guarded path
        const uint32_t nfull = (base + len <= n32 ? len : len - 1) / TILE;
        const Oct* p = buf + base + threadIdx.x;
#pragma unroll 1
        for (uint32_t t = 0; t < nfull; ++t, p += TILE) {
            Oct v[K];
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = ldg32(p + k * CTA);
            if constexpr (COV) {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    cov_count<COV>(a, 2 * static_cast<uint64_t>((p + k * CTA) - buf));
                    cov_count<COV>(a, 2 * static_cast<uint64_t>((p + k * CTA) - buf) + 1);
                }
            }
#pragma unroll
            for (int k = 0; k < K; ++k) {
                acc.fold(v[k].lo);
                acc.fold(v[k].hi);
            }
        }
        full_iters += nfull;
        if (nfull * TILE < len)
            ragged32<K, CTA, DT, COV>(a, buf, base + static_cast<uint64_t>(nfull) * TILE, n32, half, acc);
        __syncthreads();  // the prefetched claim is visible; the slot read next is not rewritten until j+2
        cur = vslot[(j + 1) & 1];
    }
    acc.n += full_iters * K;
    cta_finish<DT>(acc, true, threadIdx.x >> 5, CTA / 32, a);
}

template <int CTA, int DT, bool DYN>
static const void* ldg32_k(int k) {
#define SL_LDG32_CASE(KK)                                                                              \
    case KK:                                                                                           \
        return DYN ? reinterpret_cast<const void*>(&k_ldg32_dyn<KK, CTA, DT>)                          \
                   : reinterpret_cast<const void*>(&k_ldg32<KK, CTA, DT>);
    switch (k) {
        SL_LDG32_CASE(1)
        SL_LDG32_CASE(2)
        SL_LDG32_CASE(3)
        SL_LDG32_CASE(4)
        SL_LDG32_CASE(6)
        SL_LDG32_CASE(8)
    default: return nullptr;
    }
#undef SL_LDG32_CASE
}

template <int DT, bool DYN>
static const void* ldg32_cta(int k, int cta) {
    switch (cta) {
    case 128: return ldg32_k<128, DT, DYN>(k);
    case 256: return ldg32_k<256, DT, DYN>(k);
    case 512: return ldg32_k<512, DT, DYN>(k);
    default: return nullptr;
    }
}

template <bool DYN>
static const void* ldg32_dt(int dtype, int k, int cta) {
    switch (dtype) {
    case SL_U32: return ldg32_cta<SL_U32, DYN>(k, cta);
    case SL_F32: return ldg32_cta<SL_F32, DYN>(k, cta);
    case SL_BF16: return ldg32_cta<SL_BF16, DYN>(k, cta);
    case SL_FP8_E4M3: return ldg32_cta<SL_FP8_E4M3, DYN>(k, cta);
    default: return nullptr;
    }
}

const void* ldg32_kernel(int dtype, int k, int cta, bool dyn) {
    return dyn ? ldg32_dt<true>(dtype, k, cta) : ldg32_dt<false>(dtype, k, cta);
}

const void* ldg32_cov_kernel(int k, int cta, bool dyn) {
    if (cta != 256) return nullptr;
    switch (k) {
    case 1: return dyn ? reinterpret_cast<const void*>(&k_ldg32_dyn<1, 256, SL_U32, true>)
                       : reinterpret_cast<const void*>(&k_ldg32<1, 256, SL_U32, true>);
    case 3: return dyn ? reinterpret_cast<const void*>(&k_ldg32_dyn<3, 256, SL_U32, true>)
                       : reinterpret_cast<const void*>(&k_ldg32<3, 256, SL_U32, true>);
    case 8: return dyn ? reinterpret_cast<const void*>(&k_ldg32_dyn<8, 256, SL_U32, true>)
                       : reinterpret_cast<const void*>(&k_ldg32<8, 256, SL_U32, true>);
    default: return nullptr;
    }
}

}  // namespace sl
