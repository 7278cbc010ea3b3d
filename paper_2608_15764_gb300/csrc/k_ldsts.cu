// k_ldsts.cu -- the matched plain-load kernel of the cp.async comparison.
//
// Paper §4.3 compares cp.async, which writes shared memory with no
// destination register, against a matched ld.global -> shared-store kernel at
// equal offered concurrency.  Here each thread issues G independent 16-byte
// ld.global into registers (the same tiles and address sequence as LDG at K =
// G and cp.async at D = G), stores them to its own G shared-memory slots with
// st.shared, then reads each slot back with ld.shared and folds it -- the same
// shared-memory round trip cp.async makes, but with the data passing through
// registers and an explicit store.  Like the LDG kernel it must hold its G
// loaded vectors in registers (launch bounds allow it up to G = 16 at 256
// threads; the host rejects shapes whose register count is too small).
#include "sl_device.cuh"

namespace sl {

__device__ __forceinline__ void sts16(uint32_t saddr, const uint4& v) {
    asm volatile("st.shared.v4.u32 [%0], {%1,%2,%3,%4};" ::"r"(saddr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}

template <int G, int DT, bool COV = false>
__global__ void __launch_bounds__(G <= 8 ? 1024 : 256, 1) k_ldsts(const KArgs a) {
    extern __shared__ __align__(128) uint4 st_ring[];  // [G][cta]; 128-byte aligned (+ SL_DEBUG_SMEM_SKEW)
    cta_start(a);
    const uint32_t cta = blockDim.x;
    const uint4* __restrict__ buf = static_cast<const uint4*>(a.buf);
    const uint32_t ntiles = static_cast<uint32_t>(a.ntiles);
    const uint32_t total = static_cast<uint32_t>(a.total);
    const uint64_t tile_vec = static_cast<uint64_t>(cta) * G;
    const uint32_t skew = (static_cast<uint32_t>(a.debug) >> SL_DEBUG_SMEM_SKEW_SHIFT) & 7u;
    const uint32_t my0 = smem_addr(st_ring + skew + threadIdx.x), stride = cta * 16u;
    Acc<DT> acc;
    uint32_t full_iters = 0;
    TileCursor c;
    c.start(ntiles);
#pragma unroll 1
    for (; c.it < total; c.next(ntiles)) {
        const uint64_t base = static_cast<uint64_t>(c.tile(a)) * tile_vec;
        const uint4* p = buf + base + threadIdx.x;
        uint4 v[G];
        if (base + tile_vec <= a.nvec) {
#pragma unroll
            for (int g = 0; g < G; ++g) v[g] = ldg16<SL_COP_CG>(p + static_cast<size_t>(g) * cta);
            if constexpr (COV) {
#pragma unroll
                for (int g = 0; g < G; ++g) cov_count<COV>(a, (p + static_cast<size_t>(g) * cta) - buf);
            }
#pragma unroll
            for (int g = 0; g < G; ++g) sts16(my0 + g * stride, v[g]);
#pragma unroll
            for (int g = 0; g < G; ++g) acc.fold(lds16(my0 + g * stride));
            ++full_iters;
        } else {
            // ragged last tile: one vector at a time (keeps register pressure
            // of this rare path below the main path's)
            const uint64_t rem = a.nvec - base;
#pragma unroll 1
            for (int g = 0; g < G; ++g) {
                if (threadIdx.x + static_cast<uint64_t>(g) * cta < rem) {
                    sts16(my0 + g * stride, ldg16<SL_COP_CG>(p + static_cast<size_t>(g) * cta));
                    cov_count<COV>(a, (p + static_cast<size_t>(g) * cta) - buf);
                    acc.fold(lds16(my0 + g * stride));
                    acc.n += 1;
                }
            }
        }
    }
    acc.n += full_iters * G;
    cta_finish<DT>(acc, true, threadIdx.x >> 5, cta >> 5, a);
}

template <int DT>
static const void* ldsts_for(int g) {
    switch (g) {
    case 1: return reinterpret_cast<const void*>(&k_ldsts<1, DT>);
    case 2: return reinterpret_cast<const void*>(&k_ldsts<2, DT>);
    case 3: return reinterpret_cast<const void*>(&k_ldsts<3, DT>);
    case 4: return reinterpret_cast<const void*>(&k_ldsts<4, DT>);
    case 5: return reinterpret_cast<const void*>(&k_ldsts<5, DT>);
    case 6: return reinterpret_cast<const void*>(&k_ldsts<6, DT>);
    case 7: return reinterpret_cast<const void*>(&k_ldsts<7, DT>);
    case 8: return reinterpret_cast<const void*>(&k_ldsts<8, DT>);
    case 9: return reinterpret_cast<const void*>(&k_ldsts<9, DT>);
    case 10: return reinterpret_cast<const void*>(&k_ldsts<10, DT>);
    case 11: return reinterpret_cast<const void*>(&k_ldsts<11, DT>);
    case 12: return reinterpret_cast<const void*>(&k_ldsts<12, DT>);
    case 13: return reinterpret_cast<const void*>(&k_ldsts<13, DT>);
    case 14: return reinterpret_cast<const void*>(&k_ldsts<14, DT>);
    case 15: return reinterpret_cast<const void*>(&k_ldsts<15, DT>);
    case 16: return reinterpret_cast<const void*>(&k_ldsts<16, DT>);
    default: return nullptr;
    }
}

const void* ldsts_cov_kernel(int g) {
    if (g == 1) return reinterpret_cast<const void*>(&k_ldsts<1, SL_U32, true>);
    if (g == 16) return reinterpret_cast<const void*>(&k_ldsts<16, SL_U32, true>);
    return nullptr;
}

const void* ldsts_kernel(int dtype, int g) {
    switch (dtype) {
    case SL_U32: return ldsts_for<SL_U32>(g);
    case SL_F32: return ldsts_for<SL_F32>(g);
    case SL_BF16: return ldsts_for<SL_BF16>(g);
    case SL_FP8_E4M3: return ldsts_for<SL_FP8_E4M3>(g);
    default: return nullptr;
    }
}

}  // namespace sl
