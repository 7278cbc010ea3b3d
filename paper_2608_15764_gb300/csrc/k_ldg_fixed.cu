// k_ldg_fixed.cu -- the LDG kernel under the paper's fixed-iteration control.
//
// Paper §3 "Fixed-work control": every thread runs iters = L / (threads*K)
// iterations (integer division) of K loads, so the issued count is
// iters*threads*K, within a small rounding mismatch of the target L across
// the K sweep (the paper reports the largest, §4.2).  The paper's allocation
// sweep holds the issued volume while the allocation shrinks, so the reads
// wrap around the buffer.
//
// Here the launch covers global tiles g = 0 .. iters*grid-1 (CTA b takes
// g = b, b+grid, ... ascending, or the mirror image for SL_DESC); tile g
// covers the vectors g*CTA*K + k*CTA + t (k < K, t < CTA) taken modulo the
// buffer's vector count.  So the multiset of vectors read is exactly
// { j mod nvec : 0 <= j < iters*grid*CTA*K }.  Each CTA tracks its tile's
// start modulo nvec incrementally (the host guarantees nvec >= one tile, so
// a single subtraction wraps any index of a tile).
#include "sl_device.cuh"

namespace sl {

template <int K, int CTA, bool COV = false>
__global__ void __launch_bounds__(CTA, 1) k_ldg_fixed(const KArgs a) {
    constexpr uint32_t TILE = static_cast<uint32_t>(CTA) * K;
    cta_start(a);
    const uint4* __restrict__ buf = static_cast<const uint4*>(a.buf);
    const uint64_t nvec = a.nvec;
    const uint32_t total = static_cast<uint32_t>(a.total);  // iters * grid tiles
    const uint64_t step = (static_cast<uint64_t>(gridDim.x) * TILE) % nvec;
    Acc<SL_U32> acc;
    uint32_t iters = 0;
    uint32_t it = blockIdx.x;
    if (it < total) {
        const uint64_t g = a.desc ? static_cast<uint64_t>(total - 1 - it) : it;
        uint64_t base = (g * TILE) % nvec;
#pragma unroll 1
        for (; it < total; it += gridDim.x) {
            uint4 v[K];
            if (base + TILE <= nvec) {
                const uint4* p = buf + base + threadIdx.x;
#pragma unroll
                for (int k = 0; k < K; ++k) v[k] = ldg16<SL_COP_CG>(p + k * CTA);
                if constexpr (COV) {
#pragma unroll
                    for (int k = 0; k < K; ++k) cov_count<COV>(a, (p + k * CTA) - buf);
                }
            } else {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    uint64_t j = base + static_cast<uint64_t>(k) * CTA + threadIdx.x;
                    if (j >= nvec) j -= nvec;
                    v[k] = ldg16<SL_COP_CG>(buf + j);
                    cov_count<COV>(a, j);
                }
            }
#pragma unroll
            for (int k = 0; k < K; ++k) acc.fold(v[k]);
            ++iters;
            if (a.desc)
                base = base >= step ? base - step : base + nvec - step;
            else
                base = base + step >= nvec ? base + step - nvec : base + step;
        }
    }
    acc.n = iters * K;
    cta_finish<SL_U32>(acc, true, threadIdx.x >> 5, CTA / 32, a);
}

template <int CTA>
static const void* fixed_k(int k) {
    switch (k) {
    case 1: return reinterpret_cast<const void*>(&k_ldg_fixed<1, CTA>);
    case 2: return reinterpret_cast<const void*>(&k_ldg_fixed<2, CTA>);
    case 3: return reinterpret_cast<const void*>(&k_ldg_fixed<3, CTA>);
    case 4: return reinterpret_cast<const void*>(&k_ldg_fixed<4, CTA>);
    case 6: return reinterpret_cast<const void*>(&k_ldg_fixed<6, CTA>);
    case 8: return reinterpret_cast<const void*>(&k_ldg_fixed<8, CTA>);
    case 12: return reinterpret_cast<const void*>(&k_ldg_fixed<12, CTA>);
    case 16: return reinterpret_cast<const void*>(&k_ldg_fixed<16, CTA>);
    default: return nullptr;
    }
}

const void* ldg_fixed_cov_kernel(int k, int cta) {
    if (k == 2 && cta == 256) return reinterpret_cast<const void*>(&k_ldg_fixed<2, 256, true>);
    if (k == 8 && cta == 256) return reinterpret_cast<const void*>(&k_ldg_fixed<8, 256, true>);
    if (k == 2 && cta == 1024) return reinterpret_cast<const void*>(&k_ldg_fixed<2, 1024, true>);
    if (k == 8 && cta == 1024) return reinterpret_cast<const void*>(&k_ldg_fixed<8, 1024, true>);
    return nullptr;
}

const void* ldg_fixed_kernel(int dtype, int k, int cta) {
    if (dtype != SL_U32) return nullptr;
    switch (cta) {
    case 256: return fixed_k<256>(k);
    case 512: return fixed_k<512>(k);
    case 1024: return fixed_k<1024>(k);
    default: return nullptr;
    }
}

}  // namespace sl
