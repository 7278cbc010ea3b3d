// k_cov.cu -- coverage instantiations of the LDG kernels (grid-stride and
// SL_DYN): the same kernels with every 16-byte load also counted in
// KArgs::cov (uint32 payloads; the shapes below).
#include "k_ldg.cuh"

namespace sl {

template <int CTA>
static const void* cov_ldg(int k, bool dyn) {
    switch (k) {
    case 1: return dyn ? nullptr : reinterpret_cast<const void*>(&k_ldg<1, CTA, SL_U32, SL_COP_CG, true>);
    case 2: return dyn ? reinterpret_cast<const void*>(&k_ldg_dyn<2, CTA, SL_U32, true>) : nullptr;
    case 3: return dyn ? nullptr : reinterpret_cast<const void*>(&k_ldg<3, CTA, SL_U32, SL_COP_CG, true>);
    case 8: return dyn ? nullptr : reinterpret_cast<const void*>(&k_ldg<8, CTA, SL_U32, SL_COP_CG, true>);
    case 12: return dyn ? reinterpret_cast<const void*>(&k_ldg_dyn<12, CTA, SL_U32, true>) : nullptr;
    case 16: return dyn ? nullptr : reinterpret_cast<const void*>(&k_ldg<16, CTA, SL_U32, SL_COP_CG, true>);
    default: return nullptr;
    }
}

const void* ldg_cov_kernel(int k, int cta, bool dyn) {
    switch (cta) {
    case 128: return cov_ldg<128>(k, dyn);
    case 256: return cov_ldg<256>(k, dyn);
    case 512: return cov_ldg<512>(k, dyn);
    default: return nullptr;
    }
}

}  // namespace sl
