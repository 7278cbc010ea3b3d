// k_ldg_dyn.cu -- instantiations of the SL_DYN (dynamic contiguous chunk)
// LDG kernel: K in {1,2,3,4,6,8,12,16} x CTA {128,256,512} x every dtype.
#include "k_ldg.cuh"

namespace sl {

template <int CTA, int DT>
static const void* dyn_k(int k) {
    switch (k) {
    case 1: return reinterpret_cast<const void*>(&k_ldg_dyn<1, CTA, DT>);
    case 2: return reinterpret_cast<const void*>(&k_ldg_dyn<2, CTA, DT>);
    case 3: return reinterpret_cast<const void*>(&k_ldg_dyn<3, CTA, DT>);
    case 4: return reinterpret_cast<const void*>(&k_ldg_dyn<4, CTA, DT>);
    case 6: return reinterpret_cast<const void*>(&k_ldg_dyn<6, CTA, DT>);
    case 8: return reinterpret_cast<const void*>(&k_ldg_dyn<8, CTA, DT>);
    case 12: return reinterpret_cast<const void*>(&k_ldg_dyn<12, CTA, DT>);
    case 16: return reinterpret_cast<const void*>(&k_ldg_dyn<16, CTA, DT>);
    default: return nullptr;
    }
}

template <int DT>
static const void* dyn_cta(int k, int cta) {
    switch (cta) {
    case 128: return dyn_k<128, DT>(k);
    case 256: return dyn_k<256, DT>(k);
    case 512: return dyn_k<512, DT>(k);
    default: return nullptr;
    }
}

const void* ldg_dyn_kernel(int dtype, int k, int cta) {
    switch (dtype) {
    case SL_U32: return dyn_cta<SL_U32>(k, cta);
    case SL_F32: return dyn_cta<SL_F32>(k, cta);
    case SL_BF16: return dyn_cta<SL_BF16>(k, cta);
    case SL_FP8_E4M3: return dyn_cta<SL_FP8_E4M3>(k, cta);
    default: return nullptr;
    }
}

}  // namespace sl
