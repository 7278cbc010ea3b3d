// k_batch_ldg.cu -- LDG class-kernel instantiations of the batched form:
// K in {1,2,3,4,6,8,12,16} x CTA {128,256,512} x every dtype.
#include "k_batch.cuh"

namespace sl {

template <int CTA, int DT>
static const void* kb_ldg_k(int k) {
    switch (k) {
    case 1: return reinterpret_cast<const void*>(&kb_ldg<1, CTA, DT>);
    case 2: return reinterpret_cast<const void*>(&kb_ldg<2, CTA, DT>);
    case 3: return reinterpret_cast<const void*>(&kb_ldg<3, CTA, DT>);
    case 4: return reinterpret_cast<const void*>(&kb_ldg<4, CTA, DT>);
    case 6: return reinterpret_cast<const void*>(&kb_ldg<6, CTA, DT>);
    case 8: return reinterpret_cast<const void*>(&kb_ldg<8, CTA, DT>);
    case 12: return reinterpret_cast<const void*>(&kb_ldg<12, CTA, DT>);
    case 16: return reinterpret_cast<const void*>(&kb_ldg<16, CTA, DT>);
    default: return nullptr;
    }
}

template <int DT>
static const void* kb_ldg_cta(int k, int cta) {
    switch (cta) {
    case 128: return kb_ldg_k<128, DT>(k);
    case 256: return kb_ldg_k<256, DT>(k);
    case 512: return kb_ldg_k<512, DT>(k);
    default: return nullptr;
    }
}

const void* batch_ldg_kernel(int dtype, int k, int cta) {
    switch (dtype) {
    case SL_U32: return kb_ldg_cta<SL_U32>(k, cta);
    case SL_F32: return kb_ldg_cta<SL_F32>(k, cta);
    case SL_BF16: return kb_ldg_cta<SL_BF16>(k, cta);
    case SL_FP8_E4M3: return kb_ldg_cta<SL_FP8_E4M3>(k, cta);
    default: return nullptr;
    }
}

}  // namespace sl
