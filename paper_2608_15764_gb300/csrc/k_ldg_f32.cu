// k_ldg_f32.cu -- LDG kernel instantiations for SL_F32 payloads:
// K = 1..16, CTA = 128/256/512, load flavours .cg and .cg.L2::256B.
#include "k_ldg.cuh"

namespace sl {
template <int COP>
static const void* pick_cta(int k, int cta) {
    switch (cta) {
    case 128: return ldg_pick_k<128, SL_F32, COP>(k);
    case 256: return ldg_pick_k<256, SL_F32, COP>(k);
    case 512: return ldg_pick_k<512, SL_F32, COP>(k);
    default: return nullptr;
    }
}

const void* ldg_kernel_f32(int k, int cta, int cop) {
    switch (cop) {
    case SL_COP_CG: return pick_cta<SL_COP_CG>(k, cta);
    case SL_COP_CG_L2_256: return pick_cta<SL_COP_CG_L2_256>(k, cta);
    default: return nullptr;
    }
}
}  // namespace sl
