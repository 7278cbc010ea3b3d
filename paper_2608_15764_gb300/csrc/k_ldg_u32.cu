// k_ldg_u32.cu -- LDG kernel instantiations for uint32 payloads:
// K = 1..16, CTA = 32/128/256/512/1024, all three load flavours.
#include "k_ldg.cuh"

namespace sl {
template <int DT, int COP>
static const void* pick_cta(int k, int cta) {
    switch (cta) {
    case 32: return ldg_pick_k<32, DT, COP>(k);
    case 128: return ldg_pick_k<128, DT, COP>(k);
    case 256: return ldg_pick_k<256, DT, COP>(k);
    case 512: return ldg_pick_k<512, DT, COP>(k);
    case 1024: return ldg_pick_k<1024, DT, COP>(k);
    default: return nullptr;
    }
}

const void* ldg_kernel_u32(int k, int cta, int cop) {
    switch (cop) {
    case SL_COP_CG: return pick_cta<SL_U32, SL_COP_CG>(k, cta);
    case SL_COP_CG_L2_256: return pick_cta<SL_U32, SL_COP_CG_L2_256>(k, cta);
    case SL_COP_NC_NA_L2_256: return pick_cta<SL_U32, SL_COP_NC_NA_L2_256>(k, cta);
    default: return nullptr;
    }
}
}  // namespace sl
