// k_cpasync_g.cu -- the cp.async kernel with G = 2, 4 or 8 16-byte copies per
// commit group, D groups in flight, D*G <= 16 (the same bytes in flight per
// thread as the one-copy kernel at D*G groups).
#include "k_cpasync.cuh"

namespace sl {

template <int DT>
static const void* cpasync_g_for(int d, int g) {
    if (g == 2) {
        switch (d) {
        case 1: return cpasync_fn<1, 2, DT>();
        case 2: return cpasync_fn<2, 2, DT>();
        case 3: return cpasync_fn<3, 2, DT>();
        case 4: return cpasync_fn<4, 2, DT>();
        case 5: return cpasync_fn<5, 2, DT>();
        case 6: return cpasync_fn<6, 2, DT>();
        case 7: return cpasync_fn<7, 2, DT>();
        case 8: return cpasync_fn<8, 2, DT>();
        default: return nullptr;
        }
    }
    if (g == 4) {
        switch (d) {
        case 1: return cpasync_fn<1, 4, DT>();
        case 2: return cpasync_fn<2, 4, DT>();
        case 3: return cpasync_fn<3, 4, DT>();
        case 4: return cpasync_fn<4, 4, DT>();
        default: return nullptr;
        }
    }
    if (g == 8) {
        switch (d) {
        case 1: return cpasync_fn<1, 8, DT>();
        case 2: return cpasync_fn<2, 8, DT>();
        default: return nullptr;
        }
    }
    return nullptr;
}

const void* cpasync_g_cov_kernel(int d, int g) {
    if (d == 2 && g == 4) return reinterpret_cast<const void*>(&k_cpasync<2, 4, SL_U32, true>);
    if (d == 3 && g == 2) return reinterpret_cast<const void*>(&k_cpasync<3, 2, SL_U32, true>);
    return nullptr;
}

const void* cpasync_g_kernel(int dtype, int d, int g) {
    switch (dtype) {
    case SL_U32: return cpasync_g_for<SL_U32>(d, g);
    case SL_F32: return cpasync_g_for<SL_F32>(d, g);
    case SL_BF16: return cpasync_g_for<SL_BF16>(d, g);
    case SL_FP8_E4M3: return cpasync_g_for<SL_FP8_E4M3>(d, g);
    default: return nullptr;
    }
}

}  // namespace sl
