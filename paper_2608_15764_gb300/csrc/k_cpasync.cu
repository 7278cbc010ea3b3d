// k_cpasync.cu -- the cp.async kernel with one 16-byte copy per commit group
// (the paper's cell, D = 1..16 groups in flight) and the lookup of every
// cp.async instantiation; several copies per group are in k_cpasync_g.cu.
#include "k_cpasync.cuh"

namespace sl {

const void* cpasync_g_kernel(int dtype, int d, int g);
const void* cpasync_g_cov_kernel(int d, int g);

template <int DT>
static const void* cpasync_for(int d) {
    switch (d) {
    case 1: return cpasync_fn<1, 1, DT>();
    case 2: return cpasync_fn<2, 1, DT>();
    case 3: return cpasync_fn<3, 1, DT>();
    case 4: return cpasync_fn<4, 1, DT>();
    case 5: return cpasync_fn<5, 1, DT>();
    case 6: return cpasync_fn<6, 1, DT>();
    case 7: return cpasync_fn<7, 1, DT>();
    case 8: return cpasync_fn<8, 1, DT>();
    case 9: return cpasync_fn<9, 1, DT>();
    case 10: return cpasync_fn<10, 1, DT>();
    case 11: return cpasync_fn<11, 1, DT>();
    case 12: return cpasync_fn<12, 1, DT>();
    case 13: return cpasync_fn<13, 1, DT>();
    case 14: return cpasync_fn<14, 1, DT>();
    case 15: return cpasync_fn<15, 1, DT>();
    case 16: return cpasync_fn<16, 1, DT>();
    default: return nullptr;
    }
}

const void* cpasync_cov_kernel(int d, int g) {
    if (g != 1) return cpasync_g_cov_kernel(d, g);
    if (d == 1) return reinterpret_cast<const void*>(&k_cpasync<1, 1, SL_U32, true>);
    if (d == 4) return reinterpret_cast<const void*>(&k_cpasync<4, 1, SL_U32, true>);
    if (d == 16) return reinterpret_cast<const void*>(&k_cpasync<16, 1, SL_U32, true>);
    return nullptr;
}

const void* cpasync_kernel(int dtype, int d, int g) {
    if (g != 1) return cpasync_g_kernel(dtype, d, g);
    switch (dtype) {
    case SL_U32: return cpasync_for<SL_U32>(d);
    case SL_F32: return cpasync_for<SL_F32>(d);
    case SL_BF16: return cpasync_for<SL_BF16>(d);
    case SL_FP8_E4M3: return cpasync_for<SL_FP8_E4M3>(d);
    default: return nullptr;
    }
}

}  // namespace sl
