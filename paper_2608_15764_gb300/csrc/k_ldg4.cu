// k_ldg4.cu -- the 4-byte-width plain-load kernel (SL_LDG4).
//
// Paper §4.1 "Primitive baseline" qualifies the machine with a streaming
// read at 4-byte width and one load in flight per thread (the "K1" row that
// gates the rest of the suite).  This kernel is that row and its K sweep: K
// independent ld.global.cg.u32 per thread per iteration, issued before any is
// consumed, so one warp instruction reads 128 contiguous bytes.
//
// Tile = CTA*K words.  CTA b walks tiles b, b+grid, ... over all passes (tile
// index mod the tiles per pass; reversed for SL_DESC); load k of thread t reads
// word tile*CTA*K + k*CTA + t.  Because CTA is a multiple of 32, the parity of
// that word index is the parity of t: even threads only ever read the low
// halves of the little-endian 64-bit words and odd threads the high halves,
// so a thread's XOR goes to xl (even t) or xh (odd t) and the CTA merge yields
// the same 64-bit XOR as the 16-byte kernels.  issued_loads counts 4-byte
// loads here: passes * bytes / 4.
#include "sl_device.cuh"

namespace sl {

__device__ __forceinline__ uint32_t ldg4(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

template <int K, int CTA>
__global__ void __launch_bounds__(CTA, 1) k_ldg4(const KArgs a) {
    constexpr uint32_t TILE = static_cast<uint32_t>(CTA) * K;
    cta_start(a);
    const uint32_t* __restrict__ buf = static_cast<const uint32_t*>(a.buf);
    const uint32_t ntiles = static_cast<uint32_t>(a.ntiles);
    const uint32_t total = static_cast<uint32_t>(a.total);
    const bool last_full = (a.nvec == static_cast<uint64_t>(ntiles) * TILE);  // nvec counts words here
    uint32_t s = 0, xr = 0, full_iters = 0, n = 0;
    TileCursor c;
    c.start(ntiles);
#pragma unroll 1
    for (; c.it < total; c.next(ntiles)) {
        const uint32_t tile = c.tile(a);
        const uint32_t* p = buf + static_cast<uint64_t>(tile) * TILE + threadIdx.x;
        uint32_t v[K];
        if (last_full || tile + 1 < ntiles) {
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = ldg4(p + k * CTA);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                s += v[k];
                xr ^= v[k];
            }
            ++full_iters;
        } else {
            const uint32_t rem = static_cast<uint32_t>(a.nvec - static_cast<uint64_t>(tile) * TILE);
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = threadIdx.x + k * CTA < rem ? ldg4(p + k * CTA) : 0u;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if (threadIdx.x + k * CTA < rem) {
                    s += v[k];
                    xr ^= v[k];
                    n += 1;
                }
            }
        }
    }
    Acc<SL_U32> acc;
    acc.s = s;
    acc.xl = (threadIdx.x & 1) ? 0u : xr;
    acc.xh = (threadIdx.x & 1) ? xr : 0u;
    acc.n = n + full_iters * K;
    cta_finish<SL_U32>(acc, true, threadIdx.x >> 5, CTA / 32, a);
}

template <int CTA>
static const void* ldg4_pick_k(int k) {
    switch (k) {
    case 1: return reinterpret_cast<const void*>(&k_ldg4<1, CTA>);
    case 2: return reinterpret_cast<const void*>(&k_ldg4<2, CTA>);
    case 4: return reinterpret_cast<const void*>(&k_ldg4<4, CTA>);
    case 8: return reinterpret_cast<const void*>(&k_ldg4<8, CTA>);
    case 16: return reinterpret_cast<const void*>(&k_ldg4<16, CTA>);
    default: return nullptr;
    }
}

const void* ldg4_kernel(int dtype, int k, int cta) {
    if (dtype != SL_U32) return nullptr;
    switch (cta) {
    case 128: return ldg4_pick_k<128>(k);
    case 256: return ldg4_pick_k<256>(k);
    case 512: return ldg4_pick_k<512>(k);
    case 1024: return ldg4_pick_k<1024>(k);
    default: return nullptr;
    }
}

}  // namespace sl
