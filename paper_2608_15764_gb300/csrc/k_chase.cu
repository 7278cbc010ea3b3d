// k_chase.cu -- the pointer-chase latency probe (paper §4.1 "Primitive
// baseline": unloaded latency on a single SM from a dependent pointer chain,
// .ca and .cg).
//
// One thread follows the chain: idx = chain[idx].  Each load's address depends
// on the previous load's value, so exactly one load is in flight.  A first
// (untimed) traversal of `warm` steps brings the chain into whatever cache
// level holds it; then `hops` steps are timed with clock64 (SM cycles) and
// %globaltimer (ns).  The final index goes out so the chase cannot be
// eliminated and so the host can check it against the oracle.
#include "sl_device.cuh"

namespace sl {

template <int CA>
__device__ __forceinline__ uint32_t chase_ld(const uint32_t* p) {
    uint32_t v;
    if constexpr (CA)
        asm volatile("ld.global.ca.u32 %0, [%1];" : "=r"(v) : "l"(p));
    else
        asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// out[0] = final index, out[1] = ns, out[2] = cycles of the timed hops;
// out[3] = 1 if an index left the chain (the chase stops there).
template <int CA>
__global__ void __launch_bounds__(32) k_chase(const uint32_t* __restrict__ chain, uint64_t nwords, uint32_t start,
                                              uint64_t warm, uint64_t hops, uint64_t* out) {
    if (threadIdx.x != 0) return;
    uint32_t idx = start;
    uint64_t bad = 0;
    for (uint64_t h = 0; h < warm && !bad; ++h) {
        if (idx >= nwords) { bad = 1; break; }
        idx = chase_ld<CA>(chain + idx);
    }
    const uint64_t t0 = gtimer();
    const long long c0 = clock64();
    for (uint64_t h = 0; h < hops && !bad; ++h) {
        if (idx >= nwords) { bad = 1; break; }
        idx = chase_ld<CA>(chain + idx);
    }
    const long long c1 = clock64();
    const uint64_t t1 = gtimer();
    out[0] = idx;
    out[1] = t1 - t0;
    out[2] = static_cast<uint64_t>(c1 - c0);
    out[3] = bad;
}

cudaError_t launch_chase(const uint32_t* chain, uint64_t nwords, uint32_t start, uint64_t warm, uint64_t hops,
                         int ca, uint64_t* out, cudaStream_t s) {
    if (ca)
        k_chase<1><<<1, 32, 0, s>>>(chain, nwords, start, warm, hops, out);
    else
        k_chase<0><<<1, 32, 0, s>>>(chain, nwords, start, warm, hops, out);
    return cudaGetLastError();
}

}  // namespace sl
