// k_two.cu -- two co-resident plain-load streams in one CTA (paper §4.4).
//
// One CTA per SM holds A + B warps.  Warps [0, A) are stream A and warps
// [A, A+B) stream B; each stream runs the LDG kernel's loop on its own buffer
// with its own threads: tile = (stream threads)*K vectors, CTA b walks tiles
// b, b+grid, ... over the stream's passes, load k of stream thread t reads
// vector tile*T*K + k*T + t (T = stream threads), every warp instruction 512
// contiguous bytes, guarded ragged tail.  Both streams do fixed work, so each
// stream's checksum has a plain definition.
//
// Lane 0 of every warp stamps %globaltimer when the warp starts and when it
// has folded its last load: per stream the earliest start and the latest end
// (atomicMin / atomicMax), and for stream B also the earliest end.  Stream A's
// bandwidth is its bytes over its window; the host sizes B's work so that
// B's first warp to finish ends after A's last (B loads throughout A's run),
// and reports whether that held.  Each warp writes one partial; a one-CTA
// combine reduces them per stream.
#include "sl_device.cuh"

namespace sl {

template <int K>
__global__ void __launch_bounds__(1024, 1) k_two(const TwoArgs t) {
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool sb = warp >= t.warps_a;  // stream B?
    const uint32_t nthr = sb ? blockDim.x - t.warps_a * 32u : t.warps_a * 32u;
    const uint32_t lt = sb ? threadIdx.x - t.warps_a * 32u : threadIdx.x;
    const uint4* __restrict__ buf = sb ? t.buf_b : t.buf_a;
    const uint64_t nvec = sb ? t.nvec_b : t.nvec_a;
    const uint32_t ntiles = sb ? t.ntiles_b : t.ntiles_a;
    const uint32_t total = sb ? t.total_b : t.total_a;
    const uint64_t tile_vec = static_cast<uint64_t>(nthr) * K;
    const int si = sb ? 1 : 0;
    if (lane == 0) atomicMin(reinterpret_cast<unsigned long long*>(t.ctl + TWO_START + si), gtimer());
    Acc<SL_U32> acc;
    uint32_t full_iters = 0;
    uint32_t it = blockIdx.x, tile = blockIdx.x % max(ntiles, 1u);
#pragma unroll 1
    for (; it < total; it += gridDim.x) {
        const uint64_t base = static_cast<uint64_t>(tile) * tile_vec;
        const uint4* p = buf + base + lt;
        uint4 v[K];
        if (base + tile_vec <= nvec) {
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = ldg16<SL_COP_CG>(p + k * nthr);
#pragma unroll
            for (int k = 0; k < K; ++k) acc.fold(v[k]);
            ++full_iters;
        } else {
            const uint32_t rem = static_cast<uint32_t>(nvec - base);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if (lt + k * nthr < rem) v[k] = ldg16<SL_COP_CG>(p + k * nthr);
                else v[k] = make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if (lt + k * nthr < rem) {
                    acc.fold(v[k]);
                    acc.n += 1;
                }
            }
        }
        tile += gridDim.x;
        while (tile >= ntiles) tile -= ntiles;
    }
    acc.n += full_iters * K;
    uint32_t s = acc.s;
    uint64_t x = (static_cast<uint64_t>(acc.xh) << 32) | acc.xl, n = acc.n;
    float hi = 0.0f, lo = 0.0f;
    warp_merge<SL_U32>(s, x, n, hi, lo);
    if (lane == 0) {
        const unsigned long long now = gtimer();
        atomicMax(reinterpret_cast<unsigned long long*>(t.ctl + TWO_END + si), now);
        if (sb) atomicMin(reinterpret_cast<unsigned long long*>(t.ctl + TWO_FIRST_END_B), now);
        WarpPartial w;
        w.sum = s;
        w.pad = 0;
        w.xr = x;
        w.issued = n;
        w.hi = 0.0f;
        w.lo = 0.0f;
        t.parts[static_cast<size_t>(blockIdx.x) * 32 + warp] = w;
    }
}

// One CTA of 64 threads: warp s reduces stream s's warp partials (CTA-major,
// exact integer sums and XOR), lane 0 writes {sum, xor, issued} of the stream
// to out[3s..3s+2]; out[6..10] take the five timer words.
__global__ void __launch_bounds__(64) k_two_combine(const TwoArgs t, uint32_t grid, uint64_t* out) {
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t w0 = warp ? t.warps_a : 0u;
    const uint32_t nw = warp ? t.warps_b : t.warps_a;
    uint32_t s = 0;
    uint64_t x = 0, n = 0;
    const uint64_t count = static_cast<uint64_t>(grid) * nw;
    for (uint64_t i = lane; i < count; i += 32) {
        const WarpPartial p = t.parts[(i / nw) * 32 + w0 + i % nw];
        s += p.sum;
        x ^= p.xr;
        n += p.issued;
    }
    float hi = 0.0f, lo = 0.0f;
    warp_merge<SL_U32>(s, x, n, hi, lo);
    if (lane == 0) {
        out[3 * warp + 0] = s;
        out[3 * warp + 1] = x;
        out[3 * warp + 2] = n;
    }
    if (threadIdx.x < TWO_CTL_WORDS) out[6 + threadIdx.x] = t.ctl[threadIdx.x];
}

cudaError_t launch_two(const TwoArgs& t, int k, uint32_t grid, cudaStream_t s) {
    const unsigned block = (t.warps_a + t.warps_b) * 32u;
    switch (k) {
    case 1: k_two<1><<<grid, block, 0, s>>>(t); break;
    case 2: k_two<2><<<grid, block, 0, s>>>(t); break;
    case 4: k_two<4><<<grid, block, 0, s>>>(t); break;
    case 8: k_two<8><<<grid, block, 0, s>>>(t); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_two_combine(const TwoArgs& t, uint32_t grid, uint64_t* out, cudaStream_t s) {
    k_two_combine<<<1, 64, 0, s>>>(t, grid, out);
    return cudaGetLastError();
}

const void* two_kernel(int k) {
    switch (k) {
    case 1: return reinterpret_cast<const void*>(&k_two<1>);
    case 2: return reinterpret_cast<const void*>(&k_two<2>);
    case 4: return reinterpret_cast<const void*>(&k_two<4>);
    case 8: return reinterpret_cast<const void*>(&k_two<8>);
    default: return nullptr;
    }
}

}  // namespace sl
