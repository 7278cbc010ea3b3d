// k_util.cu -- fill, L2 flush and final combine kernels.
#include "sl_device.cuh"

namespace sl {

// splitmix64 output m of the stream seeded with `seed` (Steele, Lea and
// Flood 2014): the state after m+1 golden-ratio increments, finalised by the
// (30, 27, 31) xor-shift / multiply mix.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t m) {
    uint64_t z = seed + (m + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Vector j (16 bytes) holds outputs 2j (words 4j, 4j+1) and 2j+1 (words
// 4j+2, 4j+3), low half first.
__global__ void __launch_bounds__(256) k_fill_splitmix64(uint4* __restrict__ buf, uint64_t nvec,
                                                         uint64_t seed) {
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t j = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < nvec; j += stride) {
        const uint64_t a = splitmix64_at(seed, 2 * j);
        const uint64_t b = splitmix64_at(seed, 2 * j + 1);
        uint4 v;
        v.x = static_cast<uint32_t>(a);
        v.y = static_cast<uint32_t>(a >> 32);
        v.z = static_cast<uint32_t>(b);
        v.w = static_cast<uint32_t>(b >> 32);
        buf[j] = v;
    }
}

// Overwrite the flush buffer: its lines displace whatever was L2-resident.
__global__ void __launch_bounds__(256) k_flush(uint4* __restrict__ buf, uint64_t nvec) {
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    const uint32_t tag = blockIdx.x;
    for (uint64_t j = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < nvec; j += stride)
        buf[j] = make_uint4(tag, static_cast<uint32_t>(j), 0u, 0u);
}

// Final combine of per-CTA partials into one sl_result, as a separate
// launch (used when the load kernels do not combine in their last CTA: the
// multi-chunk host-buffer path, and empty buffers).  One CTA of
// COMBINE_THREADS threads; thread i folds partials i, i+T, ... in index order,
// then a fixed shared-memory tree merges the threads, so the FP64 float sum
// has a fixed order.  Integer parts combine exactly.  The device error word is
// reported in status and cleared; the timing window is read and reset.
constexpr int COMBINE_THREADS = 512;

__global__ void __launch_bounds__(COMBINE_THREADS) k_combine(const WarpPartial* __restrict__ parts,
                                                            uint64_t nparts, uint64_t* window,
                                                            uint32_t* err, sl_result* out) {
    __shared__ uint32_t s_sum[COMBINE_THREADS];
    __shared__ uint64_t s_xor[COMBINE_THREADS], s_n[COMBINE_THREADS];
    __shared__ double s_f[COMBINE_THREADS];
    const int t = threadIdx.x;
    uint32_t sum = 0;
    uint64_t xr = 0, n = 0;
    double f = 0.0;
    for (uint64_t i = t; i < nparts; i += COMBINE_THREADS) {
        const WarpPartial p = parts[i];
        sum += p.sum;
        xr ^= p.xr;
        n += p.issued;
        f += static_cast<double>(p.hi) + static_cast<double>(p.lo);
    }
    s_sum[t] = sum;
    s_xor[t] = xr;
    s_n[t] = n;
    s_f[t] = f;
    __syncthreads();
    for (int w = COMBINE_THREADS / 2; w > 0; w >>= 1) {
        if (t < w) {
            s_sum[t] += s_sum[t + w];
            s_xor[t] ^= s_xor[t + w];
            s_n[t] += s_n[t + w];
            s_f[t] += s_f[t + w];
        }
        __syncthreads();
    }
    if (t == 0) {
        const uint64_t t0 = window[0], t1 = window[1];
        sl_result r;
        r.xor_u64 = s_xor[0];
        r.issued_loads = s_n[0];
        r.device_ns = 0;
        r.window_ns = (nparts > 0 && t1 > t0) ? t1 - t0 : 0;
        r.fsum = s_f[0];
        r.fsum_hi = static_cast<float>(s_f[0]);
        r.fsum_lo = static_cast<float>(s_f[0] - static_cast<double>(r.fsum_hi));
        r.sum_u32 = s_sum[0];
        const uint32_t e = *err;
        r.status = e ? SL_ERR_TIMEOUT : SL_OK;
        r.grid = 0;
        r.cta = 0;
        r.resident_per_sm = 0;
        r.smem_bytes = 0;
        *out = r;
        *err = 0;
        window[0] = ~0ull;
        window[1] = 0;
    }
}

cudaError_t launch_fill_splitmix64(void* buf, uint64_t nvec, uint64_t seed, int sms, cudaStream_t s) {
    if (nvec == 0) return cudaSuccess;
    uint64_t blocks = (nvec + 255) / 256;
    const uint64_t cap = static_cast<uint64_t>(sms) * 16;
    if (blocks > cap) blocks = cap;
    k_fill_splitmix64<<<static_cast<unsigned>(blocks), 256, 0, s>>>(static_cast<uint4*>(buf), nvec, seed);
    return cudaGetLastError();
}

cudaError_t launch_flush(void* buf, uint64_t nvec, int sms, cudaStream_t s) {
    if (nvec == 0) return cudaSuccess;
    uint64_t blocks = (nvec + 255) / 256;
    const uint64_t cap = static_cast<uint64_t>(sms) * 16;
    if (blocks > cap) blocks = cap;
    k_flush<<<static_cast<unsigned>(blocks), 256, 0, s>>>(static_cast<uint4*>(buf), nvec);
    return cudaGetLastError();
}

cudaError_t launch_combine(const WarpPartial* parts, uint64_t nparts, uint64_t* window, uint32_t* err,
                           sl_result* out, cudaStream_t s) {
    k_combine<<<1, COMBINE_THREADS, 0, s>>>(parts, nparts, window, err, out);
    return cudaGetLastError();
}

}  // namespace sl
