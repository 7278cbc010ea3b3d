// k_cpasync_dyn.cu -- the cp.async kernel under the SL_DYN traversal.
//
// The copies, commit groups and slot ring are those of k_cpasync (D groups of
// G 16-byte copies per thread in flight, a thread reading back only its own
// slots), but the CTAs claim contiguous chunks of a.tile_vec vectors (a
// multiple of the tile cta*D*G, about 1 MiB) from the counter *a.next, as the
// dynamic-chunk LDG kernel does, and walk a chunk's tiles in order.  The
// group refills that run ahead of the fold cross from the last tile of a
// chunk into the first tile of the next one, so a CTA holds two claims: the
// chunk it reads and the one after it.  Thread 0 claims a third at the start
// of each chunk; a CTA barrier at the end of the chunk publishes it (three
// shared slots, each rewritten only after every thread has passed the barrier
// that follows its last read).  Integer results are exact; float sums meet the
// same bound as every traversal but are not bit-reproducible between runs.
#include "k_cpasync.cuh"

namespace sl {

template <int D, int G, int DT, bool COV = false>
__global__ void __launch_bounds__(D * G > 8 ? 512 : 1024) k_cpasync_dyn(const KArgs a) {
    extern __shared__ __align__(128) uint4 ring[];
    __shared__ uint32_t slot[3];
    cta_start(a);
    const uint32_t cta = blockDim.x;
    const uint4* __restrict__ buf = static_cast<const uint4*>(a.buf);
    const uint32_t tile = cta * (D * G);
    const uint32_t chunk_vec = a.tile_vec;  // a multiple of tile
    const uint32_t nchunks = static_cast<uint32_t>(a.ntiles);
    const uint32_t total = static_cast<uint32_t>(a.total);
    const uint64_t nvec = a.nvec;
    const uint32_t skew = (static_cast<uint32_t>(a.debug) >> SL_DEBUG_SMEM_SKEW_SHIFT) & 7u;
    const uint32_t my0 = smem_addr(ring + skew + threadIdx.x), stride = cta * 16u;
    // vectors of claim c from its first one (0 past the last claim), and the
    // address of this thread's first copy in it
    const auto chunk = [&](uint32_t c, const uint4*& p, uint32_t& len) {
        if (c >= total) {
            p = buf;
            len = 0;
            return;
        }
        const uint64_t base = static_cast<uint64_t>(c % nchunks) * chunk_vec;
        const uint64_t left = nvec - base;
        len = left < chunk_vec ? static_cast<uint32_t>(left) : chunk_vec;
        p = buf + base + threadIdx.x;
    };
    Acc<DT> acc;
    uint32_t full_tiles = 0;
    volatile uint32_t* vs = slot;
    if (threadIdx.x == 0) {
        vs[0] = atomicAdd(a.next, 1u);
        vs[1] = atomicAdd(a.next, 1u);
    }
    __syncthreads();
    const uint4* cp;  // this thread's first copy in the current chunk
    const uint4* np;  // ... in the next chunk
    uint32_t clen, nlen;
    chunk(vs[0], cp, clen);
    chunk(vs[1], np, nlen);
    if (clen) {
        // prologue: the D groups of the chunk's first tile
#pragma unroll
        for (int k = 0; k < D; ++k) {
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const uint32_t j = k * G + g;
                if (threadIdx.x + j * cta < clen) {
                    cp_async16(my0 + j * stride, cp + j * cta);
                    cov_count<COV>(a, (cp + j * cta) - buf);
                }
            }
            cp_async_commit();
        }
    }
#pragma unroll 1
    for (uint32_t it = 0; clen; ++it) {
        if (threadIdx.x == 0) vs[(it + 2) % 3] = atomicAdd(a.next, 1u);
        const uint32_t ntl = (clen + tile - 1) / tile;
#pragma unroll 1
        for (uint32_t t = 0; t < ntl; ++t) {
            // vectors from this tile's start to the chunk's end, and the same
            // for the tile its groups are refilled from (the chunk's next tile,
            // else the next chunk's first, else none)
            const uint32_t crem = clen - t * tile;
            const uint4* rp;
            uint32_t rrem;
            if (t + 1 < ntl) {
                rp = cp + (t + 1) * tile;
                rrem = crem - tile;
            } else {
                rp = np;
                rrem = nlen;
            }
            if (crem >= tile && rrem >= tile) {
                // both tiles whole: no range checks
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    cp_async_wait<D - 1>();
#pragma unroll
                    for (int g = 0; g < G; ++g) acc.fold(lds16(my0 + (k * G + g) * stride));
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        const uint32_t j = k * G + g;
                        cp_async16(my0 + j * stride, rp + j * cta);
                        cov_count<COV>(a, (rp + j * cta) - buf);
                    }
                    cp_async_commit();
                }
                ++full_tiles;
                continue;
            }
            const bool cfull = crem >= tile;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                cp_async_wait<D - 1>();
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const uint32_t j = k * G + g;
                    if (threadIdx.x + j * cta < crem) {
                        acc.fold(lds16(my0 + j * stride));
                        if (!cfull) acc.n += 1;
                    }
                }
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const uint32_t j = k * G + g;
                    if (threadIdx.x + j * cta < rrem) {
                        cp_async16(my0 + j * stride, rp + j * cta);
                        cov_count<COV>(a, (rp + j * cta) - buf);
                    }
                }
                cp_async_commit();
            }
            if (cfull) ++full_tiles;
        }
        __syncthreads();  // the claim made at the top of this chunk is visible
        cp = np;
        clen = nlen;
        chunk(vs[(it + 2) % 3], np, nlen);
    }
    cp_async_wait<0>();
    acc.n += full_tiles * (D * G);
    cta_finish<DT>(acc, true, threadIdx.x >> 5, cta >> 5, a);
}

template <int D, int G, int DT>
static const void* fn() {
    return reinterpret_cast<const void*>(&k_cpasync_dyn<D, G, DT>);
}

// Instantiated: one copy per group at D = 1, 2, 3, 4, 6, 8; D x G = 2 x 2,
// 1 x 4, 2 x 4, 1 x 8, 2 x 8.
template <int DT>
static const void* dyn_for(int d, int g) {
    if (g == 1) {
        switch (d) {
        case 1: return fn<1, 1, DT>();
        case 2: return fn<2, 1, DT>();
        case 3: return fn<3, 1, DT>();
        case 4: return fn<4, 1, DT>();
        case 6: return fn<6, 1, DT>();
        case 8: return fn<8, 1, DT>();
        default: return nullptr;
        }
    }
    if (g == 2 && d == 2) return fn<2, 2, DT>();
    if (g == 4 && d == 1) return fn<1, 4, DT>();
    if (g == 4 && d == 2) return fn<2, 4, DT>();
    if (g == 8 && d == 1) return fn<1, 8, DT>();
    if (g == 8 && d == 2) return fn<2, 8, DT>();
    return nullptr;
}

const void* cpasync_dyn_kernel(int dtype, int d, int g) {
    switch (dtype) {
    case SL_U32: return dyn_for<SL_U32>(d, g);
    case SL_F32: return dyn_for<SL_F32>(d, g);
    case SL_BF16: return dyn_for<SL_BF16>(d, g);
    case SL_FP8_E4M3: return dyn_for<SL_FP8_E4M3>(d, g);
    default: return nullptr;
    }
}

const void* cpasync_dyn_cov_kernel(int d, int g) {
    if (d == 4 && g == 1) return reinterpret_cast<const void*>(&k_cpasync_dyn<4, 1, SL_U32, true>);
    if (d == 2 && g == 4) return reinterpret_cast<const void*>(&k_cpasync_dyn<2, 4, SL_U32, true>);
    return nullptr;
}

}  // namespace sl
