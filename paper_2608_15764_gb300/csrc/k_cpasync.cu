// k_cpasync.cu -- the cp.async streaming kernel.
//
// Paper §4.3 compares cp.async, which writes shared memory without a
// destination register, against plain loads at equal offered concurrency.
// Here each thread copies 16 bytes per commit group with
// cp.async.cg.shared.global into stage slot g mod D of a D-deep ring and keeps
// D groups in flight: after committing group g+D-1 it waits until at most D-1
// groups are pending (so group g has landed), reads its own slot back with
// ld.shared and folds it.  A thread reads only the slot it wrote itself, so no
// CTA barrier is needed.
//
// The address sequence of a thread is the LDG kernel's at K = D: tile = cta*D
// vectors, CTA b walks tiles b, b+grid, ..., and chunk k of a tile is vector
// tile*cta*D + k*cta + t.  Only the way the loads are kept in flight differs.
#include "sl_device.cuh"

namespace sl {

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* gptr) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(gptr) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Position in the chunk sequence of one CTA.
struct ChunkCursor {
    TileCursor c;
    uint32_t k;
    __device__ __forceinline__ void start(uint32_t ntiles) { c.start(ntiles); k = 0; }
    template <int D>
    __device__ __forceinline__ void next(uint32_t ntiles) {
        if (++k == D) { k = 0; c.next(ntiles); }
    }
    // vector index of this thread's chunk, or ~0 when past the end
    __device__ __forceinline__ uint64_t vec(const KArgs& a, uint32_t total, uint32_t cta) const {
        if (c.it >= total) return ~0ull;
        const uint64_t idx = static_cast<uint64_t>(c.tile(a)) * a.tile_vec + k * cta + threadIdx.x;
        return idx < a.nvec ? idx : ~0ull;
    }
};

template <int D, int DT>
__global__ void __launch_bounds__(1024) k_cpasync(const KArgs a) {
    extern __shared__ __align__(16) uint4 ring[];  // [D][cta]
    cta_start(a);
    const uint32_t cta = blockDim.x;
    const uint32_t ntiles = static_cast<uint32_t>(a.ntiles);
    const uint32_t total = static_cast<uint32_t>(a.total);
    const uint4* __restrict__ buf = static_cast<const uint4*>(a.buf);
    const uint32_t my_slot0 = smem_addr(ring + threadIdx.x);
    const uint32_t slot_stride = cta * 16u;
    Acc<DT> acc;
    ChunkCursor ic, cc;  // issue and consume cursors
    ic.start(ntiles);
    cc.start(ntiles);
    uint32_t islot = 0, cslot = 0;

#pragma unroll
    for (int g = 0; g < D - 1; ++g) {
        const uint64_t idx = ic.vec(a, total, cta);
        if (idx != ~0ull) cp_async16(my_slot0 + islot * slot_stride, buf + idx);
        cp_async_commit();
        ic.next<D>(ntiles);
        islot = (islot + 1 == D) ? 0 : islot + 1;
    }
#pragma unroll 1
    while (cc.c.it < total) {
        const uint64_t idx = ic.vec(a, total, cta);
        if (idx != ~0ull) cp_async16(my_slot0 + islot * slot_stride, buf + idx);
        cp_async_commit();
        ic.next<D>(ntiles);
        islot = (islot + 1 == D) ? 0 : islot + 1;

        cp_async_wait<D - 1>();
        if (cc.vec(a, total, cta) != ~0ull) {
            acc.fold(lds16(my_slot0 + cslot * slot_stride));
            acc.n += 1;
        }
        cc.next<D>(ntiles);
        cslot = (cslot + 1 == D) ? 0 : cslot + 1;
    }
    cp_async_wait<0>();
    cta_finish<DT>(acc, true, threadIdx.x >> 5, cta >> 5, a);
}

template <int DT>
static const void* cpasync_for(int d) {
    switch (d) {
    case 1: return reinterpret_cast<const void*>(&k_cpasync<1, DT>);
    case 2: return reinterpret_cast<const void*>(&k_cpasync<2, DT>);
    case 3: return reinterpret_cast<const void*>(&k_cpasync<3, DT>);
    case 4: return reinterpret_cast<const void*>(&k_cpasync<4, DT>);
    case 5: return reinterpret_cast<const void*>(&k_cpasync<5, DT>);
    case 6: return reinterpret_cast<const void*>(&k_cpasync<6, DT>);
    case 7: return reinterpret_cast<const void*>(&k_cpasync<7, DT>);
    case 8: return reinterpret_cast<const void*>(&k_cpasync<8, DT>);
    default: return nullptr;
    }
}

const void* cpasync_kernel(int dtype, int d) {
    switch (dtype) {
    case SL_U32: return cpasync_for<SL_U32>(d);
    case SL_F32: return cpasync_for<SL_F32>(d);
    case SL_BF16: return cpasync_for<SL_BF16>(d);
    case SL_FP8_E4M3: return cpasync_for<SL_FP8_E4M3>(d);
    default: return nullptr;
    }
}

}  // namespace sl
