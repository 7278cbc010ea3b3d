// k_batch_misc.cu -- cp.async and TMA class kernels of the batched form, and
// the per-buffer combine.
#include "k_batch.cuh"
#include "sl_mbar.cuh"

namespace sl {

__device__ __forceinline__ void kb_cp_async16(uint32_t saddr, const void* gptr) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(gptr) : "memory");
}
__device__ __forceinline__ void kb_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void kb_cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// cp.async class kernel: per item, chunk j of the item is vectors
// [j*cta, (j+1)*cta); each thread copies its 16 bytes of chunk j into ring
// slot j mod D with D commit groups in flight, reads its own slot back and
// folds (as k_cpasync).  The pipeline drains at the end of each item.
template <int D, int DT>
__global__ void __launch_bounds__(1024) kb_cpasync(const BArgs a) {
    extern __shared__ __align__(128) uint4 cp_ring[];  // [D][cta], 128-byte aligned (cp.async destinations)
    __shared__ uint32_t slot;
    const uint32_t cta = blockDim.x, t = threadIdx.x;
    const uint32_t my0 = smem_addr(cp_ring + t), stride = cta * 16u;
    for (;;) {
        const uint32_t item = claim_item(a, &slot);
        if (item >= a.nitems) break;
        const BatchItem it = a.items[item];
        const uint32_t nchunks = (it.nvec + cta - 1) / cta;
        Acc<DT> acc;
        uint32_t islot = 0, cslot = 0;
#pragma unroll
        for (int g = 0; g < D - 1; ++g) {
            const uint32_t v = static_cast<uint32_t>(g) * cta + t;
            if (static_cast<uint32_t>(g) < nchunks && v < it.nvec) kb_cp_async16(my0 + islot * stride, it.ptr + v);
            kb_cp_commit();
            islot = (islot + 1 == D) ? 0 : islot + 1;
        }
#pragma unroll 1
        for (uint32_t j = 0; j < nchunks; ++j) {
            const uint32_t g = j + D - 1;
            const uint32_t v = g * cta + t;
            if (g < nchunks && v < it.nvec) kb_cp_async16(my0 + islot * stride, it.ptr + v);
            kb_cp_commit();
            islot = (islot + 1 == D) ? 0 : islot + 1;
            kb_cp_wait<D - 1>();
            if (j * cta + t < it.nvec) {
                acc.fold(lds16(my0 + cslot * stride));
                acc.n += 1;
            }
            cslot = (cslot + 1 == D) ? 0 : cslot + 1;
        }
        kb_cp_wait<0>();
        warp_item_store<DT>(acc, a.parts + it.part + (t >> 5));
    }
}

// Per-stage note from the producer to the consumers of the TMA class kernel.
struct StageMeta {
    uint32_t part;   // first partial slot of the item this stage belongs to
    uint32_t nv;     // 16-byte vectors in the stage
    uint32_t flags;  // STAGE_LAST_OF_ITEM, STAGE_DONE
    uint32_t pad;
};
constexpr uint32_t STAGE_LAST_OF_ITEM = 1, STAGE_DONE = 2;

// TMA class kernel: lane 0 of warp 0 claims items and streams them through
// the mbarrier ring stage by stage (an item of n bytes takes ceil(n / S)
// stages; the ring does not drain between items), noting in each stage which
// item it belongs to.  Consumer warps fold every stage and write their item
// partial after the item's last stage.  When the items run out the producer
// arms one more stage marked DONE with a plain arrive (no bytes).  Waits are
// bounded and issued copies are drained before exit, as in k_tma.  As there,
// a consumer thread reads its last B vectors of a stage into registers and
// its warp releases the stage before folding them (B = 4, or 1 where a
// thread reads fewer than 4 vectors of a stage).
template <int DT, int B>
__global__ void __launch_bounds__(1024) kb_tma(const BArgs a) {
    extern __shared__ __align__(128) uint8_t tma_ring[];
    __shared__ __align__(8) uint64_t full[SL_MAX_STAGES];
    __shared__ __align__(8) uint64_t empty[SL_MAX_STAGES];
    __shared__ StageMeta meta[SL_MAX_STAGES];
    __shared__ volatile int abort_flag;

    const uint32_t nst = static_cast<uint32_t>(a.nst);
    const uint32_t S = a.stage_bytes;
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t ncw = (blockDim.x >> 5) - 1;
    const uint32_t ring0 = smem_addr(tma_ring);
    const uint32_t full0 = smem_addr(full), empty0 = smem_addr(empty);
    if (threadIdx.x == 0) {
        ring_init(full0, empty0, nst, ncw);
        abort_flag = 0;
    }
    __syncthreads();

    if (warp == 0) {
        if (lane == 0) {
            uint32_t armed = 0, last_par = 0, s = 0, r = 0;
            bool stop = false;
            while (!stop) {
                const uint32_t item = atomicAdd(a.next, 1u);
                const bool done = item >= a.nitems;
                BatchItem it{nullptr, 0u, 0u};
                uint32_t nstage = 1, nbytes = 0;
                if (!done) {
                    it = a.items[item];
                    nbytes = it.nvec * 16u;
                    nstage = (nbytes + S - 1) / S;
                }
                for (uint32_t k = 0; k < nstage; ++k) {
                    if (r > 0 && !bounded_wait(empty0 + 8 * s, (r - 1) & 1u, a.err, a.timeout_ns, &abort_flag, true,
                                               DEV_ERR_TIMEOUT_EMPTY)) {
                        stop = true;
                        break;
                    }
                    if (done) {
                        // The copy this stage last carried has landed (its
                        // consumers released the stage), and the sentinel
                        // advances full[s] by one more phase: stop draining it.
                        armed &= ~(1u << s);
                        meta[s] = StageMeta{0u, 0u, STAGE_DONE, 0u};
                        mbar_arrive(full0 + 8 * s);
                    } else {
                        const uint32_t off = k * S;
                        const uint32_t len = nbytes - off < S ? nbytes - off : S;
                        meta[s] = StageMeta{it.part, len >> 4, k + 1 == nstage ? STAGE_LAST_OF_ITEM : 0u, 0u};
                        mbar_arrive_expect_tx(full0 + 8 * s, len);
                        bulk_g2s(ring0 + s * S, reinterpret_cast<const uint8_t*>(it.ptr) + off, len, full0 + 8 * s);
                        armed |= 1u << s;
                        last_par = (last_par & ~(1u << s)) | ((r & 1u) << s);
                    }
                    if (++s == nst) { s = 0; ++r; }
                }
                if (done) stop = true;
            }
            for (uint32_t q = 0; q < nst; ++q)
                if (armed & (1u << q))
                    bounded_wait(full0 + 8 * q, (last_par >> q) & 1u, a.err, a.timeout_ns, &abort_flag, false,
                                 DEV_ERR_TIMEOUT_DRAIN);
        }
        __syncwarp();
    } else {
        const uint32_t ct = threadIdx.x - 32, nct = ncw * 32;
        Acc<DT> acc;
        uint32_t s = 0, r = 0;
        for (;;) {
            const bool got =
                bounded_wait(full0 + 8 * s, r & 1u, a.err, a.timeout_ns, &abort_flag, true, DEV_ERR_TIMEOUT_FULL);
            if (!__all_sync(FULL_MASK, got)) break;
            const StageMeta m = meta[s];  // read before the stage is released
            if (m.flags & STAGE_DONE) break;
            const uint32_t base = ring0 + s * S;
            uint32_t v = ct;
#pragma unroll 1
            for (; v + B * nct < m.nv; v += B * nct) {
                uint4 x[B];
#pragma unroll
                for (int u = 0; u < B; ++u) x[u] = lds16(base + 16u * (v + u * nct));
#pragma unroll
                for (int u = 0; u < B; ++u) acc.fold(x[u]);
                acc.n += B;
            }
            uint4 x[B];
#pragma unroll
            for (int u = 0; u < B; ++u)
                if (v + u * nct < m.nv) x[u] = lds16(base + 16u * (v + u * nct));
            __syncwarp();
            if (lane == 0) mbar_arrive(empty0 + 8 * s);
#pragma unroll
            for (int u = 0; u < B; ++u)
                if (v + u * nct < m.nv) {
                    acc.fold(x[u]);
                    acc.n += 1;
                }
            if (m.flags & STAGE_LAST_OF_ITEM) {
                warp_item_store<DT>(acc, a.parts + m.part + (warp - 1));
                acc = Acc<DT>();
            }
            if (++s == nst) { s = 0; ++r; }
        }
    }
    __syncthreads();
}

// Per-buffer combine: one warp per buffer adds the buffer's partial slots in
// a fixed order (lane l takes slots l, l+32, ...; integer parts exact, float
// parts in FP64), merges the lanes with a shuffle butterfly and writes the
// buffer's sl_result.  The device error word becomes every result's status.
__global__ void __launch_bounds__(256) kb_combine(const BufSeg* __restrict__ segs, uint32_t nbuf,
                                                 const WarpPartial* __restrict__ parts, const uint32_t* err,
                                                 sl_result* __restrict__ out) {
    const uint32_t b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (b >= nbuf) return;  // warp-uniform
    const BufSeg g = segs[b];
    uint32_t sum = 0;
    uint64_t x = 0, n = 0;
    double f = 0.0;
    for (uint32_t i = lane; i < g.pcount; i += 32) {
        const WarpPartial p = parts[g.pstart + i];
        sum += p.sum;
        x ^= p.xr;
        n += p.issued;
        f += static_cast<double>(p.hi) + static_cast<double>(p.lo);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_xor_sync(FULL_MASK, sum, o);
        x ^= __shfl_xor_sync(FULL_MASK, x, o);
        n += __shfl_xor_sync(FULL_MASK, n, o);
        f += __shfl_xor_sync(FULL_MASK, f, o);
    }
    if (lane == 0) {
        sl_result r;
        r.xor_u64 = x;
        r.issued_loads = n;
        r.device_ns = 0;
        r.window_ns = 0;
        r.fsum = f;
        r.fsum_hi = static_cast<float>(f);
        r.fsum_lo = static_cast<float>(f - static_cast<double>(r.fsum_hi));
        r.sum_u32 = sum;
        r.status = *err ? SL_ERR_TIMEOUT : SL_OK;
        r.grid = 0;
        r.cta = 0;
        r.resident_per_sm = 0;
        r.smem_bytes = 0;
        out[b] = r;
    }
}

template <int DT>
static const void* kb_cp_d(int d) {
    switch (d) {
    case 1: return reinterpret_cast<const void*>(&kb_cpasync<1, DT>);
    case 2: return reinterpret_cast<const void*>(&kb_cpasync<2, DT>);
    case 3: return reinterpret_cast<const void*>(&kb_cpasync<3, DT>);
    case 4: return reinterpret_cast<const void*>(&kb_cpasync<4, DT>);
    case 5: return reinterpret_cast<const void*>(&kb_cpasync<5, DT>);
    case 6: return reinterpret_cast<const void*>(&kb_cpasync<6, DT>);
    case 7: return reinterpret_cast<const void*>(&kb_cpasync<7, DT>);
    case 8: return reinterpret_cast<const void*>(&kb_cpasync<8, DT>);
    default: return nullptr;
    }
}

const void* batch_cpasync_kernel(int dtype, int d) {
    switch (dtype) {
    case SL_U32: return kb_cp_d<SL_U32>(d);
    case SL_F32: return kb_cp_d<SL_F32>(d);
    case SL_BF16: return kb_cp_d<SL_BF16>(d);
    case SL_FP8_E4M3: return kb_cp_d<SL_FP8_E4M3>(d);
    default: return nullptr;
    }
}

template <int B>
static const void* kb_tma_b(int dtype) {
    switch (dtype) {
    case SL_U32: return reinterpret_cast<const void*>(&kb_tma<SL_U32, B>);
    case SL_F32: return reinterpret_cast<const void*>(&kb_tma<SL_F32, B>);
    case SL_BF16: return reinterpret_cast<const void*>(&kb_tma<SL_BF16, B>);
    case SL_FP8_E4M3: return reinterpret_cast<const void*>(&kb_tma<SL_FP8_E4M3, B>);
    default: return nullptr;
    }
}

const void* batch_tma_kernel(int dtype, int batch) {
    if (batch == 4) return kb_tma_b<4>(dtype);
    if (batch == 1) return kb_tma_b<1>(dtype);
    return nullptr;
}

cudaError_t launch_batch_combine(const BufSeg* segs, uint32_t nbuf, const WarpPartial* parts, const uint32_t* err,
                                 sl_result* out, cudaStream_t s) {
    if (nbuf == 0) return cudaSuccess;
    const uint32_t blocks = (nbuf + 7) / 8;  // 8 warps (buffers) per CTA
    kb_combine<<<blocks, 256, 0, s>>>(segs, nbuf, parts, err, out);
    return cudaGetLastError();
}

}  // namespace sl
