// k_tma.cu -- the TMA (bulk asynchronous copy) streaming kernels.
//
// The paper names Hopper's TMA and bulk-asynchronous copies (§2) but has no
// TMA kernel; both ring layouts below are the library's own Blackwell design.
//
// ---- k_tma: one ring per CTA (SL_RING_CTA) ----
// CTA = one producer warp + `cta` consumer threads.  The buffer is cut into
// stage-sized chunks (stage_bytes, the last one ragged); CTA b takes chunks
// b, b+grid, ... over all passes (reversed for SL_DESC).  Lane 0 of warp 0
// owns a ring of `nst` stages in dynamic shared memory with two mbarriers per
// stage:
//   full[s]  count 1: the producer arms it with arrive.expect_tx(bytes) and
//            issues one cp.async.bulk global->shared that completes the
//            transaction bytes;
//   empty[s] count = consumer warps: each consumer warp arrives once all its
//            lanes have read the stage into registers.
// The producer waits on empty[s] before refilling stage s; consumers wait on
// full[s], read the stage with ld.shared.v4 (thread t takes vectors t,
// t+cta, ...) and fold, B vectors at a time: the warp arrives on empty[s]
// once its last batch is in registers and folds that batch afterwards, so
// the refill overlaps the fold.  No multicast is used anywhere.
//
// Every wait is bounded: a wait that exceeds a.timeout_ns (by %globaltimer)
// or a hard iteration cap records an error code in the CTA's shared error word
// (published to *a.err when the CTA finishes, after any previous launch on
// the stream has completed), raises the CTA's abort flag and returns false.  Waiters also give up when they see the abort
// flag.  Before exiting after an abort, the producer waits (bounded) for
// every bulk copy it issued to land (it does so on every exit), so no copy is
// in flight into shared memory when the CTA exits.  A consumer warp leaves
// the ring only when all its lanes agree (__all_sync), so warp-wide shuffles
// after the loop see every lane.
#include "sl_mbar.cuh"

namespace sl {

template <int DT, int B, bool COV = false>
__global__ void __launch_bounds__(1024, 1) k_tma(const KArgs a) {
    extern __shared__ __align__(128) uint8_t ring[];
    __shared__ __align__(8) uint64_t full[SL_MAX_STAGES];
    __shared__ __align__(8) uint64_t empty[SL_MAX_STAGES];
    __shared__ volatile int abort_flag;
    __shared__ uint32_t cta_err;  // a bounded wait's error code, published to *a.err by cta_finish

    cta_start(a);
    const uint32_t nst = static_cast<uint32_t>(a.nst);
    const uint32_t ntiles = static_cast<uint32_t>(a.ntiles);
    const uint32_t total = static_cast<uint32_t>(a.total);
    const uint32_t stage_bytes = a.tile_vec * 16u;
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t ncw = (blockDim.x >> 5) - 1;  // consumer warps
    const uint64_t bytes = a.nvec * 16ull;
    const uint8_t* __restrict__ gbuf = static_cast<const uint8_t*>(a.buf);
    const uint32_t ring0 = smem_addr(ring);
    const uint32_t full0 = smem_addr(full), empty0 = smem_addr(empty);

    if (threadIdx.x == 0) {
        ring_init(full0, empty0, nst, ncw);
        abort_flag = 0;
        cta_err = 0;
    }
    __syncthreads();

    Acc<DT> acc;
    if (warp == 0) {
        if (lane == 0) {
            // ---- producer ----
            uint32_t armed = 0;     // bit s: stage s has had a copy issued
            uint32_t last_par = 0;  // bit s: parity of the round of stage s's last copy
            TileCursor c;
            c.start(ntiles);
            uint32_t s = 0, r = 0;  // stage and round of chunk i = r*nst + s
            for (uint32_t i = 0; c.it < total; c.next(ntiles), ++i) {
                if (r > 0 && !bounded_wait(empty0 + 8 * s, (r - 1) & 1u, &cta_err, a.timeout_ns, &abort_flag, true,
                                           DEV_ERR_TIMEOUT_EMPTY))
                    break;
                const uint64_t off = static_cast<uint64_t>(c.tile(a)) * stage_bytes;
                const uint64_t left = bytes - off;
                const uint32_t len = left < stage_bytes ? static_cast<uint32_t>(left) : stage_bytes;
                if (!((a.debug & SL_DEBUG_TMA_SKIP_STAGE) && i == 1)) {  // debug: leave chunk 1 unarmed
                    mbar_arrive_expect_tx(full0 + 8 * s, len);
                    bulk_g2s(ring0 + s * stage_bytes, gbuf + off, len, full0 + 8 * s);
                    if constexpr (COV) {
                        for (uint64_t v = off >> 4; v < (off + len) >> 4; ++v) cov_count<COV>(a, v);
                    }
                    armed |= 1u << s;
                    last_par = (last_par & ~(1u << s)) | ((r & 1u) << s);
                }
                if (++s == nst) { s = 0; ++r; }
            }
            // Drain: every issued copy must have landed before the CTA exits
            // (immediate in normal operation; bounded after an abort).
            {
                for (uint32_t s = 0; s < nst; ++s)
                    if (armed & (1u << s))
                        bounded_wait(full0 + 8 * s, (last_par >> s) & 1u, &cta_err, a.timeout_ns, &abort_flag,
                                     false, DEV_ERR_TIMEOUT_DRAIN);
            }
        }
        __syncwarp();
    } else {
        // ---- consumers ----
        const uint32_t ct = threadIdx.x - 32, nct = ncw * 32;
        TileCursor c;
        c.start(ntiles);
        uint32_t s = 0, r = 0;
        for (; c.it < total; c.next(ntiles)) {
            const bool got =
                bounded_wait(full0 + 8 * s, r & 1u, &cta_err, a.timeout_ns, &abort_flag, true, DEV_ERR_TIMEOUT_FULL);
            if (!__all_sync(FULL_MASK, got)) break;  // warp-uniform exit
            const uint64_t off = static_cast<uint64_t>(c.tile(a)) * stage_bytes;
            const uint64_t left = bytes - off;
            const uint32_t nv = (left < stage_bytes ? static_cast<uint32_t>(left) : stage_bytes) >> 4;
            const uint32_t base = ring0 + s * stage_bytes;
            // A thread's vectors of the stage are ct, ct + nct, ...: batches of
            // B while more than B remain, then the last batch (up to B) is
            // read into registers and the warp releases the stage before
            // folding it, so the producer's refill overlaps that fold.
            uint32_t v = ct;
#pragma unroll 1
            for (; v + B * nct < nv; v += B * nct) {
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
                if (v + u * nct < nv) x[u] = lds16(base + 16u * (v + u * nct));
            __syncwarp();
            if (lane == 0) mbar_arrive(empty0 + 8 * s);
#pragma unroll
            for (int u = 0; u < B; ++u)
                if (v + u * nct < nv) {
                    acc.fold(x[u]);
                    acc.n += 1;
                }
            if (++s == nst) { s = 0; ++r; }
        }
    }
    // consumer warps fold (all lanes left the ring together); warp 0 does not
    cta_finish<DT>(acc, warp != 0, warp - 1, ncw, a, &cta_err);
}

// ---- k_tma_warp: the CTA's stages dealt to its warps (SL_RING_WARP) ----
// The CTA holds the same ring of stages x stage_bytes as k_tma, without a
// producer warp: its W warps split the stages, warp w owning the nst =
// stages / W consecutive stages after those of warps 0..w-1 (a sub-ring), and
// the CTA's full barriers (one per stage, count 1) follow the stages in
// dynamic shared memory.  A warp's lane 0 is its sub-ring's only producer and
// its 32 lanes the only consumers, so a stage needs no empty barrier: once
// the warp has read stage s (__syncwarp), lane 0 re-arms it with
// arrive.expect_tx and issues the warp's next cp.async.bulk into it, after a
// proxy fence that orders the lanes' generic-proxy reads of the stage before
// the bulk copy's async-proxy writes.  The lanes' reads precede the
// __syncwarp in program order, which orders them before lane 0's fence and
// copy whether or not their values have been used yet: the EARLY refill
// below relies on that ordering alone.
//
// Chunks (stage-sized pieces of the buffer, the last one ragged) are dealt to
// warps grid-wide: global warp g = blockIdx.x * W + w takes chunks g, g + G,
// g + 2G, ... over all passes (G = grid * W; chunk c reads piece c mod
// nchunks, counted from the last piece for SL_DESC).  A warp's j-th chunk
// lives in its stage j mod nst and has landed when that stage's barrier
// completes phase j / nst; lane 0 refills a stage only after its warp has
// read it, so no barrier runs more than one phase ahead of its waiter.  A
// full stage gives each lane stage_bytes/512 vectors (8 for 4 KiB), read 8
// at a time.
//
// The warp count divides the stage count (at most SL_MAX_STAGES), so a CTA has
// at most SL_MAX_STAGES warps; registers are capped for four such CTAs per SM.
template <int DT, bool EARLY, bool COV = false>
__global__ void __launch_bounds__(SL_MAX_STAGES * 32, 4) k_tma_warp(const KArgs a) {
    extern __shared__ __align__(128) uint8_t ring[];
    __shared__ volatile int abort_flag;
    __shared__ uint32_t cta_err;

    cta_start(a);
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const uint32_t nst = static_cast<uint32_t>(a.nst) / nw;  // stages of this warp (the host checks W | stages)
    // chunk indices fit in 32 bits: the host checks total + grid * W < 2^32
    const uint32_t nchunks = static_cast<uint32_t>(a.ntiles);
    const uint32_t total = static_cast<uint32_t>(a.total);
    const uint32_t stage_bytes = a.tile_vec * 16u;
    const uint64_t bytes = a.nvec * 16ull;
    const uint8_t* __restrict__ gbuf = static_cast<const uint8_t*>(a.buf);
    const uint32_t my_ring = smem_addr(ring) + warp * nst * stage_bytes;
    const uint32_t my_full = smem_addr(ring) + static_cast<uint32_t>(a.nst) * stage_bytes + warp * nst * 8u;
    const uint32_t G = gridDim.x * nw;
    const uint32_t g0 = blockIdx.x * nw + warp;
    // debug: global warp 0 leaves its first chunk unarmed (it has one whenever
    // the buffer is not empty), so its first wait runs out
    const bool skip_one = (a.debug & SL_DEBUG_TMA_SKIP_STAGE) && g0 == 0;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        cta_err = 0;
    }
    if (lane == 0) {
        for (uint32_t s = 0; s < nst; ++s) mbar_init(my_full + 8 * s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    // byte offset and length of chunk c
    const auto piece = [&](uint32_t c, uint64_t& off, uint32_t& len) {
        uint32_t t = c < nchunks ? c : c % nchunks;
        if (a.desc) t = nchunks - 1 - t;
        off = static_cast<uint64_t>(t) * stage_bytes;
        const uint64_t left = bytes - off;
        len = left < stage_bytes ? static_cast<uint32_t>(left) : stage_bytes;
    };
    uint32_t armed = 0;     // lane 0: bit s = stage s has had a copy issued
    uint32_t last_par = 0;  // lane 0: bit s = parity of the phase of stage s's last copy
    const auto issue = [&](uint32_t s, uint32_t par, uint32_t c, uint32_t j) {
        if (skip_one && j == 0) return;  // the warp's j-th chunk (debug only)
        uint64_t off;
        uint32_t len;
        piece(c, off, len);
        mbar_arrive_expect_tx(my_full + 8 * s, len);
        bulk_g2s(my_ring + s * stage_bytes, gbuf + off, len, my_full + 8 * s);
        if constexpr (COV) {
            for (uint64_t v = off >> 4; v < (off + len) >> 4; ++v) cov_count<COV>(a, v);
        }
        armed |= 1u << s;
        last_par = (last_par & ~(1u << s)) | (par << s);
    };
    if (lane == 0) {
        for (uint32_t j = 0; j < nst; ++j) {
            const uint32_t c = g0 + j * G;
            if (c >= total) break;
            issue(j, 0u, c, j);
        }
    }

    Acc<DT> acc;
    uint32_t s = 0, r = 0;  // stage and round of the warp's current chunk (its j-th: j = r*nst + s)
#pragma unroll 1
    for (uint32_t c = g0; c < total; c += G) {
        const bool got = bounded_wait(my_full + 8 * s, r & 1u, &cta_err, a.timeout_ns, &abort_flag, true,
                                      DEV_ERR_TIMEOUT_FULL);
        if (!__all_sync(FULL_MASK, got)) break;  // warp-uniform exit
        uint64_t off;
        uint32_t len;
        piece(c, off, len);
        // Once every lane has read stage s (__syncwarp), lane 0 refills it.
        // EARLY: a full stage is refilled as soon as its last batch of
        // vectors is in registers, before that batch is folded, so the
        // refill's memory latency overlaps the fold.  Otherwise the stage is
        // refilled after the fold.  The host takes EARLY for BF16 payloads
        // (the longest fold) where each warp owns a single stage: 5-14%
        // faster there, while with two stages per warp (the other one in
        // flight during the fold) and for the shorter folds it measured
        // no faster or slower.
        const auto refill = [&]() {
            __syncwarp();
            if (lane == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                const uint32_t cn = c + nst * G;
                if (cn < total) issue(s, (r + 1) & 1u, cn, (r + 1) * nst + s);
            }
        };
        const uint32_t base = my_ring + s * stage_bytes + 16u * lane;
        if (len == stage_bytes) {
            const uint32_t per_lane = stage_bytes >> 9;  // a multiple of 8
#pragma unroll 1
            for (uint32_t i = 0; i < per_lane; i += 8) {
                uint4 v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = lds16(base + 512u * (i + u));
                if (EARLY && i + 8 == per_lane) refill();
#pragma unroll
                for (int u = 0; u < 8; ++u) acc.fold(v[u]);
            }
            acc.n += per_lane;
            if (!EARLY) refill();
        } else {
            const uint32_t nv = len >> 4;
#pragma unroll 1
            for (uint32_t v = lane; v < nv; v += 32) {
                acc.fold(lds16(my_ring + s * stage_bytes + 16u * v));
                acc.n += 1;
            }
            refill();
        }
        if (++s == nst) { s = 0; ++r; }
    }
    // Drain: every copy this warp issued must have landed before the CTA
    // exits (immediate in normal operation; bounded after an abort).
    if (lane == 0) {
        for (uint32_t t = 0; t < nst; ++t)
            if (armed & (1u << t))
                bounded_wait(my_full + 8 * t, (last_par >> t) & 1u, &cta_err, a.timeout_ns, &abort_flag, false,
                             DEV_ERR_TIMEOUT_DRAIN);
    }
    __syncwarp();
    cta_finish<DT>(acc, true, warp, nw, a, &cta_err);
}

const void* tma_cov_kernel(int batch) {
    return batch == 4 ? reinterpret_cast<const void*>(&k_tma<SL_U32, 4, true>)
                      : reinterpret_cast<const void*>(&k_tma<SL_U32, 1, true>);
}
const void* tma_warp_cov_kernel() { return reinterpret_cast<const void*>(&k_tma_warp<SL_U32, false, true>); }

const void* tma_warp_kernel(int dtype, bool early) {
    if (early) return dtype == SL_BF16 ? reinterpret_cast<const void*>(&k_tma_warp<SL_BF16, true>) : nullptr;
    switch (dtype) {
    case SL_U32: return reinterpret_cast<const void*>(&k_tma_warp<SL_U32, false>);
    case SL_F32: return reinterpret_cast<const void*>(&k_tma_warp<SL_F32, false>);
    case SL_BF16: return reinterpret_cast<const void*>(&k_tma_warp<SL_BF16, false>);
    case SL_FP8_E4M3: return reinterpret_cast<const void*>(&k_tma_warp<SL_FP8_E4M3, false>);
    default: return nullptr;
    }
}

template <int B>
static const void* tma_for(int dtype) {
    switch (dtype) {
    case SL_U32: return reinterpret_cast<const void*>(&k_tma<SL_U32, B>);
    case SL_F32: return reinterpret_cast<const void*>(&k_tma<SL_F32, B>);
    case SL_BF16: return reinterpret_cast<const void*>(&k_tma<SL_BF16, B>);
    case SL_FP8_E4M3: return reinterpret_cast<const void*>(&k_tma<SL_FP8_E4M3, B>);
    default: return nullptr;
    }
}

const void* tma_kernel(int dtype, int batch) {
    if (batch == 4) return tma_for<4>(dtype);
    if (batch == 1) return tma_for<1>(dtype);
    return nullptr;
}

}  // namespace sl
