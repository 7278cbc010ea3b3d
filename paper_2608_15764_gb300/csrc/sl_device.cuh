// sl_device.cuh -- device-side building blocks of the streaming-load kernels:
// 16-byte global loads, the checksum / compensated-sum fold, warp reduction
// and per-warp partial output.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sl_internal.h"

namespace sl {

constexpr unsigned FULL_MASK = 0xFFFFFFFFu;

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One 16-byte global load (paper §3: one ld.global per offered load; §4.2
// primary cell uses .cg, which caches in L2 only).  volatile keeps every load
// in the program and in source order.
template <int COP>
__device__ __forceinline__ uint4 ldg16(const uint4* p) {
    uint4 v;
    if constexpr (COP == SL_COP_CG) {
        asm volatile("ld.global.cg.v4.u32 {%0,%1,%2,%3}, [%4];"
                     : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    } else if constexpr (COP == SL_COP_CG_L2_256) {
        asm volatile("ld.global.cg.L2::256B.v4.u32 {%0,%1,%2,%3}, [%4];"
                     : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    } else {
        asm volatile("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0,%1,%2,%3}, [%4];"
                     : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    }
    return v;
}

__device__ __forceinline__ uint4 lds16(uint32_t saddr) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(saddr));
    return v;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- packed float pairs -------------------------------------------------------
// Two FP32 values in one 64-bit register pair (lane 0 = low word), operated on
// by the sm_100-family packed instructions add/sub.rn.f32x2: each lane is an
// ordinary IEEE round-to-nearest FP32 operation (subnormals kept), two lanes
// per instruction.
__device__ __forceinline__ uint64_t f2_pack(uint32_t lo_bits, uint32_t hi_bits) {
    uint64_t d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "r"(lo_bits), "r"(hi_bits));
    return d;
}
__device__ __forceinline__ float f2_lane0(uint64_t p) { return __uint_as_float(static_cast<uint32_t>(p)); }
__device__ __forceinline__ float f2_lane1(uint64_t p) { return __uint_as_float(static_cast<uint32_t>(p >> 32)); }
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// ---- per-vector FP8 sum ----------------------------------------------------------
// FP8 E4M3: 8 values per half vector.  cvt.rn.f16x2.e4m3x2 widens two codes to
// half exactly (every E4M3 value is a half), add.f32.f16 adds a half to an
// FP32 accumulator.  Every E4M3 value is an integer multiple of 2^-9 below
// 2^9, so any partial sum of 16 of them is a multiple of 2^-9 below 2^13 and
// fits the 24-bit FP32 significand: each half's sum, and their total, are
// exact in any order.
__device__ __forceinline__ float fp8_word_sum(uint32_t w, float acc) {
    asm("{\n\t.reg .b16 q0, q1, a0, a1, b0, b1;\n\t.reg .b32 h0, h1;\n\t"
        "mov.b32 {q0, q1}, %1;\n\t"
        "cvt.rn.f16x2.e4m3x2 h0, q0;\n\t"
        "cvt.rn.f16x2.e4m3x2 h1, q1;\n\t"
        "mov.b32 {a0, a1}, h0;\n\t"
        "mov.b32 {b0, b1}, h1;\n\t"
        "add.rn.f32.f16 %0, a0, %0;\n\t"
        "add.rn.f32.f16 %0, a1, %0;\n\t"
        "add.rn.f32.f16 %0, b0, %0;\n\t"
        "add.rn.f32.f16 %0, b1, %0;\n\t}"
        : "+f"(acc) : "r"(w));
    return acc;
}

// ---- register budget of the plain-load kernels --------------------------------
// Minimum resident CTAs per SM asked of the compiler for an LDG kernel
// (__launch_bounds__).  A bfloat16 fold (eight TwoSum steps per vector) with
// up to K = 8 loads in flight is held to 64 registers per thread, so that four
// 256-thread (two 512-thread) CTAs stay resident: with fewer warps its
// dependent TwoSum chains cannot hide the load latency (at K = 8 the
// unconstrained allocation of 78 registers leaves three CTAs and ~7% less
// bandwidth).  Every other kernel takes the registers it wants (K loaded
// vectors must stay in registers).
template <int K, int CTA, int DT>
constexpr int ldg_min_blocks() {
    return (DT == SL_BF16 && K <= 8 && CTA >= 256) ? 1024 / CTA : 1;
}

// ---- coverage audit ------------------------------------------------------------
// In the coverage instantiations (COV = true) every load of 16-byte vector i
// also adds 1 to a.cov[i]; elsewhere this compiles to nothing.
template <bool COV>
__device__ __forceinline__ void cov_count(const KArgs& a, uint64_t i) {
    if constexpr (COV) atomicAdd(a.cov + i, 1u);
}

// ---- the fold ----------------------------------------------------------------
// Per-thread accumulator.  Integer part (every dtype): wraparound uint32 sum
// of the four words and XOR of the two little-endian uint64 halves.
//
// Float part: compensated FP32 summation in which every addition's rounding
// error is recovered exactly with TwoSum (Knuth) and added to a separate
// error sum, so the represented value is s + e with an error of order u^2
// times sum|x| (u = 2^-24) instead of the 2u sum|x| of Kahan's recurrence.
// It runs as two independent lanes of packed f32x2 arithmetic (lane 0 takes
// the even-numbered values of a vector, lane 1 the odd-numbered ones), so one
// TwoSum instruction sequence serves two elements:
//   FP32: each of the 4 values goes through TwoSum (2 packed steps);
//   BF16: each of the 8 values is widened exactly to FP32 (a shift or a mask)
//         and goes through TwoSum (4 packed steps), so no addition inside a
//         vector is left uncompensated, whatever the values' range;
//   FP8:  the two half-vector sums, each exact (fp8_word_sum), go through one
//         packed TwoSum step.
template <int DT>
struct Acc {
    uint32_t s = 0, xl = 0, xh = 0;
    uint32_t n = 0;  // 16-byte loads folded by this thread (the host keeps it below 2^32)
    uint64_t fs = 0, fe = 0;  // packed (lane 0, lane 1) running sums and error sums; 0 bits = +0.0f

    // TwoSum of the packed pair x into (fs, fe), lane by lane.
    __device__ __forceinline__ void add2(uint64_t x) {
        const uint64_t t = f2_add(fs, x);
        const uint64_t bp = f2_sub(t, fs);
        const uint64_t d1 = f2_sub(fs, f2_sub(t, bp));
        const uint64_t d2 = f2_sub(x, bp);
        fe = f2_add(fe, f2_add(d1, d2));
        fs = t;
    }

    __device__ __forceinline__ void fold(const uint4& v) {
        s += (v.x + v.y) + (v.z + v.w);
        xl ^= v.x ^ v.z;
        xh ^= v.y ^ v.w;
        if constexpr (DT == SL_F32) {
            add2(f2_pack(v.x, v.y));
            add2(f2_pack(v.z, v.w));
        } else if constexpr (DT == SL_BF16) {
            // element 2i is the low half of word i, element 2i+1 the high half;
            // a bfloat16 is the top 16 bits of the FP32 with the same value
            add2(f2_pack(v.x << 16, v.x & 0xFFFF0000u));
            add2(f2_pack(v.y << 16, v.y & 0xFFFF0000u));
            add2(f2_pack(v.z << 16, v.z & 0xFFFF0000u));
            add2(f2_pack(v.w << 16, v.w & 0xFFFF0000u));
        } else if constexpr (DT == SL_FP8_E4M3) {
            const float a = fp8_word_sum(v.y, fp8_word_sum(v.x, 0.0f));
            const float b = fp8_word_sum(v.w, fp8_word_sum(v.z, 0.0f));
            add2(f2_pack(__float_as_uint(a), __float_as_uint(b)));
        }
    }

    // The float part as one double-float pair (hi, lo): the two lanes merged
    // with TwoSum and renormalised.
    __device__ __forceinline__ void float_part(float& hi, float& lo) const;
};

// Error-free sum of two floats (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Double-float add of two partials' float parts (TwoSum, then renormalise).
__device__ __forceinline__ void df_add(float& hi, float& lo, float ohi, float olo) {
    float sh, se;
    two_sum(hi, ohi, sh, se);
    se += lo + olo;
    hi = sh + se;
    lo = se - (hi - sh);
}

template <int DT>
__device__ __forceinline__ void Acc<DT>::float_part(float& hi, float& lo) const {
    hi = f2_lane0(fs);
    lo = f2_lane0(fe);
    df_add(hi, lo, f2_lane1(fs), f2_lane1(fe));
}

// Shuffle-butterfly reduction of one partial per lane: every lane ends with
// the warp total (integer parts exact; float pairs combined as double-float
// with TwoSum, in the butterfly's fixed order).
template <int DT>
__device__ __forceinline__ void warp_merge(uint32_t& s, uint64_t& x, uint64_t& n, float& hi, float& lo) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(FULL_MASK, s, o);
        x ^= __shfl_xor_sync(FULL_MASK, x, o);
        n += __shfl_xor_sync(FULL_MASK, n, o);
        if constexpr (DT != SL_U32) {
            const float ohi = __shfl_xor_sync(FULL_MASK, hi, o);
            const float olo = __shfl_xor_sync(FULL_MASK, lo, o);
            df_add(hi, lo, ohi, olo);
        }
    }
}

// Final combine of all CTAs' partials into one sl_result, run by the whole
// CTA that finished last: thread t folds partials t, t+blockDim, ... in index
// order (FP64 for the float part: (double)hi + (double)lo), then the warps
// and the per-warp results are merged by fixed shuffle butterflies, so the
// float sum has a fixed order for a given launch shape.  Integer parts are
// exact.  The device error word becomes the status and is cleared; the CTA
// counter, the chunk counter (if any) and the timing window are reset for the
// next launch.
template <typename T, typename Op>
__device__ __forceinline__ T warp_all(T v, Op op) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(FULL_MASK, v, o));
    return v;
}

// Loops are not unrolled and each field is reduced on its own, so that this
// code needs fewer registers than the streaming loop it follows.
__device__ __forceinline__ void final_combine(const KArgs& a) {
    struct Fin {
        uint32_t sum;
        uint64_t x, n;
        double f;
    };
    __shared__ Fin fw[32];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    const uint32_t n = gridDim.x;
    Fin v{0u, 0ull, 0ull, 0.0};
#pragma unroll 1
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const uint4 lo4 = __ldcg(reinterpret_cast<const uint4*>(a.parts + i));
        const uint4 hi4 = __ldcg(reinterpret_cast<const uint4*>(a.parts + i) + 1);
        v.sum += lo4.x;
        v.x ^= (static_cast<uint64_t>(lo4.w) << 32) | lo4.z;
        v.n += (static_cast<uint64_t>(hi4.y) << 32) | hi4.x;
        v.f += static_cast<double>(__uint_as_float(hi4.z)) + static_cast<double>(__uint_as_float(hi4.w));
    }
    const auto add32 = [](uint32_t p, uint32_t q) { return p + q; };
    const auto add64 = [](uint64_t p, uint64_t q) { return p + q; };
    const auto xor64 = [](uint64_t p, uint64_t q) { return p ^ q; };
    const auto addf = [](double p, double q) { return p + q; };
    for (int pass = 0; pass < 2; ++pass) {  // pass 0: within warps; pass 1: across warps (warp 0)
        v.sum = warp_all(v.sum, add32);
        v.x = warp_all(v.x, xor64);
        v.n = warp_all(v.n, add64);
        v.f = warp_all(v.f, addf);
        if (pass == 1) break;
        if (lane == 0) fw[warp] = v;
        __syncthreads();
        if (warp != 0) return;
        v = lane < nw ? fw[lane] : Fin{0u, 0ull, 0ull, 0.0};
    }
    if (lane == 0) {
        // field by field: a whole sl_result in registers would raise the
        // kernel's register count
        sl_result* r = a.result;
        r->xor_u64 = v.x;
        r->issued_loads = v.n;
        r->device_ns = 0;
        volatile uint64_t* w = a.window;
        const uint64_t t0 = w[0], t1 = w[1];
        r->window_ns = t1 > t0 ? t1 - t0 : 0;
        r->fsum = v.f;
        const float hi = static_cast<float>(v.f);
        r->fsum_hi = hi;
        r->fsum_lo = static_cast<float>(v.f - static_cast<double>(hi));
        r->sum_u32 = v.sum;
        r->status = *reinterpret_cast<volatile uint32_t*>(a.err) ? SL_ERR_TIMEOUT : SL_OK;
        r->grid = 0;
        r->cta = 0;
        r->resident_per_sm = 0;
        r->smem_bytes = 0;
        *a.err = 0;
        *a.done = 0;
        if (a.next) *a.next = 0;
        w[0] = ~0ull;
        w[1] = 0;
    }
}

// This CTA's %globaltimer start, kept in shared memory by cta_start (below)
// and published by cta_finish.
__device__ __forceinline__ uint64_t& cta_start_stamp() {
    __shared__ uint64_t t0;
    return t0;
}

// End of a streaming kernel: every folding warp (all 32 lanes present)
// reduces its accumulators and lane 0 puts the warp partial in shared memory;
// after a CTA barrier warp 0 merges the warp partials (butterfly, fixed
// order) into the CTA's partial a.parts[blockIdx.x], and thread 0 raises the
// launch's end stamp to this CTA's %globaltimer.  With
// a.result set, the last CTA to get here then runs final_combine.  `fw` is
// this warp's index among the nfw (<= 32) folding warps; `cta_err`, if given,
// is a CTA-local error code (shared memory) that thread 0 publishes to *a.err.
template <int DT>
__device__ __forceinline__ void cta_finish(const Acc<DT>& acc, bool folds, uint32_t fw, uint32_t nfw,
                                           const KArgs& a, const uint32_t* cta_err = nullptr) {
    __shared__ WarpPartial sp[32];
    const uint32_t lane = threadIdx.x & 31;
    // A launch that may have started before the previous one finished
    // (programmatic dependent launch) touches the shared scratch (partials,
    // window, CTA counter) only once that launch has completed and its writes
    // are visible; without a prerequisite grid this returns at once.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (folds) {
        uint32_t s = acc.s;
        uint64_t x = (static_cast<uint64_t>(acc.xh) << 32) | acc.xl, n = acc.n;
        float hi = 0.0f, lo = 0.0f;
        if constexpr (DT != SL_U32) acc.float_part(hi, lo);
        warp_merge<DT>(s, x, n, hi, lo);
        if (lane == 0) {
            WarpPartial p;
            p.sum = s;
            p.pad = 0;
            p.xr = x;
            p.issued = n;
            p.hi = hi;
            p.lo = lo;
            sp[fw] = p;
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t s = 0;
        uint64_t x = 0, n = 0;
        float hi = 0.0f, lo = 0.0f;
        if (lane < nfw) {
            const WarpPartial p = sp[lane];
            s = p.sum;
            x = p.xr;
            n = p.issued;
            hi = p.hi;
            lo = p.lo;
        }
        warp_merge<DT>(s, x, n, hi, lo);
        if (lane == 0) {
            WarpPartial p;
            p.sum = s;
            p.pad = 0;
            p.xr = x;
            p.issued = n;
            p.hi = hi;
            p.lo = lo;
            a.parts[blockIdx.x] = p;
            if (cta_err && *cta_err) atomicCAS(a.err, 0u, *cta_err);  // before this CTA is counted done
            atomicMin(reinterpret_cast<unsigned long long*>(a.window), cta_start_stamp());
            atomicMax(reinterpret_cast<unsigned long long*>(a.window + 1), gtimer());
        }
    }
    if (a.result == nullptr) return;
    // Last-CTA-done: publish this CTA's partial, count it, and let the CTA
    // that completes the count combine everything.
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = (atomicAdd(a.done, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        final_combine(a);
    }
}

// Tile cursor over the grid-stride sequence it = blockIdx.x, +gridDim.x, ...
// tm = it mod ntiles (the pass-local tile), tracked without division.  32-bit:
// the host keeps total tiles + grid below 2^32.
struct TileCursor {
    uint32_t it, tm;
    __device__ __forceinline__ void start(uint32_t ntiles) {
        it = blockIdx.x;
        tm = blockIdx.x % ntiles;
    }
    __device__ __forceinline__ void next(uint32_t ntiles) {
        it += gridDim.x;
        tm += gridDim.x;
        while (tm >= ntiles) tm -= ntiles;
    }
    __device__ __forceinline__ uint32_t tile(const KArgs& a) const {
        return a.desc ? (static_cast<uint32_t>(a.ntiles) - 1 - tm) : tm;
    }
};

// Start of a streaming kernel: thread 0 keeps this CTA's %globaltimer start
// in shared memory (no register holds it through the kernel), and the CTA
// lets a programmatically dependent next launch begin (griddepcontrol; a
// no-op unless the next launch asked for programmatic stream serialization).
// Nothing here touches the launch's scratch: that waits for cta_finish.
__device__ __forceinline__ void cta_start(const KArgs&) {
    if (threadIdx.x == 0) cta_start_stamp() = gtimer();
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

}  // namespace sl
