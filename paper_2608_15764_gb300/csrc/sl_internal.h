// sl_internal.h -- definitions shared by the host API and the kernels of the
// streaming-load library (not part of the public ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/streamload.h"

namespace sl {

// One CTA's (or warp's) folded contribution.  The final combine adds sum
// (mod 2^32), XORs xr, adds issued, and adds (double)hi + (double)lo in FP64.
struct __align__(16) WarpPartial {
    uint32_t sum;
    uint32_t pad;
    uint64_t xr;
    uint64_t issued;
    float hi;
    float lo;
};
static_assert(sizeof(WarpPartial) == 32, "WarpPartial layout");

// Arguments of every streaming kernel (passed by value as one struct).
struct KArgs {
    const void* buf;        // device buffer base, 16-byte aligned
    uint64_t nvec;          // 16-byte vectors in the buffer
    uint64_t ntiles;        // tiles per pass
    uint64_t total;         // tiles over all passes = ntiles * passes
    uint32_t tile_vec;      // 16-byte vectors per tile (LDG: cta*K, CPASYNC: cta*D*G,
                            // TMA: stage_bytes/16)
    int32_t desc;           // 1: walk tiles from the last one downward
    int32_t nst;            // TMA: ring stages (per CTA or per warp)
    int32_t debug;          // SL_DEBUG_* flags
    WarpPartial* parts;     // [grid]: one partial per CTA
    uint64_t* window;       // [2]: earliest CTA start, latest CTA end
                            // (%globaltimer; ~0 and 0 before the launch)
    uint32_t* err;          // device error word (0 = fine)
    uint64_t timeout_ns;    // bound of any single device wait
    sl_result* result;      // if set: the last CTA to finish combines all
                            // partials into *result (else a separate combine)
    uint32_t* done;         // CTAs finished (zero before the launch; the last
                            // CTA resets it)
    uint32_t* next;         // SL_DYN traversal: next chunk to claim (zero before
                            // the launch; the last CTA resets it), else NULL
    uint32_t* cov;          // coverage instantiations only: one counter per
                            // 16-byte vector, +1 per load of it; else NULL
};

// Device error codes written to *err (first writer wins).
enum : uint32_t { DEV_ERR_NONE = 0, DEV_ERR_TIMEOUT_FULL = 1, DEV_ERR_TIMEOUT_EMPTY = 2,
                  DEV_ERR_TIMEOUT_DRAIN = 3 };

// Kernel lookup.  Each returns the __global__ function for the given
// instantiation, or nullptr when out of range.  All take (KArgs).
const void* ldg_kernel(int dtype, int k, int cta, int cop);
const void* ldg_dyn_kernel(int dtype, int k, int cta);
const void* cpasync_kernel(int dtype, int d, int g);  // g: copies per commit group
const void* cpasync_dyn_kernel(int dtype, int d, int g);  // SL_DYN traversal
const void* ldsts_kernel(int dtype, int g);
// SL_RING_CTA: batch = vectors a consumer thread reads into registers at a
// time (4, or 1 where a thread reads fewer than 4 vectors of a stage)
const void* tma_kernel(int dtype, int batch);
// SL_RING_WARP: early = refill a stage before folding its last batch
// (instantiated for BF16 payloads; the host takes it where each warp owns a
// single stage)
const void* tma_warp_kernel(int dtype, bool early);
const void* ldg4_kernel(int dtype, int k, int cta);
const void* ldg32_kernel(int dtype, int k, int cta, bool dyn);
const void* ldg_fixed_kernel(int dtype, int k, int cta);

// Coverage instantiations (uint32 payloads, a subset of shapes): the same
// kernels with every load also counted in KArgs::cov.  nullptr when the shape
// has no coverage instantiation.
const void* ldg_cov_kernel(int k, int cta, bool dyn);
const void* ldg32_cov_kernel(int k, int cta, bool dyn);
const void* ldg_fixed_cov_kernel(int k, int cta);
const void* cpasync_cov_kernel(int d, int g);
const void* cpasync_dyn_cov_kernel(int d, int g);
const void* ldsts_cov_kernel(int g);
const void* tma_cov_kernel(int batch);
const void* tma_warp_cov_kernel();

// Two co-resident streams in one CTA (k_two.cu).  Stream A = warps
// [0, warps_a), stream B = the warps_b warps after them; one CTA per SM.
struct TwoArgs {
    const uint4* buf_a;
    const uint4* buf_b;
    uint64_t nvec_a, nvec_b;      // 16-byte vectors per pass
    uint32_t ntiles_a, ntiles_b;  // tiles per pass (stream threads * K vectors each)
    uint32_t total_a, total_b;    // tiles over all passes
    uint32_t warps_a, warps_b;
    WarpPartial* parts;           // [grid * 32]: one partial per warp slot
    uint64_t* ctl;                // TWO_CTL_WORDS %globaltimer words, set by the host before the launch
};
// Timer words: earliest warp start of A and B (min; ~0 before), latest warp
// end of A and B (max; 0 before), earliest warp end of B (min; ~0 before).
enum : int { TWO_START = 0, TWO_END = 2, TWO_FIRST_END_B = 4, TWO_CTL_WORDS = 5 };
const void* two_kernel(int k);
cudaError_t launch_two(const TwoArgs& t, int k, uint32_t grid, cudaStream_t s);
// out[0..2] = A {sum, xor, issued}, out[3..5] = B, out[6..10] = timer words.
cudaError_t launch_two_combine(const TwoArgs& t, uint32_t grid, uint64_t* out, cudaStream_t s);

// Pointer chase (k_chase.cu): out[4] = final index, ns, cycles, out-of-range flag.
cudaError_t launch_chase(const uint32_t* chain, uint64_t nwords, uint32_t start, uint64_t warm, uint64_t hops,
                         int ca, uint64_t* out, cudaStream_t s);

// Record a failure message for sl_last_error(); returns code (api.cu).
int set_error(int code, const char* msg);

// Utility launches (k_util.cu); asynchronous on `s`.
cudaError_t launch_fill_splitmix64(void* buf, uint64_t nvec, uint64_t seed, int sms, cudaStream_t s);
cudaError_t launch_flush(void* buf, uint64_t nvec, int sms, cudaStream_t s);
cudaError_t launch_combine(const WarpPartial* parts, uint64_t nparts, uint64_t* window, uint32_t* err,
                           sl_result* out, cudaStream_t s);

// Layout of the 256-byte control block shared by a launch and its combine:
// error word at byte 0, finished-CTA counter at byte 64, window at byte 128,
// chunk counter of the SL_DYN traversal at byte 192.
constexpr int CTRL_BYTES = 256;
inline uint32_t* ctrl_err(void* c) { return static_cast<uint32_t*>(c); }
inline uint32_t* ctrl_done(void* c) { return static_cast<uint32_t*>(c) + 16; }
inline uint64_t* ctrl_window(void* c) { return static_cast<uint64_t*>(c) + 16; }
inline uint32_t* ctrl_next(void* c) { return static_cast<uint32_t*>(c) + 48; }

}  // namespace sl
