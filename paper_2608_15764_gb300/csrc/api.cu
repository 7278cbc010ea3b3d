// api.cu -- host implementation of the C ABI declared in include/streamload.h.
//
// Validation, launch planning (occupancy and shared-memory feasibility),
// per-device scratch, CUDA-event timing, sweeps and the host-buffer pipeline.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <vector>
#include <mutex>
#include <tuple>

#include "sl_internal.h"

namespace sl {
const void* ldg_kernel_u32(int k, int cta, int cop);
const void* ldg_kernel_f32(int k, int cta, int cop);
const void* ldg_kernel_bf16(int k, int cta, int cop);
const void* ldg_kernel_fp8(int k, int cta, int cop);

const void* ldg_kernel(int dtype, int k, int cta, int cop) {
    switch (dtype) {
    case SL_U32: return ldg_kernel_u32(k, cta, cop);
    case SL_F32: return ldg_kernel_f32(k, cta, cop);
    case SL_BF16: return ldg_kernel_bf16(k, cta, cop);
    case SL_FP8_E4M3: return ldg_kernel_fp8(k, cta, cop);
    default: return nullptr;
    }
}
}  // namespace sl

namespace {

using sl::KArgs;
using sl::WarpPartial;

constexpr int MAX_DEVICES = 64;
constexpr uint64_t HOST_CHUNK = 256ull << 20;     // sl_run_host staging chunk
constexpr uint64_t TIMEOUT_NS = 2000000000ull;     // per-wait bound, normal runs
constexpr uint64_t DEBUG_TIMEOUT_NS = 50000000ull;  // per-wait bound, fault-injection runs
constexpr int64_t MAX_GRID = 1 << 20;
constexpr uint64_t DYN_CHUNK_VEC = 65536;          // SL_DYN chunk: 1 MiB of 16-byte vectors
constexpr int32_t STEP_COUNTERS = 4096;            // sl_enqueue_steps: SL_DYN passes per counter segment

thread_local char g_err[1024] = "";

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

// On failure: record the message, clear the runtime's last-error state (so a
// later launch check does not report this error again) and return the status.
#define CUDA_TRY(expr)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            (void)cudaGetLastError();                                                         \
            return fail(e_ == cudaErrorMemoryAllocation ? SL_ERR_OOM : SL_ERR_CUDA,           \
                        "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__,     \
                        __LINE__);                                                            \
        }                                                                                     \
    } while (0)

struct FuncInfo {
    int max_threads = 0;
    size_t local_bytes = 0;  // per-thread local memory (register spills)
    int regs = 0;            // registers per thread
    size_t smem_attr = 0;  // dynamic shared memory limit already set
};

struct DevCtx {
    bool ready = false;
    int dev = -1;
    sl_devinfo info{};
    WarpPartial* parts = nullptr;
    uint64_t parts_cap = 0;
    uint32_t* err = nullptr;    // control block (sl::CTRL_BYTES): error word, CTA counter, window
    sl_result* dres = nullptr;  // device result of sl_run / sl_run_host
    sl_result* hres = nullptr;  // pinned host copy
    uint64_t* two_dev = nullptr;   // sl_twostream: timer words [0, 8) and results [8, 24)
    uint64_t* two_host = nullptr;  // pinned copy of the results
    uint32_t* step_next = nullptr; // sl_enqueue_steps with SL_DYN: one chunk counter per pass
    void* flush = nullptr;
    uint64_t flush_bytes = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    void* stage[2] = {nullptr, nullptr};
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr}, consumed[2] = {nullptr, nullptr};
    std::map<const void*, FuncInfo> funcs;
    std::map<std::tuple<const void*, int, size_t>, int> occupancy;
    std::recursive_mutex mu;
};

DevCtx g_ctx[MAX_DEVICES];
std::mutex g_init_mu;

int query_info(int dev, sl_devinfo* out) {
    cudaDeviceProp p;
    CUDA_TRY(cudaGetDeviceProperties(&p, dev));
    std::memset(out, 0, sizeof *out);
    out->device = dev;
    out->sm_count = p.multiProcessorCount;
    out->cc_major = p.major;
    out->cc_minor = p.minor;
    out->l2_bytes = p.l2CacheSize;
    out->smem_per_block_optin = static_cast<int64_t>(p.sharedMemPerBlockOptin);
    out->smem_per_sm = static_cast<int64_t>(p.sharedMemPerMultiprocessor);
    out->global_mem_bytes = static_cast<int64_t>(p.totalGlobalMem);
    out->max_threads_per_sm = p.maxThreadsPerMultiProcessor;
    out->regs_per_sm = p.regsPerMultiprocessor;
    int v = 0;
    out->clock_khz = cudaDeviceGetAttribute(&v, cudaDevAttrClockRate, dev) == cudaSuccess ? v : 0;
    v = 0;
    out->mem_clock_khz = cudaDeviceGetAttribute(&v, cudaDevAttrMemoryClockRate, dev) == cudaSuccess ? v : 0;
    v = 0;
    out->mem_bus_bits = cudaDeviceGetAttribute(&v, cudaDevAttrGlobalMemoryBusWidth, dev) == cudaSuccess ? v : 0;
    (void)cudaGetLastError();
    cudaDriverGetVersion(&out->driver_version);
    cudaRuntimeGetVersion(&out->runtime_version);
    std::snprintf(out->name, sizeof out->name, "%s", p.name);
    return SL_OK;
}

// The context of the current device, initialised on first use.
int get_ctx(DevCtx** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(SL_ERR_NODEV, "no CUDA device: %s", cudaGetErrorString(e));
    }
    if (dev < 0 || dev >= MAX_DEVICES) return fail(SL_ERR_NODEV, "device index %d out of range", dev);
    DevCtx* c = &g_ctx[dev];
    std::lock_guard<std::mutex> g(g_init_mu);
    if (!c->ready) {
        c->dev = dev;
        int rc = query_info(dev, &c->info);
        if (rc) return rc;
        CUDA_TRY(cudaMalloc(&c->err, sl::CTRL_BYTES));
        CUDA_TRY(cudaMemset(c->err, 0, sl::CTRL_BYTES));
        CUDA_TRY(cudaMemset(sl::ctrl_window(c->err), 0xFF, sizeof(uint64_t)));  // earliest start = ~0
        CUDA_TRY(cudaMalloc(&c->dres, sizeof(sl_result)));
        CUDA_TRY(cudaMallocHost(&c->hres, sizeof(sl_result)));
        CUDA_TRY(cudaEventCreate(&c->ev0));
        CUDA_TRY(cudaEventCreate(&c->ev1));
        c->flush_bytes = ((2 * static_cast<uint64_t>(c->info.l2_bytes)) + (1u << 20) - 1) & ~((1ull << 20) - 1);
        if (c->flush_bytes < (64ull << 20)) c->flush_bytes = 64ull << 20;
        CUDA_TRY(cudaMalloc(&c->flush, c->flush_bytes));
        CUDA_TRY(cudaDeviceSynchronize());
        c->ready = true;
    }
    *out = c;
    return SL_OK;
}

// Grow the per-CTA partial scratch.  Growing waits for the device to go idle
// first, since enqueued work may still use the old buffer.
int ensure_scratch(DevCtx* c, uint64_t nparts) {
    if (nparts > c->parts_cap) {
        uint64_t cap = std::max<uint64_t>(nparts, 1 << 16);
        CUDA_TRY(cudaDeviceSynchronize());
        if (c->parts) CUDA_TRY(cudaFree(c->parts));
        c->parts = nullptr;
        c->parts_cap = 0;
        CUDA_TRY(cudaMalloc(&c->parts, cap * sizeof(WarpPartial)));
        c->parts_cap = cap;
    }
    return SL_OK;
}

struct Plan {
    const void* fn = nullptr;
    int block = 0;            // threads per CTA launched
    int64_t grid = 0;         // CTAs (0: nothing to launch)
    size_t smem = 0;          // dynamic shared memory
    int resident = 0;         // occupancy-API CTAs per SM
    uint64_t warps = 0;       // folding warps per CTA (each CTA writes one partial)
    KArgs args{};
};

int func_info(DevCtx* c, const void* fn, size_t smem, FuncInfo** out) {
    FuncInfo& fi = c->funcs[fn];
    if (fi.max_threads == 0) {
        cudaFuncAttributes fa;
        CUDA_TRY(cudaFuncGetAttributes(&fa, fn));
        fi.max_threads = fa.maxThreadsPerBlock;
        fi.local_bytes = fa.localSizeBytes;
        fi.regs = fa.numRegs;
    }
    if (smem > 0 && fi.smem_attr < smem) {  // static smem counts too: opt in for any dynamic size
        CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
        fi.smem_attr = smem;
    }
    *out = &fi;
    return SL_OK;
}

int occupancy(DevCtx* c, const void* fn, int block, size_t smem, int* out) {
    auto key = std::make_tuple(fn, block, smem);
    auto it = c->occupancy.find(key);
    if (it != c->occupancy.end()) {
        *out = it->second;
        return SL_OK;
    }
    int n = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, block, smem));
    c->occupancy[key] = n;
    *out = n;
    return SL_OK;
}

// G, the 16-byte copies per commit group of SL_CPASYNC (0 in the config means 1).
int copies_per_group(const sl_config* cfg) { return cfg->copies == 0 ? 1 : cfg->copies; }

// SL_RING_CTA: vectors a consumer thread reads into registers before folding
// them.  4 where each of the cta consumer threads reads at least 4 vectors of
// a stage; 1 below that, where the registers of a larger batch would cost
// CTAs per SM (measured: 4 KiB stages read by 128 or 256 threads).
int tma_batch(const sl_config* cfg) { return cfg->stage_bytes / 16 >= 4 * cfg->cta ? 4 : 1; }

int make_plan(DevCtx* c, const void* buf, uint64_t bytes, int32_t dtype, const sl_config* cfg, Plan* p) {
    if (!cfg) return fail(SL_ERR_ARG, "cfg is NULL");
    if (dtype < SL_U32 || dtype > SL_FP8_E4M3) return fail(SL_ERR_ARG, "bad dtype %d", dtype);
    if ((bytes & 15u) != 0) return fail(SL_ERR_ALIGN, "bytes (%llu) not a multiple of 16", (unsigned long long)bytes);
    if (bytes > 0 && !buf) return fail(SL_ERR_ARG, "buffer is NULL");
    if ((reinterpret_cast<uintptr_t>(buf) & 15u) != 0) return fail(SL_ERR_ALIGN, "buffer not 16-byte aligned");
    if (cfg->passes < 0) return fail(SL_ERR_ARG, "passes %d < 0", cfg->passes);
    if (cfg->order != SL_ASC && cfg->order != SL_DESC && cfg->order != SL_DYN)
        return fail(SL_ERR_ARG, "bad order %d", cfg->order);
    if (cfg->mech != SL_CPASYNC && cfg->copies != 0 && cfg->copies != 1)
        return fail(SL_ERR_ARG, "copies per commit group (%d) applies to SL_CPASYNC only", cfg->copies);
    const bool dyn = cfg->order == SL_DYN;
    const bool fixed = cfg->target_loads > 0;
    if (fixed && cfg->mech != SL_LDG) return fail(SL_ERR_ARG, "the fixed-iteration control is implemented for SL_LDG");
    if (dyn && ((cfg->mech != SL_LDG && cfg->mech != SL_LDG32 && cfg->mech != SL_CPASYNC) || cfg->cop != SL_COP_CG))
        return fail(SL_ERR_ARG, "the SL_DYN traversal is implemented for SL_LDG / SL_LDG32 / SL_CPASYNC with SL_COP_CG");
    const uint64_t passes = cfg->passes == 0 ? 1 : static_cast<uint64_t>(cfg->passes);
    const int cta = cfg->cta;
    if (cta < 32 || cta > 1024 || (cta & 31)) return fail(SL_ERR_ARG, "cta %d not a multiple of 32 in 32..1024", cta);

    uint64_t tile_vec = 0;
    *p = Plan{};
    switch (cfg->mech) {
    case SL_LDG:
        if (cfg->k < 1 || cfg->k > SL_MAX_K) return fail(SL_ERR_ARG, "LDG K %d not in 1..%d", cfg->k, SL_MAX_K);
        if (cfg->cop < SL_COP_CG || cfg->cop > SL_COP_NC_NA_L2_256) return fail(SL_ERR_ARG, "bad cop %d", cfg->cop);
        if (fixed) {
            if (dyn || cfg->cop != SL_COP_CG || dtype != SL_U32 || cfg->passes > 1)
                return fail(SL_ERR_ARG, "the fixed-iteration control takes SL_ASC / SL_DESC, SL_COP_CG, uint32 "
                            "payloads and passes <= 1");
            p->fn = sl::ldg_fixed_kernel(dtype, cfg->k, cta);
            if (!p->fn)
                return fail(SL_ERR_ARG, "no fixed-iteration LDG kernel for K %d, cta %d (K in {1,2,3,4,6,8,12,16}, "
                            "cta 256/512/1024)", cfg->k, cta);
            if (bytes / 16 < static_cast<uint64_t>(cta) * cfg->k)
                return fail(SL_ERR_ARG, "the fixed-iteration control needs a buffer of at least one tile "
                            "(%d x %d vectors)", cta, cfg->k);
            p->block = cta;
            p->smem = 0;
            tile_vec = static_cast<uint64_t>(cta) * cfg->k;
            p->warps = cta / 32;
            break;
        }
        p->fn = dyn ? sl::ldg_dyn_kernel(dtype, cfg->k, cta) : sl::ldg_kernel(dtype, cfg->k, cta, cfg->cop);
        if (!p->fn && dyn)
            return fail(SL_ERR_ARG, "no SL_DYN LDG kernel for K %d, cta %d (K in {1,2,3,4,6,8,12,16}, "
                        "cta 128/256/512)", cfg->k, cta);
        if (!p->fn)
            return fail(SL_ERR_ARG, "no LDG kernel for dtype %d, K %d, cta %d, cop %d (cta must be 32/128/256/512/1024 "
                        "for uint32, 128/256/512 for floats; cop 2 is uint32 only)", dtype, cfg->k, cta, cfg->cop);
        p->block = cta;
        p->smem = 0;
        tile_vec = static_cast<uint64_t>(cta) * cfg->k;
        if (dyn) tile_vec *= std::max<uint64_t>(1, DYN_CHUNK_VEC / tile_vec);  // chunk of ~1 MiB
        p->warps = cta / 32;
        break;
    case SL_LDG4:
        if (dtype != SL_U32) return fail(SL_ERR_ARG, "SL_LDG4 reads uint32 payloads only");
        if (cfg->cop != SL_COP_CG) return fail(SL_ERR_ARG, "SL_LDG4 has the SL_COP_CG flavour only");
        p->fn = sl::ldg4_kernel(dtype, cfg->k, cta);
        if (!p->fn)
            return fail(SL_ERR_ARG, "no 4-byte LDG kernel for K %d, cta %d (K in {1,2,4,8,16}, cta 128/256/512/1024)",
                        cfg->k, cta);
        p->block = cta;
        p->smem = 0;
        tile_vec = static_cast<uint64_t>(cta) * cfg->k;  // in 4-byte words
        p->warps = cta / 32;
        break;
    case SL_LDG32:
        if ((reinterpret_cast<uintptr_t>(buf) & 31u) != 0)
            return fail(SL_ERR_ALIGN, "SL_LDG32 needs a 32-byte aligned buffer");
        if (cfg->cop != SL_COP_CG) return fail(SL_ERR_ARG, "SL_LDG32 has the SL_COP_CG flavour only");
        p->fn = sl::ldg32_kernel(dtype, cfg->k, cta, dyn);
        if (!p->fn)
            return fail(SL_ERR_ARG, "no 32-byte LDG kernel for K %d, cta %d (K in {1,2,3,4,6,8}, cta 128/256/512)",
                        cfg->k, cta);
        p->block = cta;
        p->smem = 0;
        tile_vec = static_cast<uint64_t>(cta) * cfg->k;  // in 32-byte units
        if (dyn) tile_vec *= std::max<uint64_t>(1, (DYN_CHUNK_VEC / 2) / tile_vec);
        p->warps = cta / 32;
        break;
    case SL_CPASYNC:
    case SL_LDSTS: {
        if (cfg->k < 1 || cfg->k > SL_MAX_D)
            return fail(SL_ERR_ARG, "%s depth %d not in 1..%d", cfg->mech == SL_CPASYNC ? "cp.async" : "ld/st.shared",
                        cfg->k, SL_MAX_D);
        const int g = copies_per_group(cfg);
        if (g != 1 && g != 2 && g != 4 && g != 8)
            return fail(SL_ERR_ARG, "cp.async copies per commit group %d not in {1, 2, 4, 8}", g);
        if (cfg->k * g > SL_MAX_D)
            return fail(SL_ERR_ARG, "cp.async D x G = %d x %d copies in flight exceeds %d", cfg->k, g, SL_MAX_D);
        if (cfg->mech == SL_CPASYNC && dyn) {
            p->fn = sl::cpasync_dyn_kernel(dtype, cfg->k, g);
            if (!p->fn)
                return fail(SL_ERR_ARG, "no SL_DYN cp.async kernel for D %d x G %d (D 1/2/3/4/6/8 with one copy per "
                            "group; D x G 2 x 2, 1 x 4, 2 x 4, 1 x 8, 2 x 8)", cfg->k, g);
        } else {
            p->fn = cfg->mech == SL_CPASYNC ? sl::cpasync_kernel(dtype, cfg->k, g) : sl::ldsts_kernel(dtype, cfg->k);
        }
        p->block = cta;
        p->smem = static_cast<size_t>(cfg->k) * g * cta * 16 +
                  (((cfg->debug_flags >> SL_DEBUG_SMEM_SKEW_SHIFT) & 7) ? 128 : 0);  // room for a skewed ring
        tile_vec = static_cast<uint64_t>(cta) * cfg->k * g;
        if (dyn) tile_vec *= std::max<uint64_t>(1, DYN_CHUNK_VEC / tile_vec);  // chunk of ~1 MiB
        p->warps = cta / 32;
        break;
    }
    case SL_TMA:
        if (cfg->stage_bytes != 4096 && cfg->stage_bytes != 16384 && cfg->stage_bytes != 65536)
            return fail(SL_ERR_INFEASIBLE, "TMA stage size %d not 4096/16384/65536", cfg->stage_bytes);
        if (cfg->stages < SL_MIN_STAGES || cfg->stages > SL_MAX_STAGES)
            return fail(SL_ERR_ARG, "TMA stages %d not in %d..%d", cfg->stages, SL_MIN_STAGES, SL_MAX_STAGES);
        if (cfg->tma_ring == SL_RING_WARP) {
            // the CTA's stages dealt to its warps, each filled by its warp's
            // own lane 0; the full barriers follow the stages in dynamic
            // shared memory
            if (cfg->stages % (cta / 32) != 0)
                return fail(SL_ERR_ARG, "SL_RING_WARP deals the %d stages to %d warps: the warp count must divide "
                            "the stage count", cfg->stages, cta / 32);
            p->fn = sl::tma_warp_kernel(dtype, dtype == SL_BF16 && cfg->stages == cta / 32);
            p->block = cta;
            p->smem = static_cast<size_t>(cfg->stages) * (static_cast<size_t>(cfg->stage_bytes) + 8);
        } else if (cfg->tma_ring == SL_RING_CTA) {
            if (cta > 992) return fail(SL_ERR_ARG, "TMA consumer threads %d > 992", cta);
            p->fn = sl::tma_kernel(dtype, tma_batch(cfg));
            p->block = cta + 32;
            p->smem = static_cast<size_t>(cfg->stages) * cfg->stage_bytes;
        } else {
            return fail(SL_ERR_ARG, "bad tma_ring %d", cfg->tma_ring);
        }
        tile_vec = static_cast<uint64_t>(cfg->stage_bytes) / 16;
        p->warps = cta / 32;
        break;
    default:
        return fail(SL_ERR_ARG, "bad mech %d", cfg->mech);
    }
    if (!p->fn) return fail(SL_ERR_ARG, "no kernel instantiated for this configuration");
    if (p->smem > static_cast<size_t>(c->info.smem_per_block_optin))
        return fail(SL_ERR_INFEASIBLE, "%zu bytes of shared memory exceed the %lld-byte per-block limit", p->smem,
                    (long long)c->info.smem_per_block_optin);
    FuncInfo* fi = nullptr;
    int rc = func_info(c, p->fn, p->smem, &fi);
    if (rc) return rc;
    if (fi->local_bytes > 0)
        return fail(SL_ERR_INFEASIBLE, "this kernel spills registers (%zu bytes of local memory per thread)",
                    fi->local_bytes);
    // K in-flight 16-byte loads need 4K registers.  Where the CTA size caps
    // registers below that (CTA 1024 with large K), the compiler interleaves
    // loads with folds and K would no longer be the offered ILP.
    // (the fixed-iteration kernel keeps fewer values live besides the loaded
    // vectors: its floor is K vectors + pointer, tile start and checksum)
    if ((cfg->mech == SL_LDG || cfg->mech == SL_LDSTS) && fi->regs < 4 * cfg->k + (fixed ? 8 : 16))
        return fail(SL_ERR_INFEASIBLE, "%d registers per thread cannot hold K=%d loads in flight at cta %d",
                    fi->regs, cfg->k, cta);
    if (cfg->mech == SL_LDG32 && fi->regs < 8 * cfg->k + 16)
        return fail(SL_ERR_INFEASIBLE, "%d registers per thread cannot hold K=%d 32-byte loads in flight at cta %d",
                    fi->regs, cfg->k, cta);
    if (cfg->mech == SL_LDG4 && fi->regs < cfg->k + 16)
        return fail(SL_ERR_INFEASIBLE, "%d registers per thread cannot hold K=%d 4-byte loads in flight at cta %d",
                    fi->regs, cfg->k, cta);
    if (p->block > fi->max_threads)
        return fail(SL_ERR_INFEASIBLE, "%d threads per CTA exceed this kernel's limit of %d", p->block,
                    fi->max_threads);
    rc = occupancy(c, p->fn, p->block, p->smem, &p->resident);
    if (rc) return rc;
    if (p->resident < 1) return fail(SL_ERR_INFEASIBLE, "configuration has zero occupancy");

    // nvec: 16-byte vectors (4-byte words for SL_LDG4); units: what a tile counts
    // (SL_LDG32: 32-byte units, a final half unit included)
    const uint64_t nvec = bytes / (cfg->mech == SL_LDG4 ? 4 : 16);
    const uint64_t units = cfg->mech == SL_LDG32 ? (nvec + 1) / 2 : nvec;
    int64_t grid = cfg->grid;
    if (grid <= 0) grid = static_cast<int64_t>(std::min(4, p->resident)) * c->info.sm_count;
    if (grid > MAX_GRID) return fail(SL_ERR_ARG, "grid %lld > %lld", (long long)grid, (long long)MAX_GRID);
    // fixed-iteration control: iters tiles per CTA, all grid*iters tiles wrap
    // around the buffer; otherwise the tiles that cover the buffer once
    const uint64_t fixed_iters = fixed ? cfg->target_loads / (static_cast<uint64_t>(grid) * tile_vec) : 0;
    const uint64_t ntiles = fixed ? fixed_iters * static_cast<uint64_t>(grid) : (units + tile_vec - 1) / tile_vec;
    p->grid = (nvec == 0 || (fixed && fixed_iters == 0)) ? 0 : grid;
    // The kernels count tiles and per-thread loads in 32 bits (the per-warp
    // TMA ring's chunk index runs up to total + stages * grid).
    const uint64_t total = ntiles * passes;
    const uint64_t per_thread = ((total + grid - 1) / grid) * ((tile_vec + cta - 1) / cta);
    // (SL_DYN counters run up to three claims per CTA past the last chunk)
    const uint64_t ahead = static_cast<uint64_t>(grid) *
                           ((cfg->mech == SL_TMA && cfg->tma_ring == SL_RING_WARP) ? cfg->stages : dyn ? 3 : 1);
    if (total + ahead >= (1ull << 32) || per_thread >= (1ull << 32))
        return fail(SL_ERR_ARG, "passes x tiles too large for one launch (%llu tiles); lower passes",
                    (unsigned long long)total);
    KArgs& a = p->args;
    a.buf = buf;
    a.nvec = nvec;
    a.ntiles = ntiles;
    a.total = ntiles * passes;
    a.tile_vec = static_cast<uint32_t>(tile_vec);
    a.desc = cfg->order == SL_DESC ? 1 : 0;
    a.next = nullptr;  // set by the caller for SL_DYN
    a.nst = cfg->mech == SL_TMA ? cfg->stages : 0;
    a.debug = cfg->debug_flags;
    a.timeout_ns = (cfg->debug_flags & SL_DEBUG_TMA_SKIP_STAGE) ? DEBUG_TIMEOUT_NS : TIMEOUT_NS;
    return SL_OK;
}

int launch(const Plan& p, cudaStream_t s, bool programmatic = false) {
    if (p.grid == 0) return SL_OK;
    KArgs a = p.args;
    void* args[] = {&a};
    if (!programmatic) {
        CUDA_TRY(cudaLaunchKernel(p.fn, dim3(static_cast<unsigned>(p.grid)), dim3(p.block), args, p.smem, s));
        return SL_OK;
    }
    // programmatic dependent launch: may begin once every CTA of the previous
    // kernel on the stream has executed griddepcontrol.launch_dependents
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t lc{};
    lc.gridDim = dim3(static_cast<unsigned>(p.grid));
    lc.blockDim = dim3(p.block);
    lc.dynamicSmemBytes = p.smem;
    lc.stream = s;
    lc.attrs = attr;
    lc.numAttrs = 1;
    CUDA_TRY(cudaLaunchKernelExC(&lc, p.fn, args));
    return SL_OK;
}

void fill_shape(const Plan& p, sl_result* r) {
    r->grid = static_cast<int32_t>(p.grid);
    r->cta = p.block;
    r->resident_per_sm = p.resident;
    r->smem_bytes = static_cast<int32_t>(p.smem);
}

// Enqueue [flush], events, the load kernel and the combine on stream s.
// The coverage instantiation matching cfg's kernel, or nullptr.
const void* coverage_fn(const sl_config* cfg) {
    const bool dyn = cfg->order == SL_DYN;
    switch (cfg->mech) {
    case SL_LDG:
        if (cfg->target_loads) return sl::ldg_fixed_cov_kernel(cfg->k, cfg->cta);
        return cfg->cop == SL_COP_CG ? sl::ldg_cov_kernel(cfg->k, cfg->cta, dyn) : nullptr;
    case SL_LDG32: return sl::ldg32_cov_kernel(cfg->k, cfg->cta, dyn);
    case SL_CPASYNC:
        return dyn ? sl::cpasync_dyn_cov_kernel(cfg->k, copies_per_group(cfg))
                   : sl::cpasync_cov_kernel(cfg->k, copies_per_group(cfg));
    case SL_LDSTS: return sl::ldsts_cov_kernel(cfg->k);
    case SL_TMA: return cfg->tma_ring == SL_RING_WARP ? sl::tma_warp_cov_kernel() : sl::tma_cov_kernel(tma_batch(cfg));
    default: return nullptr;
    }
}

int enqueue_locked(DevCtx* c, const void* buf, uint64_t bytes, int32_t dtype, const sl_config* cfg,
                   sl_result* dev_out, bool events, Plan* plan_out, uint32_t* cov = nullptr) {
    Plan p;
    int rc = make_plan(c, buf, bytes, dtype, cfg, &p);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cfg->stream);
    if (cov) {
        // coverage audit: the same launch shape with the counting instantiation
        const void* fn = dtype == SL_U32 ? coverage_fn(cfg) : nullptr;
        if (!fn)
            return fail(SL_ERR_ARG, "no coverage instantiation for this configuration (uint32; LDG K 1/3/8/16 "
                        "grid-stride or 2/12 SL_DYN at cta 128/256/512; SL_LDG32 K 1/3/8 at cta 256; "
                        "fixed-iteration K 2/8 at cta 256/1024; cp.async D 1/4/16, D x G 2 x 4 and 3 x 2, SL_DYN D 4 and 2 x 4; "
                        "SL_LDSTS G 1/16; TMA)");
        FuncInfo* fi = nullptr;
        rc = func_info(c, fn, p.smem, &fi);
        if (rc) return rc;
        if (fi->local_bytes > 0 || p.block > fi->max_threads)
            return fail(SL_ERR_INFEASIBLE, "the coverage instantiation does not fit this launch shape");
        int res = 0;
        rc = occupancy(c, fn, p.block, p.smem, &res);
        if (rc) return rc;
        if (res < 1) return fail(SL_ERR_INFEASIBLE, "the coverage instantiation has zero occupancy");
        p.fn = fn;
        p.args.cov = cov;
        CUDA_TRY(cudaMemsetAsync(cov, 0, (bytes / 16) * sizeof(uint32_t), s));
    }
    rc = ensure_scratch(c, static_cast<uint64_t>(p.grid));
    if (rc) return rc;
    p.args.parts = c->parts;
    p.args.window = sl::ctrl_window(c->err);
    p.args.err = sl::ctrl_err(c->err);
    p.args.done = sl::ctrl_done(c->err);
    p.args.result = dev_out;  // the kernel's last CTA writes the result
    if (cfg->order == SL_DYN) p.args.next = sl::ctrl_next(c->err);
    if (cfg->flush_l2) CUDA_TRY(sl::launch_flush(c->flush, c->flush_bytes / 16, c->info.sm_count, s));
    if (events) CUDA_TRY(cudaEventRecord(c->ev0, s));
    rc = launch(p, s);
    if (rc) return rc;
    if (events) CUDA_TRY(cudaEventRecord(c->ev1, s));
    if (p.grid == 0)  // empty buffer: no load kernel, the combine writes the zero result
        CUDA_TRY(sl::launch_combine(c->parts, 0, sl::ctrl_window(c->err), c->err, dev_out, s));
    if (plan_out) *plan_out = p;
    return SL_OK;
}

int run_locked(DevCtx* c, const void* buf, uint64_t bytes, int32_t dtype, const sl_config* cfg, sl_result* out,
               uint32_t* cov = nullptr) {
    Plan p;
    int rc = enqueue_locked(c, buf, bytes, dtype, cfg, c->dres, true, &p, cov);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cfg->stream);
    CUDA_TRY(cudaMemcpyAsync(c->hres, c->dres, sizeof(sl_result), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    float ms = 0.0f;
    CUDA_TRY(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    *out = *c->hres;
    out->device_ns = static_cast<uint64_t>(static_cast<double>(ms) * 1e6 + 0.5);
    fill_shape(p, out);
    if (out->status != SL_OK) return fail(out->status, "a bounded device wait timed out");
    return SL_OK;
}

}  // namespace

namespace sl {
// Record a failure for sl_last_error() from another translation unit.
int set_error(int code, const char* msg) { return fail(code, "%s", msg); }
}  // namespace sl

extern "C" {

const char* sl_last_error(void) { return g_err; }

int sl_device_info(sl_devinfo* out) {
    if (!out) return fail(SL_ERR_ARG, "out is NULL");
    DevCtx* c = nullptr;
    int rc = get_ctx(&c);
    if (rc) return rc;
    *out = c->info;
    return SL_OK;
}

int sl_fill_splitmix64(void* dev_buf, uint64_t bytes, uint64_t seed, void* stream) {
    if ((bytes & 15u) != 0 || (reinterpret_cast<uintptr_t>(dev_buf) & 15u) != 0)
        return fail(SL_ERR_ALIGN, "fill needs a 16-byte aligned buffer and a multiple of 16 bytes");
    if (bytes > 0 && !dev_buf) return fail(SL_ERR_ARG, "buffer is NULL");
    DevCtx* c = nullptr;
    int rc = get_ctx(&c);
    if (rc) return rc;
    CUDA_TRY(sl::launch_fill_splitmix64(dev_buf, bytes / 16, seed, c->info.sm_count, static_cast<cudaStream_t>(stream)));
    return SL_OK;
}

int sl_flush_l2(void* stream) {
    DevCtx* c = nullptr;
    int rc = get_ctx(&c);
    if (rc) return rc;
    CUDA_TRY(sl::launch_flush(c->flush, c->flush_bytes / 16, c->info.sm_count, static_cast<cudaStream_t>(stream)));
    return SL_OK;
}

int sl_plan(uint64_t bytes, int32_t dtype, const sl_config* cfg, sl_result* out) {
    if (!out) return fail(SL_ERR_ARG, "out is NULL");
    DevCtx* c = nullptr;
    int rc = get_ctx(&c);
    if (rc) return rc;
    std::lock_guard<std::recursive_mutex> g(c->mu);
    Plan p;
    // a dummy aligned address: planning never dereferences the buffer
    rc = make_plan(c, reinterpret_cast<const void*>(uintptr_t(256)), bytes, dtype, cfg, &p);
    std::memset(out, 0, sizeof *out);
    if (rc) {
        out->status = rc;
        return rc;
    }
    fill_shape(p, out);
    if (p.grid == 0) {
        // empty buffer: report the shape a non-empty one would get
        int64_t grid = cfg->grid > 0 ? cfg->grid : static_cast<int64_t>(std::min(4, p.resident)) * c->info.sm_count;
        out->grid = static_cast<int32_t>(grid);
    }
    return SL_OK;
}

int sl_run(const void* dev_buf, uint64_t bytes, int32_t dtype, const sl_config* cfg, sl_result* out) {
    if (!out) return fail(SL_ERR_ARG, "out is NULL");
    DevCtx* c = nullptr;
    int rc = get_ctx(&c);
    if (rc) return rc;
    std::lock_guard<std::recursive_mutex> g(c->mu);
    return run_locked(c, dev_buf, bytes, dtype, cfg, out);
}

int sl_enqueue(const void* dev_buf, uint64_t bytes, int32_t dtype, const sl_config* cfg, sl_result* dev_out) {
    if (!dev_out || (reinterpret_cast<uintptr_t>(dev_out) & 7u)) return fail(SL_ERR_ARG, "dev_out NULL or misaligned");
    DevCtx* c = nullptr;
    int rc = get_ctx(&c);
    if (rc) return rc;
    std::lock_guard<std::recursive_mutex> g(c->mu);
    return enqueue_locked(c, dev_buf, bytes, dtype, cfg, dev_out, false, nullptr);
}

int sl_coverage(const void* dev_buf, uint64_t bytes, const sl_config* cfg, uint32_t* dev_counts, sl_result* out) {
    if (!out || !cfg) return fail(SL_ERR_ARG, "NULL argument");
    if (!dev_counts || (reinterpret_cast<uintptr_t>(dev_counts) & 3u))
        return fail(SL_ERR_ARG, "dev_counts NULL or not 4-byte aligned");
    if (cfg->mech == SL_LDG4) return fail(SL_ERR_ARG, "no coverage instantiation for SL_LDG4");
    DevCtx* c = nullptr;
    int rc = get_ctx(&c);
    if (rc) return rc;
    std::lock_guard<std::recursive_mutex> g(c->mu);
    return run_locked(c, dev_buf, bytes, SL_U32, cfg, out, dev_counts);
}

int sl_enqueue_steps(const void* const* dev_bufs, int32_t nbufs, uint64_t bytes, int32_t dtype, const sl_config* cfg,
                     int32_t steps, sl_result* dev_out) {
    if (!cfg) return fail(SL_ERR_ARG, "cfg is NULL");
    if (!dev_out || (reinterpret_cast<uintptr_t>(dev_out) & 7u)) return fail(SL_ERR_ARG, "dev_out NULL or misaligned");
    if (steps < 1) return fail(SL_ERR_ARG, "steps %d < 1", steps);
    if (!dev_bufs || nbufs < 1) return fail(SL_ERR_ARG, "need at least one buffer");
    const bool dyn = cfg->order == SL_DYN;
    if (cfg->flush_l2) return fail(SL_ERR_ARG, "sl_enqueue_steps takes flush_l2 == 0");
    DevCtx* c = nullptr;
    int rc = get_ctx(&c);
    if (rc) return rc;
    std::lock_guard<std::recursive_mutex> g(c->mu);
    // One full wave: grid = resident CTAs per SM x SMs, so that a pass's CTAs
    // get SM slots only as the previous pass's CTAs exit (the passes overlap
    // in the tail, never side by side).
    Plan p;
    sl_config full = *cfg;
    full.grid = 0;
    rc = make_plan(c, dev_bufs[0], bytes, dtype, &full, &p);
    if (rc) return rc;
    const int32_t wave = p.resident * c->info.sm_count;
    if (cfg->grid > 0 && cfg->grid != wave)
        return fail(SL_ERR_ARG, "sl_enqueue_steps runs one full wave: grid must be 0 or %d (%d CTAs/SM x %d SMs)",
                    wave, p.resident, c->info.sm_count);
    full.grid = wave;
    std::vector<Plan> plans(static_cast<size_t>(nbufs));
    for (int32_t b = 0; b < nbufs; ++b) {
        rc = make_plan(c, dev_bufs[b], bytes, dtype, &full, &plans[b]);
        if (rc) return rc;
    }
    if (plans[0].grid == 0) {  // empty buffer (or no fixed iteration): zero results
        for (int32_t i = 0; i < steps; ++i) {
            rc = enqueue_locked(c, dev_bufs[i % nbufs], bytes, dtype, &full, dev_out + i, false, nullptr);
            if (rc) return rc;
        }
        return SL_OK;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cfg->stream);
    rc = ensure_scratch(c, static_cast<uint64_t>(plans[0].grid));
    if (rc) return rc;
    if (dyn && !c->step_next) CUDA_TRY(cudaMalloc(&c->step_next, STEP_COUNTERS * sizeof(uint32_t)));
    for (int32_t i = 0; i < steps; ++i) {
        // SL_DYN claims chunks from its counter from its first instruction, so
        // every pass gets a counter of its own, zeroed (in stream order, before
        // the segment's first pass) for up to STEP_COUNTERS passes at a time;
        // a segment's first pass is an ordinary launch.
        const int32_t slot = i % STEP_COUNTERS;
        if (dyn && slot == 0)
            CUDA_TRY(cudaMemsetAsync(c->step_next, 0,
                                     std::min<int32_t>(STEP_COUNTERS, steps - i) * sizeof(uint32_t), s));
        Plan& q = plans[i % nbufs];
        q.args.parts = c->parts;
        q.args.window = sl::ctrl_window(c->err);
        q.args.err = sl::ctrl_err(c->err);
        q.args.done = sl::ctrl_done(c->err);
        q.args.next = dyn ? c->step_next + slot : nullptr;
        q.args.result = dev_out + i;
        rc = launch(q, s, i > 0 && !(dyn && slot == 0));
        if (rc) return rc;
    }
    return SL_OK;
}

int sl_sweep(const void* dev_buf, uint64_t bytes, int32_t dtype, const sl_config* cells, int32_t ncells,
             int32_t repeats, int32_t warmup, int32_t sweep_order, sl_result* out) {
    if (!cells || !out || ncells < 0 || repeats < 1 || warmup < 0)
        return fail(SL_ERR_ARG, "bad sweep arguments");
    if (sweep_order != SL_ASC && sweep_order != SL_DESC) return fail(SL_ERR_ARG, "bad sweep order");
    DevCtx* c = nullptr;
    int rc = get_ctx(&c);
    if (rc) return rc;
    std::lock_guard<std::recursive_mutex> g(c->mu);
    for (int32_t j = 0; j < ncells; ++j) {
        const int32_t cell = sweep_order == SL_ASC ? j : ncells - 1 - j;
        sl_result* row = out + static_cast<int64_t>(cell) * repeats;
        sl_result tmp;
        int st = SL_OK;
        for (int32_t w = 0; w < warmup && st == SL_OK; ++w) st = run_locked(c, dev_buf, bytes, dtype, &cells[cell], &tmp);
        for (int32_t r = 0; r < repeats; ++r) {
            if (st == SL_OK) st = run_locked(c, dev_buf, bytes, dtype, &cells[cell], &row[r]);
            if (st != SL_OK) {
                std::memset(&row[r], 0, sizeof row[r]);
                row[r].status = st;
            }
        }
        if (st == SL_ERR_CUDA || st == SL_ERR_OOM || st == SL_ERR_NODEV) return st;
    }
    return SL_OK;
}

int sl_chase(const void* dev_chain, uint64_t bytes, uint32_t start, uint64_t warm, uint64_t hops, int32_t cache_l1,
             void* stream, sl_chase_result* out) {
    if (!out || !dev_chain) return fail(SL_ERR_ARG, "NULL argument");
    if ((bytes & 3u) || (reinterpret_cast<uintptr_t>(dev_chain) & 3u))
        return fail(SL_ERR_ALIGN, "chain must be 4-byte aligned and a multiple of 4 bytes");
    if (bytes / 4 == 0 || start >= bytes / 4) return fail(SL_ERR_ARG, "start index outside the chain");
    DevCtx* c = nullptr;
    int rc = get_ctx(&c);
    if (rc) return rc;
    std::lock_guard<std::recursive_mutex> g(c->mu);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint64_t* dout = reinterpret_cast<uint64_t*>(c->dres);  // sl_result scratch holds 4 words
    CUDA_TRY(sl::launch_chase(static_cast<const uint32_t*>(dev_chain), bytes / 4, start, warm, hops, cache_l1 ? 1 : 0,
                              dout, s));
    uint64_t h[4];
    CUDA_TRY(cudaMemcpyAsync(c->hres, dout, sizeof h, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    std::memcpy(h, c->hres, sizeof h);
    if (h[3]) return fail(SL_ERR_ARG, "the chain left the buffer (an index beyond its end)");
    out->final_index = static_cast<uint32_t>(h[0]);
    out->reserved = 0;
    out->hops = hops;
    out->ns = h[1];
    out->cycles = h[2];
    out->ns_per_hop = hops ? static_cast<double>(h[1]) / hops : 0.0;
    out->cycles_per_hop = hops ? static_cast<double>(h[2]) / hops : 0.0;
    return SL_OK;
}

int sl_twostream(const void* buf_a, uint64_t bytes_a, const void* buf_b, uint64_t bytes_b, int32_t passes_b,
                 int32_t warps_a, int32_t warps_b, int32_t k, int32_t flush_l2, void* stream,
                 sl_twostream_result* out) {
    if (!out) return fail(SL_ERR_ARG, "out is NULL");
    if (warps_a < 1 || warps_b < 0 || warps_a + warps_b > 32)
        return fail(SL_ERR_ARG, "warps_a %d / warps_b %d: need warps_a >= 1, warps_b >= 0, sum <= 32", warps_a, warps_b);
    if (!sl::two_kernel(k)) return fail(SL_ERR_ARG, "K %d not in {1,2,4,8}", k);
    if (passes_b < 0) return fail(SL_ERR_ARG, "passes_b %d < 0", passes_b);
    if (!buf_a || bytes_a == 0) return fail(SL_ERR_ARG, "stream A needs a non-empty buffer");
    if (warps_b > 0 && (!buf_b || bytes_b == 0)) return fail(SL_ERR_ARG, "stream B needs a non-empty buffer");
    if ((bytes_a & 15u) || (bytes_b & 15u) || (reinterpret_cast<uintptr_t>(buf_a) & 15u) ||
        (reinterpret_cast<uintptr_t>(buf_b) & 15u))
        return fail(SL_ERR_ALIGN, "buffers must be 16-byte aligned and multiples of 16 bytes");
    DevCtx* c = nullptr;
    int rc = get_ctx(&c);
    if (rc) return rc;
    std::lock_guard<std::recursive_mutex> g(c->mu);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint32_t grid = static_cast<uint32_t>(c->info.sm_count);
    const int block = 32 * (warps_a + warps_b);
    FuncInfo* fi = nullptr;
    rc = func_info(c, sl::two_kernel(k), 0, &fi);
    if (rc) return rc;
    if (fi->local_bytes > 0)
        return fail(SL_ERR_INFEASIBLE, "this kernel spills registers (%zu bytes of local memory per thread)",
                    fi->local_bytes);
    if (fi->regs < 4 * k + 16)
        return fail(SL_ERR_INFEASIBLE, "%d registers per thread cannot hold K=%d loads in flight", fi->regs, k);
    int resident = 0;
    rc = occupancy(c, sl::two_kernel(k), block, 0, &resident);
    if (rc) return rc;
    if (resident < 1) return fail(SL_ERR_INFEASIBLE, "a CTA of %d threads does not fit on an SM", block);
    if (!c->two_dev) {
        CUDA_TRY(cudaMalloc(&c->two_dev, 24 * sizeof(uint64_t)));
        CUDA_TRY(cudaMallocHost(&c->two_host, 24 * sizeof(uint64_t)));
    }
    rc = ensure_scratch(c, static_cast<uint64_t>(grid) * 32);
    if (rc) return rc;
    sl::TwoArgs t{};
    t.buf_a = static_cast<const uint4*>(buf_a);
    t.buf_b = static_cast<const uint4*>(warps_b > 0 ? buf_b : buf_a);
    t.warps_a = static_cast<uint32_t>(warps_a);
    t.warps_b = static_cast<uint32_t>(warps_b);
    const uint64_t pb = passes_b == 0 ? 1 : static_cast<uint64_t>(passes_b);
    const uint64_t tv_a = 32ull * warps_a * k, tv_b = 32ull * (warps_b > 0 ? warps_b : 1) * k;
    t.nvec_a = bytes_a / 16;
    t.nvec_b = warps_b > 0 ? bytes_b / 16 : 0;
    const uint64_t nt_a = (t.nvec_a + tv_a - 1) / tv_a, nt_b = (t.nvec_b + tv_b - 1) / tv_b;
    // 32-bit tile and per-thread load counters in the kernel
    if (nt_a + grid >= (1ull << 32) || nt_b * pb + grid >= (1ull << 32) ||
        (nt_b * pb / grid + 1) * k >= (1ull << 32))
        return fail(SL_ERR_ARG, "buffers or passes too large for one launch");
    t.ntiles_a = static_cast<uint32_t>(nt_a);
    t.total_a = static_cast<uint32_t>(nt_a);
    t.ntiles_b = static_cast<uint32_t>(nt_b);
    t.total_b = static_cast<uint32_t>(nt_b * pb);
    t.parts = c->parts;
    t.ctl = c->two_dev;
    if (flush_l2) CUDA_TRY(sl::launch_flush(c->flush, c->flush_bytes / 16, c->info.sm_count, s));
    // timer words: starts ~0, ends 0, B's first end ~0
    CUDA_TRY(cudaMemsetAsync(c->two_dev + sl::TWO_START, 0xFF, 2 * sizeof(uint64_t), s));
    CUDA_TRY(cudaMemsetAsync(c->two_dev + sl::TWO_END, 0, 2 * sizeof(uint64_t), s));
    CUDA_TRY(cudaMemsetAsync(c->two_dev + sl::TWO_FIRST_END_B, 0xFF, sizeof(uint64_t), s));
    CUDA_TRY(cudaEventRecord(c->ev0, s));
    CUDA_TRY(sl::launch_two(t, k, grid, s));
    CUDA_TRY(cudaEventRecord(c->ev1, s));
    CUDA_TRY(sl::launch_two_combine(t, grid, c->two_dev + 8, s));
    CUDA_TRY(cudaMemcpyAsync(c->two_host, c->two_dev + 8, 11 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    float ms = 0.0f;
    CUDA_TRY(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    const uint64_t* h = c->two_host;
    std::memset(out, 0, sizeof *out);
    for (int i = 0; i < 2; ++i) {
        out->sum_u32[i] = static_cast<uint32_t>(h[3 * i]);
        out->xor_u64[i] = h[3 * i + 1];
        out->issued_loads[i] = h[3 * i + 2];
        const uint64_t t0 = h[6 + sl::TWO_START + i], t1 = h[6 + sl::TWO_END + i];
        out->window_ns[i] = (i == 0 || warps_b > 0) && t1 > t0 ? t1 - t0 : 0;
    }
    const uint64_t a0 = h[6 + sl::TWO_START], a1 = h[6 + sl::TWO_END], bfe = h[6 + sl::TWO_FIRST_END_B];
    out->b_first_end_ns = warps_b > 0 && bfe > a0 ? bfe - a0 : 0;
    out->b_covers_a = warps_b == 0 || bfe >= a1 ? 1 : 0;
    out->device_ns = static_cast<uint64_t>(static_cast<double>(ms) * 1e6 + 0.5);
    out->grid = static_cast<int32_t>(grid);
    out->cta = block;
    return SL_OK;
}

int sl_run_host(const void* host_buf, uint64_t bytes, int32_t dtype, const sl_config* cfg, sl_result* out) {
    if (!out || !cfg) return fail(SL_ERR_ARG, "NULL argument");
    if (cfg->target_loads) return fail(SL_ERR_ARG, "sl_run_host runs exact fixed work only (target_loads 0)");
    if (bytes > 0 && !host_buf) return fail(SL_ERR_ARG, "host buffer is NULL");
    if ((bytes & 15u) != 0) return fail(SL_ERR_ALIGN, "bytes not a multiple of 16");
    DevCtx* c = nullptr;
    int rc = get_ctx(&c);
    if (rc) return rc;
    std::lock_guard<std::recursive_mutex> g(c->mu);
    cudaStream_t s = static_cast<cudaStream_t>(cfg->stream);
    if (cfg->host_direct) {
        // The kernel reads the host buffer in place: pinned memory through its
        // device mapping, pageable memory where the device can address it.
        const void* dptr = nullptr;
        if (bytes > 0) {
            cudaPointerAttributes pa;
            if (cudaPointerGetAttributes(&pa, host_buf) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
                pa.devicePointer) {
                dptr = pa.devicePointer;
            } else {
                (void)cudaGetLastError();
                int pageable = 0;
                cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, c->dev);
                (void)cudaGetLastError();
                if (!pageable) return fail(SL_ERR_ARG, "the device cannot address this host buffer directly");
                dptr = host_buf;
            }
        }
        CUDA_TRY(cudaEventRecord(c->ev0, s));
        Plan p;
        int rc2 = enqueue_locked(c, dptr, bytes, dtype, cfg, c->dres, false, &p);
        if (rc2) return rc2;
        CUDA_TRY(cudaMemcpyAsync(c->hres, c->dres, sizeof(sl_result), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaEventRecord(c->ev1, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        float ms = 0.0f;
        CUDA_TRY(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
        *out = *c->hres;
        out->device_ns = static_cast<uint64_t>(static_cast<double>(ms) * 1e6 + 0.5);
        fill_shape(p, out);
        if (out->status != SL_OK) return fail(out->status, "a bounded device wait timed out");
        return SL_OK;
    }
    if (!c->stage[0]) {
        for (int b = 0; b < 2; ++b) {
            CUDA_TRY(cudaMalloc(&c->stage[b], HOST_CHUNK));
            CUDA_TRY(cudaEventCreateWithFlags(&c->copied[b], cudaEventDisableTiming));
            CUDA_TRY(cudaEventCreateWithFlags(&c->consumed[b], cudaEventDisableTiming));
        }
        CUDA_TRY(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    }
    const uint64_t chunk = std::min<uint64_t>(bytes, HOST_CHUNK);
    const uint64_t nchunks = bytes == 0 ? 0 : (bytes + HOST_CHUNK - 1) / HOST_CHUNK;
    // One launch shape for every chunk (planned on a full chunk), so every
    // chunk's kernel writes all of its partial slots.
    Plan p;
    rc = make_plan(c, c->stage[0], chunk, dtype, cfg, &p);
    if (rc) return rc;
    const uint64_t per_parts = static_cast<uint64_t>(p.grid);  // one partial per CTA
    rc = ensure_scratch(c, per_parts * nchunks);
    if (rc) return rc;
    const uint64_t passes = cfg->passes == 0 ? 1 : static_cast<uint64_t>(cfg->passes);

    CUDA_TRY(cudaEventRecord(c->ev0, s));
    CUDA_TRY(cudaStreamWaitEvent(c->copy_stream, c->ev0, 0));
    for (uint64_t i = 0; i < nchunks; ++i) {
        const int b = static_cast<int>(i & 1);
        const uint64_t off = i * HOST_CHUNK;
        const uint64_t len = std::min<uint64_t>(HOST_CHUNK, bytes - off);
        if (i >= 2) CUDA_TRY(cudaStreamWaitEvent(c->copy_stream, c->consumed[b], 0));
        CUDA_TRY(cudaMemcpyAsync(c->stage[b], static_cast<const uint8_t*>(host_buf) + off, len,
                                 cudaMemcpyHostToDevice, c->copy_stream));
        CUDA_TRY(cudaEventRecord(c->copied[b], c->copy_stream));
        CUDA_TRY(cudaStreamWaitEvent(s, c->copied[b], 0));
        KArgs a = p.args;
        const uint64_t nvec = len / (cfg->mech == SL_LDG4 ? 4 : 16);
        const uint64_t units = cfg->mech == SL_LDG32 ? (nvec + 1) / 2 : nvec;
        a.buf = c->stage[b];
        a.nvec = nvec;
        a.ntiles = (units + a.tile_vec - 1) / a.tile_vec;
        a.total = a.ntiles * passes;
        a.parts = c->parts + i * per_parts;
        a.window = sl::ctrl_window(c->err);
        a.err = c->err;
        a.result = nullptr;  // combined over all chunks below
        a.done = nullptr;
        if (cfg->order == SL_DYN) {  // no last-CTA reset here: clear the chunk counter per launch
            a.next = sl::ctrl_next(c->err);
            CUDA_TRY(cudaMemsetAsync(a.next, 0, sizeof(uint32_t), s));
        }
        void* args[] = {&a};
        CUDA_TRY(cudaLaunchKernel(p.fn, dim3(static_cast<unsigned>(p.grid)), dim3(p.block), args, p.smem, s));
        CUDA_TRY(cudaEventRecord(c->consumed[b], s));
    }
    if (cfg->order == SL_DYN)  // leave the chunk counter at zero for the next launch
        CUDA_TRY(cudaMemsetAsync(sl::ctrl_next(c->err), 0, sizeof(uint32_t), s));
    CUDA_TRY(sl::launch_combine(c->parts, per_parts * nchunks, sl::ctrl_window(c->err), c->err, c->dres, s));
    CUDA_TRY(cudaMemcpyAsync(c->hres, c->dres, sizeof(sl_result), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaEventRecord(c->ev1, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    float ms = 0.0f;
    CUDA_TRY(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    *out = *c->hres;
    out->device_ns = static_cast<uint64_t>(static_cast<double>(ms) * 1e6 + 0.5);
    fill_shape(p, out);
    if (nchunks == 0) out->grid = 0;
    if (out->status != SL_OK) return fail(out->status, "a bounded device wait timed out");
    return SL_OK;
}

}  // extern "C"
