// noalloc.cu -- sl_run_noalloc: the LDG streaming checksum for callers that
// cannot allocate device memory.
//
// Who needs this: code that runs where a cudaMalloc is not acceptable --
// inside a framework whose own pool allocator owns (nearly) all device
// memory, so an allocation behind its back can fail or fragment the pool;
// in a latency-critical loop, where cudaMalloc/cudaFree may synchronize the
// device; or in a plugin or callback whose host contract forbids allocating.
// The regular entry points allocate their scratch lazily (and may grow it,
// which synchronizes the device), so such callers cannot use them.
//
// Here the scratch -- per-CTA partials and a 256-byte control block (device
// error word, finished-CTA counter, timing window) -- lives in one file-scope
// __device__ array of fixed size
// (SL_NOALLOC_SCRATCH_BYTES).  Every GPU that loads this library holds that
// array until the process exits.  Host code never uses the array's name as an
// address (on the host it is only a stand-in); it asks the runtime for the
// device address with cudaGetSymbolAddress, once per device, with that device
// current, and passes that pointer to the kernels.  The address belongs to
// the device's context: the cache remembers which context it was looked up
// in (by the driver's unique context id) and looks it up again once that
// context has been replaced, e.g. after cudaDeviceReset.
#include <cstdint>
#include <mutex>

#include <cuda.h>  // CUcontext / CUresult types only; the driver is reached through the runtime

#include "sl_internal.h"

namespace {

constexpr uint64_t NA_MAX_CTAS = SL_NOALLOC_MAX_CTAS;
constexpr uint64_t NA_PARTS_OFF = 0;
constexpr uint64_t NA_CTRL_OFF = NA_PARTS_OFF + NA_MAX_CTAS * sizeof(sl::WarpPartial);
constexpr uint64_t NA_BYTES = NA_CTRL_OFF + sl::CTRL_BYTES;
static_assert(NA_BYTES == SL_NOALLOC_SCRATCH_BYTES, "scratch layout");

// The fixed scratch.  Shared by every sl_run_noalloc call on a device; it
// keeps the previous call's contents, so the control block is cleared before
// each launch (the partials are fully rewritten by the kernel).
static __device__ __align__(256) unsigned char g_noalloc_scratch[SL_NOALLOC_SCRATCH_BYTES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mu;
unsigned char* g_na_ptr[NA_MAX_DEVICES] = {};
unsigned long long g_na_ctx[NA_MAX_DEVICES] = {};  // context id the address was looked up in

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// The driver's unique id of the calling thread's current context, or 0 if
// there is none (or the driver cannot tell).  Ids are never reused within a
// process, so a replaced context never matches an old id.
unsigned long long current_ctx_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(p);
        (void)cudaGetLastError();
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of g_noalloc_scratch on device `dev` (which must be
// current): looked up once per device, and again if the device's context
// has been replaced since (the old address belonged to the old context).
int scratch_for(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> g(g_na_mu);
    const unsigned long long ctx = current_ctx_id();
    if (!g_na_ptr[dev] || (ctx != 0 && ctx != g_na_ctx[dev])) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return sl::set_error(SL_ERR_CUDA, "cudaGetSymbolAddress of the fixed scratch failed");
        }
        g_na_ptr[dev] = static_cast<unsigned char*>(p);
        g_na_ctx[dev] = current_ctx_id();  // the lookup made a context current if there was none
    }
    *out = g_na_ptr[dev];
    return SL_OK;
}

int na_fail(int code, const char* msg) { return sl::set_error(code, msg); }

}  // namespace

extern "C" int sl_run_noalloc(const void* dev_buf, uint64_t bytes, int32_t dtype, const sl_config* cfg,
                              sl_result* dev_out) {
    if (!cfg) return na_fail(SL_ERR_ARG, "cfg is NULL");
    if (cfg->mech != SL_LDG) return na_fail(SL_ERR_ARG, "sl_run_noalloc supports the LDG mechanism only");
    if (cfg->flush_l2) return na_fail(SL_ERR_ARG, "sl_run_noalloc cannot flush L2 (the flush buffer is allocated)");
    if (cfg->debug_flags) return na_fail(SL_ERR_ARG, "sl_run_noalloc takes no debug flags");
    if (cfg->target_loads) return na_fail(SL_ERR_ARG, "sl_run_noalloc runs exact fixed work only (target_loads 0)");
    if (dtype < SL_U32 || dtype > SL_FP8_E4M3) return na_fail(SL_ERR_ARG, "bad dtype");
    if (!dev_out || (reinterpret_cast<uintptr_t>(dev_out) & 7u)) return na_fail(SL_ERR_ARG, "dev_out NULL or not 8-byte aligned");
    if ((bytes & 15u) != 0) return na_fail(SL_ERR_ALIGN, "bytes not a multiple of 16");
    if (bytes > 0 && !dev_buf) return na_fail(SL_ERR_ARG, "buffer is NULL");
    if ((reinterpret_cast<uintptr_t>(dev_buf) & 15u) != 0) return na_fail(SL_ERR_ALIGN, "buffer not 16-byte aligned");
    if (cfg->passes < 0) return na_fail(SL_ERR_ARG, "passes < 0");
    if (cfg->order != SL_ASC && cfg->order != SL_DESC) return na_fail(SL_ERR_ARG, "bad order");
    if (cfg->k < 1 || cfg->k > SL_MAX_K) return na_fail(SL_ERR_ARG, "K not in 1..16");
    const int cta = cfg->cta;
    const void* fn = sl::ldg_kernel(dtype, cfg->k, cta, cfg->cop);
    if (!fn) return na_fail(SL_ERR_ARG, "no LDG kernel for this dtype / K / cta / cop");

    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        (void)cudaGetLastError();
        return na_fail(SL_ERR_NODEV, "no usable CUDA device");
    }
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
        (void)cudaGetLastError();
        return na_fail(SL_ERR_CUDA, "cudaFuncGetAttributes failed");
    }
    if (fa.localSizeBytes > 0 || fa.numRegs < 4 * cfg->k + 16)
        return na_fail(SL_ERR_INFEASIBLE, "this LDG kernel cannot keep K loads in registers at this cta");
    int resident = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, fn, cta, 0) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return na_fail(SL_ERR_CUDA, "occupancy / SM-count query failed");
    }
    if (resident < 1) return na_fail(SL_ERR_INFEASIBLE, "zero occupancy");
    const uint64_t grid = cfg->grid > 0 ? static_cast<uint64_t>(cfg->grid)
                                        : static_cast<uint64_t>(resident < 4 ? resident : 4) * sms;
    if (grid > NA_MAX_CTAS)
        return na_fail(SL_ERR_ARG, "launch exceeds the fixed scratch: at most SL_NOALLOC_MAX_CTAS (4096) CTAs");

    {
        const uint64_t tv = static_cast<uint64_t>(cta) * cfg->k;
        const uint64_t tot = (bytes / 16 + tv - 1) / tv * (cfg->passes == 0 ? 1 : static_cast<uint64_t>(cfg->passes));
        if (tot + grid >= (1ull << 32) || (tot + grid - 1) / grid * cfg->k >= (1ull << 32))
            return na_fail(SL_ERR_ARG, "passes x tiles too large for one launch; lower passes");
    }
    unsigned char* base = nullptr;
    int rc = scratch_for(dev, &base);
    if (rc) return rc;
    sl::WarpPartial* parts = reinterpret_cast<sl::WarpPartial*>(base + NA_PARTS_OFF);
    void* ctrl = base + NA_CTRL_OFF;
    cudaStream_t s = static_cast<cudaStream_t>(cfg->stream);

    // error word and CTA counter start at zero, the window at (~0, 0)
    if (cudaMemsetAsync(ctrl, 0, sl::CTRL_BYTES, s) != cudaSuccess ||
        cudaMemsetAsync(sl::ctrl_window(ctrl), 0xFF, sizeof(uint64_t), s) != cudaSuccess) {
        (void)cudaGetLastError();
        return na_fail(SL_ERR_CUDA, "clearing the control block failed");
    }
    const uint64_t nvec = bytes / 16;
    const uint64_t passes = cfg->passes == 0 ? 1 : static_cast<uint64_t>(cfg->passes);
    const uint64_t launched = nvec == 0 ? 0 : grid;
    if (launched) {
        sl::KArgs a{};
        const uint64_t tile_vec = static_cast<uint64_t>(cta) * cfg->k;
        a.buf = dev_buf;
        a.nvec = nvec;
        a.ntiles = (nvec + tile_vec - 1) / tile_vec;
        a.total = a.ntiles * passes;
        a.tile_vec = static_cast<uint32_t>(tile_vec);
        a.desc = cfg->order == SL_DESC ? 1 : 0;
        a.parts = parts;
        a.window = sl::ctrl_window(ctrl);
        a.err = sl::ctrl_err(ctrl);
        a.timeout_ns = 2000000000ull;
        a.result = dev_out;  // the last CTA writes the result
        a.done = sl::ctrl_done(ctrl);
        void* args[] = {&a};
        if (cudaLaunchKernel(fn, dim3(static_cast<unsigned>(grid)), dim3(cta), args, 0, s) != cudaSuccess) {
            (void)cudaGetLastError();
            return na_fail(SL_ERR_CUDA, "kernel launch failed");
        }
    }
    if (!launched &&
        sl::launch_combine(parts, 0, sl::ctrl_window(ctrl), sl::ctrl_err(ctrl), dev_out, s) != cudaSuccess) {
        (void)cudaGetLastError();
        return na_fail(SL_ERR_CUDA, "combine launch failed");
    }
    return SL_OK;
}
