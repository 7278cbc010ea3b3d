// batch_api.cu -- host side of the batched form (sl_batch_*).
//
// Planning: each buffer goes to the first tuning-table entry that matches
// its dtype and size; buffers of one entry (a size class) and one dtype form
// a group that one persistent class kernel streams.  Buffers are cut into
// work items of at most ITEM_BYTES; each item owns one partial slot per
// folding warp of its group's kernel, and a buffer's items (hence its slots)
// are contiguous.  The CUDA graph -- memset of the item counters and the
// error word, the class kernels as parallel branches, then the per-buffer
// combine -- is captured once and replayed by sl_batch_run.
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "k_batch.cuh"

namespace sl {
const void* batch_ldg_kernel(int dtype, int k, int cta);
const void* batch_cpasync_kernel(int dtype, int d);
const void* batch_tma_kernel(int dtype, int batch);
cudaError_t launch_batch_combine(const BufSeg* segs, uint32_t nbuf, const WarpPartial* parts, const uint32_t* err,
                                 sl_result* out, cudaStream_t s);
}  // namespace sl

namespace {

using sl::BatchItem;
using sl::BufSeg;
using sl::WarpPartial;

constexpr uint64_t ITEM_BYTES = 1ull << 20;
constexpr uint64_t TIMEOUT_NS = 2000000000ull;

int bfail(int code, const char* msg) { return sl::set_error(code, msg); }

#define B_TRY(expr, what)                                   \
    do {                                                    \
        cudaError_t e_ = (expr);                            \
        if (e_ != cudaSuccess) {                            \
            (void)cudaGetLastError();                       \
            return bfail(e_ == cudaErrorMemoryAllocation ? SL_ERR_OOM : SL_ERR_CUDA, what); \
        }                                                   \
    } while (0)

struct Group {
    int entry = -1;
    int dtype = 0;
    sl_config cfg{};
    const void* fn = nullptr;
    int block = 0;
    size_t smem = 0;
    int grid = 0;
    uint32_t warps = 0;       // folding warps per CTA (partial slots per item)
    std::vector<BatchItem> items;
    uint64_t item_off = 0;    // offset of this group's items in the device item array
};

}  // namespace

struct sl_batch {
    int dev = -1;
    int n = 0;
    std::vector<int32_t> class_of;
    std::vector<Group> groups;
    BatchItem* d_items = nullptr;
    BufSeg* d_segs = nullptr;
    WarpPartial* d_parts = nullptr;
    sl_result* d_results = nullptr;
    uint32_t* d_ctrl = nullptr;  // [0]: error word; [16 + g]: item counter of group g
    size_t ctrl_bytes = 0;
    sl_result* h_results = nullptr;
    uint32_t* h_err = nullptr;   // pinned copy of the error word after each run
    cudaStream_t stream = nullptr;
    std::vector<cudaStream_t> branch;
    std::vector<cudaEvent_t> branch_ev;
    cudaEvent_t fork_ev = nullptr, e0 = nullptr, e1 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

void release(sl_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto e : b->branch_ev) cudaEventDestroy(e);
    for (auto s : b->branch) cudaStreamDestroy(s);
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    if (b->e0) cudaEventDestroy(b->e0);
    if (b->e1) cudaEventDestroy(b->e1);
    if (b->stream) cudaStreamDestroy(b->stream);
    cudaFree(b->d_items);
    cudaFree(b->d_segs);
    cudaFree(b->d_parts);
    cudaFree(b->d_results);
    cudaFree(b->d_ctrl);
    cudaFreeHost(b->h_results);
    cudaFreeHost(b->h_err);
    (void)cudaGetLastError();
    delete b;
}

// Kernel, block shape, shared memory and persistent grid of one group.
int plan_group(Group& g, int sms, int smem_optin) {
    const sl_config& c = g.cfg;
    if (c.cta < 32 || c.cta > 1024 || (c.cta & 31)) return bfail(SL_ERR_ARG, "tuning entry: bad cta");
    if (c.target_loads) return bfail(SL_ERR_ARG, "tuning entry: the batched form runs exact fixed work (target_loads 0)");
    if (c.copies != 0 && c.copies != 1)
        return bfail(SL_ERR_ARG, "tuning entry: the batched cp.async class kernel puts one copy in each commit "
                     "group (copies must be 0 or 1)");
    switch (c.mech) {
    case SL_LDG:
        g.fn = sl::batch_ldg_kernel(g.dtype, c.k, c.cta);
        if (!g.fn) return bfail(SL_ERR_ARG, "tuning entry: no batched LDG kernel (K in {1,2,3,4,6,8,12,16}, cta 128/256/512)");
        g.block = c.cta;
        g.smem = 0;
        g.warps = c.cta / 32;
        break;
    case SL_CPASYNC:
        g.fn = sl::batch_cpasync_kernel(g.dtype, c.k);
        if (!g.fn) return bfail(SL_ERR_ARG, "tuning entry: cp.async depth not in 1..8");
        g.block = c.cta;
        g.smem = static_cast<size_t>(c.k) * c.cta * 16;
        g.warps = c.cta / 32;
        break;
    case SL_TMA:
        if (c.stage_bytes != 4096 && c.stage_bytes != 16384 && c.stage_bytes != 65536)
            return bfail(SL_ERR_INFEASIBLE, "tuning entry: TMA stage size not 4096/16384/65536");
        if (c.stages < SL_MIN_STAGES || c.stages > SL_MAX_STAGES) return bfail(SL_ERR_ARG, "tuning entry: TMA stages");
        if (c.cta > 992) return bfail(SL_ERR_ARG, "tuning entry: TMA consumer threads > 992");
        if (c.tma_ring != SL_RING_CTA)
            return bfail(SL_ERR_ARG, "tuning entry: the batched TMA class kernel has one ring per CTA "
                         "(tma_ring must be SL_RING_CTA)");
        // consumer threads read their last 4 vectors of a stage (1 where they
        // read fewer) into registers before releasing it
        g.fn = sl::batch_tma_kernel(g.dtype, c.stage_bytes / 16 >= 4 * c.cta ? 4 : 1);
        g.block = c.cta + 32;
        g.smem = static_cast<size_t>(c.stages) * c.stage_bytes;
        g.warps = c.cta / 32;
        break;
    default:
        return bfail(SL_ERR_ARG, "tuning entry: bad mech");
    }
    if (g.smem > static_cast<size_t>(smem_optin)) return bfail(SL_ERR_INFEASIBLE, "tuning entry: shared memory over the limit");
    cudaFuncAttributes fa;
    B_TRY(cudaFuncGetAttributes(&fa, g.fn), "cudaFuncGetAttributes failed");
    if (fa.localSizeBytes > 0) return bfail(SL_ERR_INFEASIBLE, "tuning entry: kernel spills registers");
    if (g.block > fa.maxThreadsPerBlock) return bfail(SL_ERR_INFEASIBLE, "tuning entry: too many threads for this kernel");
    if (g.smem > 0)
        B_TRY(cudaFuncSetAttribute(g.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(g.smem)),
              "cudaFuncSetAttribute failed");
    int res = 0;
    B_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&res, g.fn, g.block, g.smem), "occupancy query failed");
    if (res < 1) return bfail(SL_ERR_INFEASIBLE, "tuning entry: zero occupancy");
    g.grid = c.grid > 0 ? c.grid : res * sms;
    return SL_OK;
}

// Everything after the argument checks; the caller releases b on failure.
int build_batch(sl_batch* b, const sl_batch_desc* descs, int32_t n, const sl_tune_entry* table, int32_t ntable,
                int sms, int optin) {
    // ---- group the buffers
    std::map<std::pair<int, int>, int> gidx;  // (entry, dtype) -> group
    for (int32_t i = 0; i < n; ++i) {
        const sl_batch_desc& d = descs[i];
        if (d.dtype < SL_U32 || d.dtype > SL_FP8_E4M3) return bfail(SL_ERR_ARG, "bad dtype in a descriptor");
        if ((d.bytes & 15u) || (reinterpret_cast<uintptr_t>(d.ptr) & 15u))
            return bfail(SL_ERR_ALIGN, "a descriptor is not 16-byte aligned or its size is not a multiple of 16");
        if (d.bytes > 0 && !d.ptr) return bfail(SL_ERR_ARG, "a descriptor has a NULL pointer");
        int e = -1;
        for (int32_t j = 0; j < ntable && e < 0; ++j)
            if ((table[j].dtype < 0 || table[j].dtype == d.dtype) && d.bytes >= table[j].min_bytes &&
                d.bytes <= table[j].max_bytes)
                e = j;
        if (e < 0) return bfail(SL_ERR_ARG, "no tuning-table entry matches a buffer");
        auto key = std::make_pair(e, static_cast<int>(d.dtype));
        if (!gidx.count(key)) {
            Group g;
            g.entry = e;
            g.dtype = d.dtype;
            g.cfg = table[e].cfg;
            int rc = plan_group(g, sms, optin);
            if (rc) return rc;
            gidx[key] = static_cast<int>(b->groups.size());
            b->groups.push_back(std::move(g));
        }
        b->class_of[i] = gidx[key];
    }

    // ---- items, partial slots, per-buffer segments (buffers in order)
    std::vector<BufSeg> segs(n);
    uint64_t slots = 0;
    for (int32_t i = 0; i < n; ++i) {
        Group& g = b->groups[b->class_of[i]];
        segs[i].pstart = static_cast<uint32_t>(slots);
        const uint64_t bytes = descs[i].bytes;
        const uint8_t* p = static_cast<const uint8_t*>(descs[i].ptr);
        for (uint64_t off = 0; off < bytes; off += ITEM_BYTES) {
            const uint64_t len = std::min<uint64_t>(ITEM_BYTES, bytes - off);
            BatchItem it;
            it.ptr = reinterpret_cast<const uint4*>(p + off);
            it.nvec = static_cast<uint32_t>(len / 16);
            it.part = static_cast<uint32_t>(slots);
            g.items.push_back(it);
            slots += g.warps;
        }
        segs[i].pcount = static_cast<uint32_t>(slots - segs[i].pstart);
        if (slots >= (1ull << 32)) return bfail(SL_ERR_ARG, "batch too large");
    }
    std::vector<BatchItem> all;
    for (Group& g : b->groups) {
        g.item_off = all.size();
        all.insert(all.end(), g.items.begin(), g.items.end());
    }

    // ---- device tables (allocated before capture)
    const size_t ng = b->groups.size();
    b->ctrl_bytes = (16 + ng) * sizeof(uint32_t);
    B_TRY(cudaMalloc(&b->d_items, std::max<size_t>(all.size(), 1) * sizeof(BatchItem)), "cudaMalloc failed");
    B_TRY(cudaMalloc(&b->d_segs, std::max<size_t>(n, 1) * sizeof(BufSeg)), "cudaMalloc failed");
    B_TRY(cudaMalloc(&b->d_parts, std::max<uint64_t>(slots, 1) * sizeof(WarpPartial)), "cudaMalloc failed");
    B_TRY(cudaMalloc(&b->d_results, std::max<size_t>(n, 1) * sizeof(sl_result)), "cudaMalloc failed");
    B_TRY(cudaMalloc(&b->d_ctrl, b->ctrl_bytes), "cudaMalloc failed");
    B_TRY(cudaMallocHost(&b->h_results, std::max<size_t>(n, 1) * sizeof(sl_result)), "cudaMallocHost failed");
    B_TRY(cudaMallocHost(&b->h_err, sizeof(uint32_t)), "cudaMallocHost failed");
    if (!all.empty())
        B_TRY(cudaMemcpy(b->d_items, all.data(), all.size() * sizeof(BatchItem), cudaMemcpyHostToDevice), "copy failed");
    if (n > 0) B_TRY(cudaMemcpy(b->d_segs, segs.data(), n * sizeof(BufSeg), cudaMemcpyHostToDevice), "copy failed");
    B_TRY(cudaMemset(b->d_ctrl, 0, b->ctrl_bytes), "memset failed");

    // ---- streams and events, then capture the graph
    B_TRY(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking), "stream create failed");
    B_TRY(cudaEventCreate(&b->e0), "event create failed");
    B_TRY(cudaEventCreate(&b->e1), "event create failed");
    B_TRY(cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming), "event create failed");
    for (size_t g = 0; g < ng; ++g) {
        cudaStream_t s;
        cudaEvent_t e;
        B_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream create failed");
        b->branch.push_back(s);
        B_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event create failed");
        b->branch_ev.push_back(e);
    }
    B_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture failed");
    cudaError_t ce = cudaMemsetAsync(b->d_ctrl, 0, b->ctrl_bytes, b->stream);
    if (ce == cudaSuccess) ce = cudaEventRecord(b->fork_ev, b->stream);
    for (size_t g = 0; g < ng && ce == cudaSuccess; ++g) {
        Group& gr = b->groups[g];
        ce = cudaStreamWaitEvent(b->branch[g], b->fork_ev, 0);
        if (ce != cudaSuccess) break;
        sl::BArgs a{};
        a.items = b->d_items + gr.item_off;
        a.nitems = static_cast<uint32_t>(gr.items.size());
        a.stage_bytes = static_cast<uint32_t>(gr.cfg.stage_bytes);
        a.next = b->d_ctrl + 16 + g;
        a.parts = b->d_parts;
        a.err = b->d_ctrl;
        a.timeout_ns = TIMEOUT_NS;
        a.nst = gr.cfg.mech == SL_TMA ? gr.cfg.stages : 0;
        void* args[] = {&a};
        if (a.nitems > 0) ce = cudaLaunchKernel(gr.fn, dim3(gr.grid), dim3(gr.block), args, gr.smem, b->branch[g]);
        if (ce == cudaSuccess) ce = cudaEventRecord(b->branch_ev[g], b->branch[g]);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(b->stream, b->branch_ev[g], 0);
    }
    if (ce == cudaSuccess)
        ce = sl::launch_batch_combine(b->d_segs, static_cast<uint32_t>(n), b->d_parts, b->d_ctrl, b->d_results,
                                      b->stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b->stream, &graph);
    b->graph = graph;
    if (ce != cudaSuccess || ee != cudaSuccess) {
        (void)cudaGetLastError();
        return bfail(SL_ERR_CUDA, "capturing the batch graph failed");
    }
    B_TRY(cudaGraphInstantiate(&b->exec, b->graph, 0), "graph instantiation failed");
    return SL_OK;
}

}  // namespace

extern "C" {

int sl_batch_create(const sl_batch_desc* descs, int32_t n, const sl_tune_entry* table, int32_t ntable,
                    sl_batch** out) {
    if (!out) return bfail(SL_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 0 || (n > 0 && !descs) || ntable < 1 || !table) return bfail(SL_ERR_ARG, "bad batch arguments");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return bfail(SL_ERR_NODEV, "no CUDA device");
    }
    int sms = 0, optin = 0;
    B_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device query failed");
    B_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "device query failed");
    sl_batch* b = new (std::nothrow) sl_batch();
    if (!b) return bfail(SL_ERR_OOM, "out of host memory");
    b->dev = dev;
    b->n = n;
    b->class_of.assign(n, -1);
    const int rc = build_batch(b, descs, n, table, ntable, sms, optin);
    if (rc) {
        release(b);
        return rc;
    }
    *out = b;
    return SL_OK;
}

int sl_batch_run(sl_batch* b, sl_result* per_buffer, uint64_t* total_ns) {
    if (!b) return bfail(SL_ERR_ARG, "batch is NULL");
    B_TRY(cudaEventRecord(b->e0, b->stream), "event record failed");
    B_TRY(cudaGraphLaunch(b->exec, b->stream), "graph launch failed");
    B_TRY(cudaEventRecord(b->e1, b->stream), "event record failed");
    if (per_buffer && b->n > 0)
        B_TRY(cudaMemcpyAsync(b->h_results, b->d_results, b->n * sizeof(sl_result), cudaMemcpyDeviceToHost, b->stream),
              "result copy failed");
    B_TRY(cudaMemcpyAsync(b->h_err, b->d_ctrl, sizeof(uint32_t), cudaMemcpyDeviceToHost, b->stream),
          "error-word copy failed");
    B_TRY(cudaStreamSynchronize(b->stream), "batch run failed");
    float ms = 0.0f;
    B_TRY(cudaEventElapsedTime(&ms, b->e0, b->e1), "event timing failed");
    if (total_ns) *total_ns = static_cast<uint64_t>(static_cast<double>(ms) * 1e6 + 0.5);
    int st = *b->h_err ? SL_ERR_TIMEOUT : SL_OK;
    if (per_buffer && b->n > 0) {
        std::memcpy(per_buffer, b->h_results, b->n * sizeof(sl_result));
        for (int i = 0; i < b->n; ++i)
            if (per_buffer[i].status != SL_OK) st = per_buffer[i].status;
    }
    if (st != SL_OK) return bfail(st, "a bounded device wait timed out");
    return SL_OK;
}

int sl_batch_info(const sl_batch* b, int32_t* nclasses, int32_t* class_of_buffer) {
    if (!b) return bfail(SL_ERR_ARG, "batch is NULL");
    if (nclasses) *nclasses = static_cast<int32_t>(b->groups.size());
    if (class_of_buffer)
        for (int i = 0; i < b->n; ++i) class_of_buffer[i] = b->class_of[i];
    return SL_OK;
}

void sl_batch_destroy(sl_batch* b) { release(b); }

}  // extern "C"
