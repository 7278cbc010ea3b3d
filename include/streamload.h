/*
 * streamload.h -- C ABI of the GB300 (sm_103a) streaming global-load library.
 *
 * The library measures how attained HBM bandwidth responds to offered load
 * concurrency, the quantity studied by "Concurrency Response of Plain Global
 * Loads on the NVIDIA H100" (arXiv 2608.15764).  One data-parallel hot path:
 * every 16-byte vector of a device buffer is loaded exactly once per pass and
 * folded into a checksum (paper §3 "Instruments": loaded values go into a sink
 * so that no load is dead), with the total number of issued 16-byte loads held
 * fixed across offered ILP K (paper §3 "Fixed-work control").  Three load
 * mechanisms:
 *
 *   SL_LDG      plain ld.global: each thread issues K independent 16-byte
 *               loads per iteration before consuming them (paper §3 "The axis
 *               K"; §4.2 primary cell: .cg, 16 B).
 *   SL_CPASYNC  cp.async 16-byte copies into shared memory with D commit
 *               groups in flight (paper §4.3 compares cp.async with plain
 *               loads).
 *   SL_TMA      Blackwell bulk-async copies (cp.async.bulk) of whole stages
 *               through an mbarrier ring of `stages` stages per CTA, read by
 *               all of the CTA's warps or dealt to them (sl_tma_ring) (paper
 *               §2 names the TMA and bulk copies; the paper has no TMA
 *               kernel, the rings are this library's design).
 *
 * and two layered forms: float payloads (FP32 / BF16 / FP8-E4M3) summed with
 * compensated FP32 accumulation (every addition's rounding error recovered
 * with TwoSum) and an FP64 final combine, and a batched form (many
 * buffers, one CUDA-graph launch) declared further below.
 *
 * Conventions for every function:
 *   - Return an int status: SL_OK (0) or a negative SL_ERR_* code.  They never
 *     abort, trap or print; sl_last_error() returns a message for the calling
 *     thread's most recent failure.
 *   - Device pointers are CUDA device addresses (e.g. torch tensor
 *     data_ptr()) on the CURRENT device; the caller owns them and keeps them
 *     alive until the call returns (sl_run, sl_sweep, sl_run_host) or until
 *     the enqueued work completes (sl_enqueue).
 *   - The library owns its scratch memory (per-warp partials, timestamps, an
 *     error word, an L2-flush buffer, staging buffers, events), allocated
 *     lazily per device and kept until process exit.  Calls that use scratch
 *     on one device must be ordered: issue them from one host thread at a time
 *     and on one stream at a time (work on two streams at once races on the
 *     scratch).
 *   - Byte counts must be multiples of 16 and buffers 16-byte aligned
 *     (SL_ERR_ALIGN otherwise); a zero byte count is valid and gives an all-
 *     zero result.
 */
#ifndef STREAMLOAD_H
#define STREAMLOAD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define SL_OK              0
#define SL_ERR_ARG        -1  /* null pointer, bad enum, K/D/stages/cta out of range */
#define SL_ERR_ALIGN      -2  /* buffer not 16-byte aligned, bytes not a multiple of 16 */
#define SL_ERR_INFEASIBLE -3  /* configuration cannot launch: shared memory or
                                 registers exceed the limit, zero occupancy, or
                                 stage size not 4/16/64 KiB */
#define SL_ERR_TIMEOUT    -4  /* a bounded device wait gave up (TMA ring) */
#define SL_ERR_CUDA       -5  /* a CUDA runtime error; see sl_last_error() */
#define SL_ERR_OOM        -6  /* scratch allocation failed */
#define SL_ERR_NODEV      -7  /* no CUDA device */

/* ---- enums ------------------------------------------------------------ */
typedef enum { SL_U32 = 0, SL_F32 = 1, SL_BF16 = 2, SL_FP8_E4M3 = 3 } sl_dtype;
/* SL_LDSTS: the matched plain-load kernel of paper §4.3 -- G independent
 * 16-byte ld.global per thread, stored to the thread's shared-memory slots
 * with st.shared, read back and folded (cp.async's round trip with the data
 * passing through registers); G = k, 1..16. */
/* SL_LDG4: paper §4.1's streaming-read qualification row -- K independent
 * 4-byte ld.global.cg per thread per iteration (the paper's gate is K = 1);
 * uint32 payloads, K in {1,2,4,8,16}, cta 128/256/512/1024, SL_COP_CG, no
 * SL_DYN.  Its issued_loads counts 4-byte loads: passes*bytes/4. */
/* SL_LDG32: the 32-byte width (256-bit ld.global.cg.v8.u32, sm_100 class):
 * K independent 32-byte loads per thread per iteration, K in {1,2,3,4,6,8},
 * cta 128/256/512, every dtype, SL_ASC / SL_DESC / SL_DYN, SL_COP_CG; the
 * buffer must be 32-byte aligned (SL_ERR_ALIGN).  issued_loads counts loads:
 * passes * ceil(bytes/32) (a final 16-byte remainder is one 16-byte load). */
typedef enum { SL_LDG = 0, SL_CPASYNC = 1, SL_TMA = 2, SL_LDSTS = 3, SL_LDG4 = 4, SL_LDG32 = 5 } sl_mech;
/* Traversal of the buffer by the CTAs.  SL_ASC / SL_DESC: CTA b takes tiles
 * b, b+grid, ... from the first (or last) tile on (the paper's layout).
 * SL_DYN (SL_LDG, SL_LDG32 and SL_CPASYNC): CTAs claim contiguous chunks of
 * about 1 MiB from an atomic counter; integer results are exact, float sums
 * meet the same bound but are not bit-reproducible between runs. */
typedef enum { SL_ASC = 0, SL_DESC = 1, SL_DYN = 2 } sl_order;
/* LDG load flavour: SL_COP_CG is the paper's primary cell (ld.global.cg,
 * §4.2); the other two ask L2 for 256-byte prefetch granules. */
typedef enum { SL_COP_CG = 0, SL_COP_CG_L2_256 = 1, SL_COP_NC_NA_L2_256 = 2 } sl_cop;

#define SL_MAX_K 16
#define SL_MAX_D 16
#define SL_MIN_STAGES 2
#define SL_MAX_STAGES 8

/* ---- launch configuration ---------------------------------------------- */
typedef struct sl_config {
    int32_t mech;        /* sl_mech */
    int32_t k;           /* SL_LDG: K = independent 16-byte loads per thread per
                            iteration, 1..16.  SL_CPASYNC: D = commit groups in
                            flight per thread, 1..16 (of `copies` each).  SL_LDSTS: G = loads per
                            thread staged through shared memory, 1..16.
                            SL_LDG4 / SL_LDG32: K loads of 4 / 32 bytes.
                            SL_TMA: ignored. */
    int32_t stage_bytes; /* SL_TMA: bytes per ring stage, 4096, 16384 or 65536 */
    int32_t stages;      /* SL_TMA: ring depth, 2..8 */
    int32_t cta;         /* threads per CTA that fold loads, a multiple of 32:
                            32..1024 for LDG/CPASYNC (LDG with K > 8: up to 512);
                            TMA: 32..992 with SL_RING_CTA, which adds one
                            producer warp; with SL_RING_WARP, cta/32 must
                            divide `stages`. */
    int32_t grid;        /* CTAs; <= 0 selects min(4, resident CTAs per SM) x SMs */
    int32_t order;       /* sl_order: traversal of the tiles; never changes the
                            integer result */
    int32_t flush_l2;    /* nonzero: overwrite a scratch buffer of twice the L2
                            size before the launch, outside the timed interval */
    int32_t passes;      /* read the buffer this many times, >= 1 (0 means 1) */
    int32_t cop;         /* sl_cop, SL_LDG only */
    int32_t debug_flags; /* 0 in normal use; SL_DEBUG_TMA_SKIP_STAGE makes the
                            TMA producer leave one stage unarmed so that the
                            consumers' bounded wait expires (failure-detection
                            test: the call returns SL_ERR_TIMEOUT and the CUDA
                            context stays usable) */
    int32_t host_direct; /* sl_run_host only: nonzero = the load kernel reads the
                            host buffer directly over the CPU-GPU link (pinned
                            memory, or pageable memory where the device can
                            address it), with no staging copies */
    int32_t tma_ring;    /* SL_TMA only: sl_tma_ring, how the stages are shared */
    int32_t copies;      /* SL_CPASYNC only: G = 16-byte copies a thread puts in
                            each commit group, 1 (0 means 1; the paper's cell),
                            2, 4 or 8, with D x G <= 16.  A tile is cta*D*G
                            vectors; a thread keeps D*G*16 bytes in flight and
                            pays one commit and one wait per G copies.  Other
                            mechanisms and the batched form: 0 or 1
                            (SL_ERR_ARG otherwise). */
    uint64_t target_loads; /* 0 (default): exact fixed work, every vector read
                            once per pass.  > 0: the paper's fixed-iteration
                            control (§3 "Fixed-work control"): every thread runs
                            iters = floor(target_loads / (grid*cta*K)) iterations
                            of K 16-byte loads, wrapping around the buffer
                            (global tile g covers vectors g*cta*K .. (g+1)*cta*K-1
                            mod bytes/16), so issued_loads = iters*grid*cta*K.
                            SL_LDG with SL_ASC / SL_DESC, uint32 payloads, cta
                            256/512/1024, passes <= 1, buffer of at least one
                            tile (SL_ERR_ARG otherwise). */
    void*   stream;      /* cudaStream_t to launch on; NULL = legacy default stream */
} sl_config;

/* Layout of the TMA rings (SL_TMA).
 *   SL_RING_CTA:  one ring of `stages` stages of stage_bytes per CTA, filled by
 *                 a dedicated producer warp (one elected lane issues every bulk
 *                 copy) and read by all cta/32 consumer warps together: each
 *                 stage costs every consumer warp one full-barrier wait and one
 *                 empty-barrier arrive.  Dynamic shared memory stages *
 *                 stage_bytes.
 *   SL_RING_WARP: the same CTA ring of `stages` stages, dealt to the CTA's
 *                 cta/32 warps (no producer warp): each warp owns stages /
 *                 (cta/32) stages, filled by its own lane 0 and read by its
 *                 own 32 lanes only, so a stage costs one wait per warp and no
 *                 cross-warp synchronisation (small stages no longer pay a
 *                 CTA-wide protocol per 16 bytes a thread reads; a 4 KiB stage
 *                 gives each lane 8 vectors).  Chunks are dealt to warps
 *                 grid-wide.  Dynamic shared memory stages * (stage_bytes +
 *                 8). */
typedef enum { SL_RING_CTA = 0, SL_RING_WARP = 1 } sl_tma_ring;

#define SL_DEBUG_TMA_SKIP_STAGE 1
/* Experiment knob for SL_CPASYNC and SL_LDSTS: place the shared-memory ring n
 * x 16 bytes (n = 0..7) past a 128-byte boundary instead of on it, to measure
 * how the destination alignment of cp.async changes its L2 requests. */
#define SL_DEBUG_SMEM_SKEW_SHIFT 8
#define SL_DEBUG_SMEM_SKEW(n) (((n) & 7) << SL_DEBUG_SMEM_SKEW_SHIFT)

/* ---- results ----------------------------------------------------------- */
typedef struct sl_result {
    uint64_t xor_u64;         /* XOR of the little-endian uint64 words read */
    uint64_t issued_loads;    /* 16-byte logical loads folded; = passes*bytes/16
                                 (SL_LDG4: 4-byte loads, passes*bytes/4;
                                 SL_LDG32: passes*ceil(bytes/32)) */
    uint64_t device_ns;       /* CUDA-event time of the load kernel (sl_run);
                                 of the whole call (sl_run_host); 0 (sl_enqueue) */
    uint64_t window_ns;       /* %globaltimer: first CTA start to last CTA end */
    double   fsum;            /* float dtypes: sum of the decoded payload */
    float    fsum_hi;         /* fsum as a float pair: hi = fl(fsum) */
    float    fsum_lo;         /*                       lo = fl(fsum - hi) */
    uint32_t sum_u32;         /* sum of the uint32 words read, mod 2^32 */
    int32_t  status;          /* SL_OK or SL_ERR_TIMEOUT (device-reported) */
    int32_t  grid;            /* CTAs launched */
    int32_t  cta;             /* threads per CTA launched (TMA: incl. producer warp) */
    int32_t  resident_per_sm; /* occupancy-API residency of this launch shape */
    int32_t  smem_bytes;      /* dynamic shared memory per CTA */
} sl_result;

typedef struct sl_devinfo {
    int32_t device;
    int32_t sm_count;
    int32_t cc_major;
    int32_t cc_minor;
    int64_t l2_bytes;
    int64_t smem_per_block_optin;
    int64_t smem_per_sm;
    int64_t global_mem_bytes;
    int32_t max_threads_per_sm;
    int32_t regs_per_sm;
    int32_t clock_khz;        /* 0 where the runtime no longer reports it */
    int32_t mem_clock_khz;    /* 0 where the runtime no longer reports it */
    int32_t mem_bus_bits;
    int32_t driver_version;
    int32_t runtime_version;
    int32_t reserved;
    char    name[256];
} sl_devinfo;

/* ---- device, errors ---------------------------------------------------- */

/* Properties of the current device (paper §3 "Environment" capture). */
int sl_device_info(sl_devinfo* out);

/* Message of the calling thread's most recent failed call ("" if none).  The
 * pointer stays valid until the next call from the same thread. */
const char* sl_last_error(void);

/* ---- inputs and cache state -------------------------------------------- */

/* Fill a device buffer with the splitmix64 stream seeded with `seed`
 * (Steele, Lea and Flood 2014; counter form: output m = mix(seed +
 * (m+1)*0x9E3779B97F4A7C15)); uint32 word 2m / 2m+1 is the low / high half
 * of output m.  `bytes` a multiple of 16.  Asynchronous on `stream`. */
int sl_fill_splitmix64(void* dev_buf, uint64_t bytes, uint64_t seed, void* stream);

/* Overwrite the library's L2-flush buffer (twice the L2 size) so that no part
 * of a previously read buffer stays L2-resident.  Asynchronous on `stream`. */
int sl_flush_l2(void* stream);

/* ---- the streaming checksum ------------------------------------------- */

/* Resolve a configuration without launching: fills grid, cta,
 * resident_per_sm and smem_bytes of *out (other fields zero) or returns
 * SL_ERR_ARG / SL_ERR_ALIGN / SL_ERR_INFEASIBLE.  Used by sweeps to record
 * infeasible cells. */
int sl_plan(uint64_t bytes, int32_t dtype, const sl_config* cfg, sl_result* out);

/* One streaming pass set over dev_buf[0, bytes): the call
 * sl_run(buf, bytes, dtype, mech, K or D, cta, grid, order) -> checksum,
 * device ns, issued-load count.  Tiles: LDG and CPASYNC walk tiles of
 * cta*K (or cta*D) 16-byte vectors, CTA b taking tiles b, b+grid, ...
 * (paper §3: each warp's access is contiguous and fully coalesced at every
 * K); load k of thread t reads vector tile*cta*K + k*cta + t; the last tile is
 * guarded so that issued loads = passes*bytes/16 exactly at every K.  TMA
 * walks stage-sized chunks the same way.  dtype selects the fold: SL_U32
 * computes sum_u32 / xor_u64; float dtypes also compute fsum (per-thread
 * compensated FP32 sum -- FP32 and BF16: every element; FP8: the two exact
 * sums of each half vector -- with each addition's error recovered by TwoSum,
 * double-float merges of warps and CTAs, FP64 combine of per-CTA partials).  Synchronous: returns
 * after the result is on the host. */
int sl_run(const void* dev_buf, uint64_t bytes, int32_t dtype, const sl_config* cfg,
           sl_result* out);

/* As sl_run but asynchronous on cfg->stream: enqueues [L2 flush] and the
 * load kernel, whose last CTA to finish combines all per-CTA partials (FP64
 * for float sums) and writes an sl_result (device_ns and the launch-shape
 * fields are 0) to the DEVICE pointer dev_out (8-byte aligned).  Successive enqueues on one stream may share the
 * library's scratch; enqueues on different streams at once race. */
int sl_enqueue(const void* dev_buf, uint64_t bytes, int32_t dtype, const sl_config* cfg,
               sl_result* dev_out);

/* Enqueue `steps` (>= 1) back-to-back passes of one configuration on
 * cfg->stream: pass i reads dev_bufs[i % nbufs] (nbufs >= 1 buffers of
 * `bytes` each, e.g. two copies so that consecutive passes never read the
 * same lines) and writes its sl_result to dev_out[i] (DEVICE pointer, 8-byte
 * aligned, room for `steps` results).  Pass 0 is launched like sl_enqueue;
 * passes 1.. are programmatic dependent launches of the pass before them: a
 * pass's CTAs may start while the previous pass's last CTAs are still
 * running (the buffers are only read), and touch the library's scratch only
 * after that pass has completed -- so each pass's result is the same as a
 * separate sl_enqueue's, and the passes' ramp-up and tail overlap.  Every
 * pass runs one full wave (grid = resident CTAs per SM x SMs; cfg->grid must
 * be 0 or that number), so a pass's CTAs get SM slots only as the previous
 * pass's CTAs exit.  Every mechanism and traversal (SL_DYN passes claim
 * chunks from a counter of their own, zeroed in stream order before every
 * 4,096 passes, where one ordinary launch restarts the overlap; SL_TMA
 * publishes a bounded wait's error only when the CTA finishes), with
 * flush_l2 == 0.  No paper counterpart: the paper times one launch per
 * cell. */
int sl_enqueue_steps(const void* const* dev_bufs, int32_t nbufs, uint64_t bytes, int32_t dtype,
                     const sl_config* cfg, int32_t steps, sl_result* dev_out);

/* Sweep (paper §3 "Fixed-work control": run each K sweep ascending and
 * reversed; the warm-up launch is excluded as in §3 "Hardware counters").
 * Runs the ncells configurations in cell order (sweep_order = SL_ASC) or in
 * reverse (SL_DESC); for each cell `warmup` discarded runs then `repeats`
 * timed sl_run calls.  Row out[c*repeats + r] holds cell c's r-th repeat
 * whatever the sweep order.  An infeasible cell fills its rows with status
 * SL_ERR_INFEASIBLE and the sweep continues; a CUDA error stops it. */
int sl_sweep(const void* dev_buf, uint64_t bytes, int32_t dtype, const sl_config* cells,
             int32_t ncells, int32_t repeats, int32_t warmup, int32_t sweep_order,
             sl_result* out);

/* End-to-end form: the payload is in HOST memory (page-locked for full
 * speed).  Staged mode (cfg->host_direct == 0): copies it to a library-owned
 * device staging ring in chunks of 256 MiB on a copy stream, overlapped with
 * the load kernel on each chunk, then combines all chunks.  Direct mode
 * (cfg->host_direct != 0): one load kernel reads the host buffer in place
 * through its device mapping (SL_ERR_ARG if the device cannot address it).
 * Either way the result is copied back and device_ns covers the whole call
 * (first transfer to result on the host).  Synchronous. */
int sl_run_host(const void* host_buf, uint64_t bytes, int32_t dtype, const sl_config* cfg,
                sl_result* out);

/* ---- pointer-chase latency probe ---------------------------------------- */

typedef struct sl_chase_result {
    uint32_t final_index;    /* word index reached after warm + hops steps */
    uint32_t reserved;
    uint64_t hops;           /* timed steps */
    uint64_t ns;             /* %globaltimer over the timed steps */
    uint64_t cycles;         /* clock64 (SM cycles) over the timed steps */
    double   ns_per_hop;
    double   cycles_per_hop;
} sl_chase_result;

/* Unloaded load latency (paper §4.1 "Primitive baseline": a dependent pointer
 * chain on a single SM, .ca and .cg).  dev_chain holds uint32 word indices:
 * from word `start`, one thread replaces the index by the word it points to,
 * first `warm` untimed steps (to bring the chain into the cache level that
 * holds it), then `hops` timed steps; each load depends on the previous one.
 * cache_l1 nonzero loads with ld.global.ca (L1-allocating), else .cg (L2).
 * bytes: chain size (a multiple of 4).  SL_ERR_ARG if an index leaves the
 * chain.  Synchronous on `stream`.  Chains come from any generator; the
 * library's tests use one random cycle through every element. */
int sl_chase(const void* dev_chain, uint64_t bytes, uint32_t start, uint64_t warm, uint64_t hops, int32_t cache_l1,
             void* stream, sl_chase_result* out);

/* ---- coverage audit ------------------------------------------------------ */

/* As sl_run on a uint32 payload, but with the configuration's coverage
 * instantiation: the same kernel and launch shape, where every load also
 * adds 1 to dev_counts[i] for the 16-byte vector i it reads (a 32-byte load
 * counts both of its vectors; cp.async counts at each copy, TMA at each bulk
 * copy, per 16 bytes).  dev_counts: DEVICE array of bytes/16 uint32 counters,
 * zeroed by the call.  Under exact fixed work every counter ends at `passes`;
 * under the fixed-iteration control at q or q+1 (issued = q*n + r: the first r
 * vectors q+1).  Instantiations exist for: SL_LDG K 1/3/8/16 grid-stride and
 * K 2/12 SL_DYN at cta 128/256/512 (SL_COP_CG); SL_LDG32 K 1/3/8 at cta 256
 * (grid-stride or SL_DYN); the fixed-iteration control at K 2/8, cta 256/1024;
 * SL_CPASYNC D 1/4/16 (one copy per group) and D x G = 2 x 4, 3 x 2; SL_LDSTS
 * G 1/16; SL_TMA (either ring layout) -- SL_ERR_ARG otherwise.  A debug tool (the counting atomics slow the kernel); no paper
 * counterpart. */
int sl_coverage(const void* dev_buf, uint64_t bytes, const sl_config* cfg, uint32_t* dev_counts, sl_result* out);

/* ---- two co-resident streams in one CTA ---------------------------------- */

typedef struct sl_twostream_result {
    uint64_t xor_u64[2];       /* [0] stream A, [1] stream B: as sl_result */
    uint64_t issued_loads[2];  /* 16-byte loads folded: passes*bytes/16 */
    uint64_t window_ns[2];     /* %globaltimer, earliest warp start to latest
                                  warp end of the stream, over all CTAs */
    uint64_t b_first_end_ns;   /* earliest end of a stream-B warp, measured
                                  from stream A's earliest start (0: no B) */
    uint64_t device_ns;        /* CUDA-event time of the load kernel */
    uint32_t sum_u32[2];
    int32_t  grid;             /* CTAs (one per SM) */
    int32_t  cta;              /* threads per CTA = 32*(warps_a + warps_b) */
    int32_t  b_covers_a;       /* 1 if every stream-B warp was still loading when
                                  stream A's last warp finished (or warps_b == 0) */
    int32_t  reserved;
} sl_twostream_result;

/* Two plain-load streams in the same CTA (paper §4.4): one CTA per SM with
 * warps_a warps reading buf_a (bytes_a, one pass) and, after them, warps_b
 * warps reading buf_b (bytes_b, passes_b passes), both with the LDG loop at
 * K independent 16-byte ld.global.cg per thread (K in {1,2,4,8}).  Stream A's
 * bandwidth is bytes_a / window_ns[0]; compared with the same call at
 * warps_b = 0 it gives A's displacement by B.  Size B's work (passes_b) so
 * that b_covers_a is 1, or the B load ended before A did.
 * Arguments: warps_a >= 1, warps_b >= 0, warps_a + warps_b <= 32; buffers
 * 16-byte aligned, bytes multiples of 16, bytes_a > 0, bytes_b > 0 when
 * warps_b > 0 (SL_ERR_ARG / SL_ERR_ALIGN otherwise).  flush_l2 nonzero
 * overwrites an L2-sized scratch buffer first (untimed).  Synchronous on
 * `stream`.  The buffers stay caller-owned; the library's scratch is reused. */
int sl_twostream(const void* buf_a, uint64_t bytes_a, const void* buf_b, uint64_t bytes_b, int32_t passes_b,
                 int32_t warps_a, int32_t warps_b, int32_t k, int32_t flush_l2, void* stream,
                 sl_twostream_result* out);

/* ---- batched form -------------------------------------------------------- */

/* One device buffer of a batch (24 bytes). */
typedef struct sl_batch_desc {
    const void* ptr;    /* device address, 16-byte aligned (caller-owned) */
    uint64_t    bytes;  /* a multiple of 16; 0 gives an all-zero result */
    int32_t     dtype;  /* sl_dtype */
    int32_t     reserved;
} sl_batch_desc;

/* One size class of the tuning table: buffers with min_bytes <= bytes <=
 * max_bytes (and dtype == dtype, or dtype == -1 for any) run with cfg.  In
 * cfg: mech, k (LDG K in {1,2,3,4,6,8,12,16}, cp.async D 1..8), stage_bytes,
 * stages, cta (LDG: 128/256/512) and grid (<= 0: resident CTAs per SM x
 * SMs, a persistent grid) are used (TMA classes run one ring per CTA:
 * tma_ring must be SL_RING_CTA; cp.async classes put one copy in each commit
 * group: copies must be 0 or 1); order, passes, flush_l2, cop, debug_flags
 * and stream are ignored. */
typedef struct sl_tune_entry {
    uint64_t  min_bytes;
    uint64_t  max_bytes;
    int32_t   dtype;
    int32_t   reserved;
    sl_config cfg;
} sl_tune_entry;

typedef struct sl_batch sl_batch;  /* opaque */

/* Build a batched streaming checksum over n buffers (the batched form: a
 * persistent kernel per size class streaming many uneven buffers, in one
 * CUDA-graph launch; no paper counterpart).  Each buffer goes to the first
 * table entry that matches it (SL_ERR_ARG if none).  Buffers are cut into
 * work items of at most 1 MiB; each class kernel runs a persistent grid whose
 * CTAs claim items from an atomic counter, fold them with the class's
 * mechanism and write one partial per warp per item; a combine kernel with
 * one warp per buffer adds each buffer's partials (integer parts exactly,
 * float parts in FP64, in a fixed order) into its sl_result.  The graph --
 * a memset of the counters, the class kernels as parallel branches, then the
 * combine -- is captured once here and replayed by sl_batch_run.  The batch
 * owns its device tables, results, streams and graph until sl_batch_destroy;
 * the caller keeps the buffers alive and unchanged in size.  Asynchronous
 * work of other calls must not overlap a batch run on the same buffers'
 * device (the class kernels may fill the whole GPU). */
int sl_batch_create(const sl_batch_desc* descs, int32_t n, const sl_tune_entry* table, int32_t ntable,
                    sl_batch** out);

/* Launch the batch's graph once and wait.  per_buffer (host, n entries, may
 * be NULL to skip the copy-back) receives each buffer's result in descriptor
 * order (device_ns = 0 in each); *total_ns (may be NULL) receives the
 * CUDA-event time of the whole graph launch.  Returns SL_ERR_TIMEOUT if a
 * bounded device wait gave up during the run (with or without per_buffer). */
int sl_batch_run(sl_batch* b, sl_result* per_buffer, uint64_t* total_ns);

/* Number of class kernels (graph kernel nodes besides the combine) and the
 * class each buffer went to (host array of n, may be NULL). */
int sl_batch_info(const sl_batch* b, int32_t* nclasses, int32_t* class_of_buffer);

void sl_batch_destroy(sl_batch* b);

/* ---- allocation-free variant ------------------------------------------- */

/* The paper has no counterpart to this entry point; it exists for callers of
 * this library that cannot allocate device memory: code running under a
 * framework whose own pool allocator owns (nearly) all device memory, code in
 * a latency-critical loop where cudaMalloc/cudaFree may synchronize the
 * device, or a plugin or callback whose host contract forbids allocating.
 * The other entry points allocate their scratch lazily and may grow it.
 *
 * sl_run_noalloc runs the LDG mechanism (cfg->mech must be SL_LDG; no L2
 * flush, no debug flags) like sl_enqueue: asynchronous on cfg->stream, the
 * result written to the DEVICE pointer dev_out (8-byte aligned), computing
 * the same checksum, issued-load count and float sum as sl_run.  It calls no
 * cudaMalloc, cudaFree or other allocating routine.  Its scratch (one
 * 32-byte partial per CTA plus a 256-byte control block: the timing window,
 * the finished-CTA counter and the error word) is one fixed file-scope
 * __device__ array of SL_NOALLOC_SCRATCH_BYTES bytes, held by every GPU that
 * loads the library until the process exits.  Limit: at most SL_NOALLOC_MAX_CTAS CTAs
 * per call; larger launches are rejected with SL_ERR_ARG and a message.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  The address is kept per device together with
 * the driver's id of the context it was looked up in, and looked up again by
 * the first call after that context has been replaced (e.g. by
 * cudaDeviceReset).  Every call on a device shares the one array,
 * which keeps the previous call's contents (the error word is cleared by each
 * call): calls whose work overlaps on the GPU (different streams, or other
 * threads) race and must be serialized by the caller. */
#define SL_NOALLOC_MAX_CTAS 4096
#define SL_NOALLOC_SCRATCH_BYTES (SL_NOALLOC_MAX_CTAS * 32 + 256)
int sl_run_noalloc(const void* dev_buf, uint64_t bytes, int32_t dtype, const sl_config* cfg,
                   sl_result* dev_out);

#ifdef __cplusplus
}
#endif

#endif /* STREAMLOAD_H */
