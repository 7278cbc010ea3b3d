"""GB300 (sm_103a) streaming global-load library: Python binding.

The functions below carry the C ABI's names (include/streamload.h) and only
marshal arguments; every step of the path -- loading, folding, reducing,
timing -- runs in ``libstreamload.so``.  PyTorch is used for device memory and
streams: pass CUDA tensors (or raw device addresses) and, optionally, a
``torch.cuda.Stream``.

    import torch, paper_2608_15764_gb300 as sl
    buf = torch.empty(1 << 28, dtype=torch.uint8, device="cuda")
    sl.sl_fill_splitmix64(buf, seed=1)
    r = sl.sl_run(buf, dtype=sl.SL_U32, cfg=sl.config("ldg", k=2, cta=256))
    print(r.sum_u32, r.xor_u64, r.issued_loads, r.device_ns)
"""
from __future__ import annotations

import ctypes

from ._abi import (  # noqa: F401  (re-exported constants)
    SL_ASC, SL_BF16, SL_COP_CG, SL_COP_CG_L2_256, SL_COP_NC_NA_L2_256, SL_CPASYNC,
    SL_DEBUG_SMEM_SKEW, SL_DEBUG_TMA_SKIP_STAGE, SL_DESC, SL_DYN, SL_ERR_ALIGN, SL_ERR_ARG, SL_ERR_CUDA, SL_ERR_INFEASIBLE,
    SL_ERR_NODEV, SL_ERR_OOM, SL_ERR_TIMEOUT, SL_F32, SL_FP8_E4M3, SL_LDG, SL_LDG4, SL_LDG32, SL_LDSTS, SL_MAX_D, SL_MAX_K,
    SL_MAX_STAGES, SL_MIN_STAGES, SL_NOALLOC_MAX_CTAS, SL_OK, SL_RING_CTA, SL_RING_WARP, SL_TMA, SL_U32,
    STATUS_NAMES, RESULT_BYTES, load, sl_batch_desc, sl_chase_result, sl_config, sl_devinfo, sl_result,
    sl_tune_entry, sl_twostream_result,
)

MECHS = {"ldg": SL_LDG, "cpasync": SL_CPASYNC, "tma": SL_TMA, "ldsts": SL_LDSTS, "ldg4": SL_LDG4, "ldg32": SL_LDG32}
DTYPES = {"u32": SL_U32, "f32": SL_F32, "bf16": SL_BF16, "fp8": SL_FP8_E4M3}
ORDERS = {"asc": SL_ASC, "desc": SL_DESC, "dyn": SL_DYN}
RINGS = {"cta": SL_RING_CTA, "warp": SL_RING_WARP}


class SLError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _check(status: int) -> int:
    if status != SL_OK:
        raise SLError(status, load().sl_last_error().decode(errors="replace"))
    return status


def _addr(buf) -> int:
    if buf is None:
        return 0
    if isinstance(buf, int):
        return buf
    if hasattr(buf, "data_ptr"):
        return int(buf.data_ptr())
    if hasattr(buf, "ctypes"):  # numpy array (host memory)
        return int(buf.ctypes.data)
    raise TypeError(f"cannot take the address of {type(buf).__name__}")


def _nbytes(buf, nbytes):
    if nbytes is not None:
        return int(nbytes)
    if hasattr(buf, "nbytes"):
        return int(buf.nbytes)
    if hasattr(buf, "element_size"):
        return int(buf.numel() * buf.element_size())
    raise TypeError("nbytes is required for a raw address")


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return int(torch.cuda.current_stream().cuda_stream) or None
        except Exception:  # pragma: no cover
            pass
        return None
    if isinstance(stream, int):
        return stream or None
    return int(stream.cuda_stream) or None


def config(mech="ldg", k: int = 2, cta: int = 256, grid: int = 0, order="asc", *, stage_bytes: int = 16384,
           stages: int = 4, flush_l2: bool = False, passes: int = 1, cop: int = SL_COP_CG,
           debug_flags: int = 0, host_direct: bool = False, target_loads: int = 0, ring="cta",
           copies: int = 1, stream=None) -> sl_config:
    """Build an sl_config.  mech: "ldg" / "cpasync" / "tma" (or the enum);
    k: K for LDG, depth D for cp.async; copies: G, the 16-byte copies per
    cp.async commit group (1, 2, 4 or 8, D*G <= 16); stage_bytes/stages/ring
    for TMA (ring "cta": the CTA's stages read by all its consumer warps,
    filled by a producer warp; "warp": the CTA's stages dealt to its warps,
    cta/32 dividing stages)."""
    c = sl_config()
    c.mech = MECHS[mech] if isinstance(mech, str) else int(mech)
    c.k = int(k)
    c.stage_bytes = int(stage_bytes)
    c.stages = int(stages)
    c.cta = int(cta)
    c.grid = int(grid)
    c.order = ORDERS[order] if isinstance(order, str) else int(order)
    c.flush_l2 = int(bool(flush_l2))
    c.passes = int(passes)
    c.cop = int(cop)
    c.debug_flags = int(debug_flags)
    c.host_direct = int(bool(host_direct))
    c.target_loads = int(target_loads)
    c.tma_ring = RINGS[ring] if isinstance(ring, str) else int(ring)
    c.copies = int(copies)
    c.stream = _stream_handle(stream)
    return c


def _dtype(dtype) -> int:
    return DTYPES[dtype] if isinstance(dtype, str) else int(dtype)


def sl_device_info() -> dict:
    info = sl_devinfo()
    _check(load().sl_device_info(ctypes.byref(info)))
    return info.as_dict()


def sl_last_error() -> str:
    return load().sl_last_error().decode(errors="replace")


def sl_fill_splitmix64(buf, nbytes=None, seed: int = 1, stream=None) -> None:
    _check(load().sl_fill_splitmix64(_addr(buf), _nbytes(buf, nbytes), seed, _stream_handle(stream)))


def sl_flush_l2(stream=None) -> None:
    _check(load().sl_flush_l2(_stream_handle(stream)))


def sl_plan(nbytes: int, dtype=SL_U32, cfg: sl_config | None = None) -> sl_result:
    """Resolve a configuration without launching; raises SLError if it is
    infeasible or invalid."""
    cfg = cfg or config()
    r = sl_result()
    _check(load().sl_plan(int(nbytes), _dtype(dtype), ctypes.byref(cfg), ctypes.byref(r)))
    return r


def sl_run(buf, nbytes=None, dtype=SL_U32, cfg: sl_config | None = None) -> sl_result:
    cfg = cfg or config()
    r = sl_result()
    _check(load().sl_run(_addr(buf), _nbytes(buf, nbytes), _dtype(dtype), ctypes.byref(cfg), ctypes.byref(r)))
    return r


def sl_enqueue(buf, dev_out, nbytes=None, dtype=SL_U32, cfg: sl_config | None = None) -> None:
    """Asynchronous form: dev_out is a device buffer of at least RESULT_BYTES
    (one sl_result) that receives the result."""
    cfg = cfg or config()
    _check(load().sl_enqueue(_addr(buf), _nbytes(buf, nbytes), _dtype(dtype), ctypes.byref(cfg), _addr(dev_out)))


def sl_coverage(buf, counts, nbytes=None, cfg: sl_config | None = None) -> sl_result:
    """Coverage audit of a uint32 run: counts (a device array of nbytes/16
    uint32, zeroed by the call) receives how many times each 16-byte vector
    was loaded."""
    cfg = cfg or config()
    r = sl_result()
    _check(load().sl_coverage(_addr(buf), _nbytes(buf, nbytes), ctypes.byref(cfg), _addr(counts), ctypes.byref(r)))
    return r


def sl_enqueue_steps(bufs, dev_out, steps: int, nbytes=None, dtype=SL_U32, cfg: sl_config | None = None) -> None:
    """`steps` back-to-back passes on cfg.stream, pass i reading bufs[i %
    len(bufs)] (one buffer or a list of equal-size buffers) and writing its
    result to the i-th RESULT_BYTES slot of the device buffer dev_out; passes
    after the first are programmatic dependent launches (their start overlaps
    the previous pass's tail), each one full wave of CTAs."""
    cfg = cfg or config()
    if not isinstance(bufs, (list, tuple)):
        bufs = [bufs]
    arr = (ctypes.c_void_p * len(bufs))(*[_addr(b) for b in bufs])
    _check(load().sl_enqueue_steps(arr, len(bufs), _nbytes(bufs[0], nbytes), _dtype(dtype), ctypes.byref(cfg),
                                   int(steps), _addr(dev_out)))


def sl_sweep(buf, cells, nbytes=None, dtype=SL_U32, repeats: int = 1, warmup: int = 1,
             sweep_order=SL_ASC) -> list[list[sl_result]]:
    """Returns rows[cell][repeat] (in cell order whatever the sweep order)."""
    n = len(cells)
    arr = (sl_config * n)(*cells)
    out = (sl_result * (n * repeats))()
    order = ORDERS[sweep_order] if isinstance(sweep_order, str) else int(sweep_order)
    _check(load().sl_sweep(_addr(buf), _nbytes(buf, nbytes), _dtype(dtype), arr, n, repeats, warmup, order, out))
    return [[out[c * repeats + r] for r in range(repeats)] for c in range(n)]


def sl_run_host(host_buf, nbytes=None, dtype=SL_U32, cfg: sl_config | None = None) -> sl_result:
    """End-to-end form over a HOST buffer (numpy array, pinned torch tensor or
    address)."""
    cfg = cfg or config()
    r = sl_result()
    _check(load().sl_run_host(_addr(host_buf), _nbytes(host_buf, nbytes), _dtype(dtype), ctypes.byref(cfg),
                              ctypes.byref(r)))
    return r


def sl_run_noalloc(buf, dev_out, nbytes=None, dtype=SL_U32, cfg: sl_config | None = None) -> None:
    """Allocation-free LDG checksum for callers that cannot allocate device
    memory (a framework pool that owns the memory, a latency-critical loop,
    a no-allocation plugin contract).  Like sl_enqueue: asynchronous, result
    written to the device buffer dev_out (RESULT_BYTES).  Scratch is a fixed
    device array shared by every call on the device: calls that overlap on
    the GPU race.  Launches above SL_NOALLOC_MAX_CTAS CTAs are rejected."""
    cfg = cfg or config()
    _check(load().sl_run_noalloc(_addr(buf), _nbytes(buf, nbytes), _dtype(dtype), ctypes.byref(cfg),
                                 _addr(dev_out)))


def tune_entry(min_bytes: int, max_bytes: int, cfg: sl_config, dtype: int = -1) -> sl_tune_entry:
    """One size class of a batch's tuning table (dtype -1 matches any)."""
    e = sl_tune_entry()
    e.min_bytes = int(min_bytes)
    e.max_bytes = int(max_bytes)
    e.dtype = int(dtype)
    e.cfg = cfg
    return e


class sl_batch:
    """Handle of a batch built by sl_batch_create (sl_batch_destroy frees it;
    so does garbage collection)."""

    def __init__(self, handle: int, n: int, nbytes: int, keepalive):
        self.handle = handle
        self.n = n
        self.nbytes = nbytes
        self._keep = keepalive

    def __del__(self):
        try:
            sl_batch_destroy(self)
        except Exception:  # pragma: no cover
            pass


def sl_batch_create(buffers, table) -> sl_batch:
    """buffers: sequence of (device buffer or address, nbytes, dtype);
    table: sequence of sl_tune_entry (see tune_entry)."""
    n = len(buffers)
    descs = (sl_batch_desc * max(n, 1))()
    total = 0
    for i, (buf, nb, dt) in enumerate(buffers):
        descs[i].ptr = _addr(buf)
        descs[i].bytes = int(nb)
        descs[i].dtype = _dtype(dt)
        total += int(nb)
    tab = (sl_tune_entry * len(table))(*table)
    h = ctypes.c_void_p()
    _check(load().sl_batch_create(descs, n, tab, len(table), ctypes.byref(h)))
    return sl_batch(h.value, n, total, [b for b, _, _ in buffers])


def sl_batch_run(b: sl_batch, results: bool = True):
    """Launch the batch's graph once; returns (list of per-buffer sl_result or
    None, device ns of the graph launch)."""
    out = (sl_result * max(b.n, 1))() if results else None
    ns = ctypes.c_uint64()
    _check(load().sl_batch_run(b.handle, out, ctypes.byref(ns)))
    return ([out[i] for i in range(b.n)] if results else None), int(ns.value)


def sl_batch_info(b: sl_batch):
    """(number of class kernels, class index of every buffer)."""
    nc = ctypes.c_int32()
    cls = (ctypes.c_int32 * max(b.n, 1))()
    _check(load().sl_batch_info(b.handle, ctypes.byref(nc), cls))
    return int(nc.value), [cls[i] for i in range(b.n)]


def sl_batch_destroy(b: sl_batch) -> None:
    if b.handle:
        load().sl_batch_destroy(b.handle)
        b.handle = None


def sl_twostream(buf_a, buf_b=None, warps_a: int = 1, warps_b: int = 0, k: int = 2, passes_b: int = 1,
                 flush_l2: bool = True, nbytes_a=None, nbytes_b=None, stream=None) -> sl_twostream_result:
    """Two plain-load streams in one CTA per SM: warps_a warps read buf_a
    once, warps_b warps read buf_b passes_b times (paper §4.4)."""
    r = sl_twostream_result()
    has_b = buf_b is not None
    _check(load().sl_twostream(_addr(buf_a), _nbytes(buf_a, nbytes_a), _addr(buf_b) if has_b else None,
                               _nbytes(buf_b, nbytes_b) if has_b else 0, int(passes_b), int(warps_a), int(warps_b),
                               int(k), int(bool(flush_l2)), _stream_handle(stream), ctypes.byref(r)))
    return r


def sl_chase(chain, start: int = 0, warm: int = 0, hops: int = 1 << 16, cache_l1: bool = False, nbytes=None,
             stream=None) -> sl_chase_result:
    """Pointer-chase latency probe: one thread follows the chain (uint32 word
    indices) `warm` untimed then `hops` timed steps from word `start`."""
    r = sl_chase_result()
    _check(load().sl_chase(_addr(chain), _nbytes(chain, nbytes), int(start), int(warm), int(hops),
                           int(bool(cache_l1)), _stream_handle(stream), ctypes.byref(r)))
    return r
