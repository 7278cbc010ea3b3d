"""Parity at the benchmark's full size: the 4 GiB uint32 splitmix64(seed=1)
buffer, filled on the GPU, in every launch configuration the benchmark
measures (its candidate set, from which it times the fastest, as single
launches and as overlapped back-to-back passes over two copies), checked
bit-exactly against the oracle's checksum of the same words generated on the
host.  Also the 256 MiB LDG cells (K = 1, 2, 4, 8; 256 threads; 4 x SMs) and
the allocation sweep's largest buffer (20 GiB)."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2608_15764_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _oracle_parallel(words):
    t = os.cpu_count() or 1
    per = (words.size // t) // 4 * 4
    cuts = [i * per for i in range(t)] + [words.size]
    with ThreadPoolExecutor(t) as ex:
        return oracle.combine(ex.map(lambda i: oracle.checksum(words[cuts[i]:cuts[i + 1]]), range(t)))


@pytest.fixture(scope="module")
def sl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_15764_gb300 as sl
    sl.load()
    return sl


def _feasible(sl, points, nbytes):
    """The catalogue's points that can launch (the catalogue also lists ring
    sets too large for one CTA's shared memory, recorded as infeasible)."""
    out = []
    for p in points:
        try:
            sl.sl_plan(nbytes, sl.SL_U32, p.cfg())
            out.append(p)
        except sl.SLError as e:
            assert e.status == sl.SL_ERR_INFEASIBLE, p.label()
    return out


@pytest.mark.parametrize("gib", [0.25, 4])
def test_full_size_all_candidates(sl, gib):
    from paper_2608_15764_gb300 import tune
    nbytes = int(gib * (1 << 30))
    dev = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    sl.sl_fill_splitmix64(dev, seed=1)
    want = _oracle_parallel(workloads.splitmix_u32(1, nbytes // 4))
    sms = sl.sl_device_info()["sm_count"]
    points = _feasible(sl, tune.default_points(), nbytes)
    if gib < 1:
        points = [tune.Point(sl.SL_LDG, k=k, cta=256, grid=4 * sms) for k in (1, 2, 4, 8)]
    for p in points:
        # the dynamic-chunk points run in their own traversal (twice: the chunk
        # counter must reset between launches), the others in both orders
        for order in (("dyn", "dyn") if p.order == sl.SL_DYN else ("asc", "desc")):
            r = sl.sl_run(dev, dtype=sl.SL_U32, cfg=p.cfg(order=order))
            assert (r.sum_u32, r.xor_u64) == want, (p.label(), order)
            loads = nbytes // 32 if p.mech == sl.SL_LDG32 else nbytes // 16
            assert r.issued_loads == loads, (p.label(), order)
    del dev
    torch.cuda.empty_cache()


def test_run_host_multi_chunk(sl):
    """The host-buffer entry point over more than two 256 MiB staging chunks
    plus a ragged tail."""
    nbytes = (600 << 20) + 16 * 3
    host = workloads.splitmix_u32(7, nbytes // 4)
    want = _oracle_parallel(host)
    pinned = torch.from_numpy(host.view(np.uint8)).pin_memory()
    for cfg in [sl.config("ldg", k=2), sl.config("cpasync", k=4), sl.config("tma", stage_bytes=65536, stages=3),
                sl.config("ldg", k=16, order="dyn", host_direct=True)]:
        r = sl.sl_run_host(pinned, dtype=sl.SL_U32, cfg=cfg)
        assert (r.sum_u32, r.xor_u64) == want and r.issued_loads == nbytes // 16


def _oracle_generated(seed, nwords, chunk=1 << 26):
    """The oracle's checksum of splitmix64 words [0, nwords), generated and
    folded chunk by chunk on the host threads (no full host copy)."""
    t = os.cpu_count() or 1
    starts = list(range(0, nwords, chunk))

    def one(s):
        return oracle.checksum(workloads.splitmix_u32(seed, min(chunk, nwords - s), first_word=s))
    with ThreadPoolExecutor(t) as ex:
        return oracle.combine(ex.map(one, starts))


def test_overlapped_passes_full_size(sl):
    """The benchmark's timed launch configuration for grid-stride points:
    back-to-back passes as programmatic dependent launches, one full wave per
    pass, alternating between two resident 4 GiB copies."""
    from paper_2608_15764_gb300 import tune
    nbytes = 4 << 30
    bufs = [torch.empty(nbytes, dtype=torch.uint8, device="cuda") for _ in range(2)]
    for b in bufs:
        sl.sl_fill_splitmix64(b, seed=1)
    want = _oracle_generated(1, nbytes // 4)
    steps = 3
    out = torch.zeros(steps * sl.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    for p in [p for p in _feasible(sl, tune.default_points(), nbytes) if p.overlapped]:
        sl.sl_enqueue_steps(bufs, out, steps, dtype=sl.SL_U32, cfg=p.cfg(grid=0))
        torch.cuda.synchronize()
        raw = out.cpu().numpy().tobytes()
        for i in range(steps):
            r = sl.sl_result.from_buffer_copy(raw[i * sl.RESULT_BYTES:(i + 1) * sl.RESULT_BYTES])
            assert (r.sum_u32, r.xor_u64, r.issued_loads) == (*want, p.loads(nbytes)), (p.label(), i)
    del bufs
    torch.cuda.empty_cache()


def test_allocation_sweep_largest_size(sl):
    """The allocation sweep's largest buffer (20 GiB, above L2 many times):
    LDG K = 1, 2, 4, 8, 16 in both orders against the oracle."""
    nbytes = 20 << 30
    free, _ = torch.cuda.mem_get_info()
    if free < nbytes + (2 << 30):
        pytest.skip("not enough free device memory for a 20 GiB buffer")
    dev = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    sl.sl_fill_splitmix64(dev, seed=1)
    want = _oracle_generated(1, nbytes // 4)
    sms = sl.sl_device_info()["sm_count"]
    for k in (1, 2, 4, 8, 16):
        for order in ("asc", "desc"):
            r = sl.sl_run(dev, dtype=sl.SL_U32, cfg=sl.config("ldg", k=k, cta=256, grid=4 * sms, order=order))
            assert (r.sum_u32, r.xor_u64, r.issued_loads) == (*want, nbytes // 16), (k, order)
    del dev
    torch.cuda.empty_cache()


@pytest.mark.parametrize("payload", ["f32", "bf16", "fp8", "bf16-cancel"])
def test_precision_full_size(sl, payload):
    """The precision form at the benchmark's size (4 GiB per payload) through
    the points it most often picks (LDG dynamic chunks K=8, cp.async D=6, TMA
    with 4 KiB stages dealt to the warps, LDG K=8 grid-stride): raw-word
    checksums bit-exact, float sums within 2e-6 of the oracle's FP64 sum of
    the whole payload (computed on the host threads)."""
    import math
    from paper_2608_15764_gb300 import workloads as wl
    nbytes = 4 << 30
    if payload == "bf16-cancel":
        dt, host = wl.BF16, wl.bf16_cancel(nbytes // 16)
    else:
        dt = {"f32": wl.F32, "bf16": wl.BF16, "fp8": wl.FP8_E4M3}[payload]
        host = wl.payload(dt, nbytes // wl.ELEM_BYTES[dt])
    n = host.size
    t = os.cpu_count() or 1
    cut = [i * (n // t) // 16 * 16 for i in range(t)] + [n]
    with ThreadPoolExecutor(t) as ex:
        parts = list(ex.map(lambda i: oracle.fsum(dt, host[cut[i]:cut[i + 1]]), range(t)))
    ref, absum = math.fsum(p[0] for p in parts), math.fsum(p[1] for p in parts)
    if payload == "bf16-cancel":
        assert ref == (nbytes // 16) * (1 + 2.0 ** -5)
    want = _oracle_parallel(host.view(np.uint32))
    dev = torch.from_numpy(host.view(np.uint8)).cuda()
    gate = 2e-6 * (absum if abs(ref) < 1e-3 * absum / math.sqrt(n) else abs(ref))
    for cfg in [sl.config("ldg", k=8, cta=256, order="dyn"), sl.config("cpasync", k=6, cta=256),
                sl.config("cpasync", k=2, copies=8, cta=256), sl.config("cpasync", k=2, copies=8, cta=256, order="dyn"),
                sl.config("tma", cta=256, stage_bytes=4096, stages=8, ring="warp"), sl.config("ldg", k=8, cta=256)]:
        r = sl.sl_run(dev, dtype=dt, cfg=cfg)
        assert (r.sum_u32, r.xor_u64, r.issued_loads, r.status) == (*want, nbytes // 16, 0)
        assert abs(r.fsum - ref) <= gate, (payload, r.fsum, ref)
    del dev
    torch.cuda.empty_cache()
