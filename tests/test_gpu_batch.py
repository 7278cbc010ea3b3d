"""GPU parity of the batched form (sl_batch_*: per-class persistent kernels in
one CUDA graph) against the CPU oracle, buffer by buffer: uint32 checksums
and issued loads bit-exact, float sums within 2e-6 relative (condition-
normalised where the exact sum is small), and identical results on every
replay of the graph."""
import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2608_15764_gb300 import autotune
from paper_2608_15764_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 2e-6
KIB, MIB = 1 << 10, 1 << 20
# ragged sizes across all three size classes (bytes, multiples of 16)
SIZES = [0, 16, 48, 4096 + 16, 64 * KIB, 100 * KIB + 16, MIB - 16, MIB, MIB + 48, 3 * MIB + 16, 5 * MIB,
         16 * MIB, 17 * MIB + 32, 40 * MIB + 16]


@pytest.fixture(scope="module")
def sl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_15764_gb300 as sl
    sl.load()
    return sl


def _gate(got, ref, absum, n):
    err = abs(got - ref)
    if abs(ref) >= 1e-3 * absum / math.sqrt(max(n, 1)):
        return err <= TOL * abs(ref)
    return err <= TOL * absum


def _make(dtype, sizes, seed0=100):
    """Host payloads (one per size) and the device buffers holding them."""
    host, dev = [], []
    for i, nb in enumerate(sizes):
        if dtype == wl.U32:
            h = wl.splitmix_u32(seed0 + i, nb // 4).view(np.uint8)
        else:
            h = wl.payload(dtype, nb // wl.ELEM_BYTES[dtype], seed=seed0 + i).view(np.uint8)
        host.append(h)
        d = torch.empty(max(nb, 16), dtype=torch.uint8, device="cuda")
        if nb:
            d[:nb].copy_(torch.from_numpy(h))
        dev.append(d)
    return host, dev


def _check(results, host, dtypes):
    for r, h, dt in zip(results, host, dtypes):
        assert r.status == 0
        assert (r.sum_u32, r.xor_u64) == oracle.checksum(h)
        assert r.issued_loads == h.size // 16
        if dt != wl.U32 and h.size:
            ref, absum = oracle.fsum(dt, h)
            assert _gate(r.fsum, ref, absum, h.size // wl.ELEM_BYTES[dt]), (r.fsum, ref)


def _mixed_table(sl, dtype=-1):
    return [sl.tune_entry(0, MIB - 1, sl.config("ldg", k=4, cta=256), dtype),
            sl.tune_entry(MIB, 16 * MIB - 1, sl.config("cpasync", k=4, cta=256), dtype),
            sl.tune_entry(16 * MIB, 1 << 62, sl.config("tma", cta=256, stage_bytes=16384, stages=4), dtype)]


@pytest.mark.parametrize("dtype", [wl.U32, wl.F32, wl.BF16, wl.FP8_E4M3])
def test_batch_three_classes(sl, dtype):
    host, dev = _make(dtype, SIZES)
    b = sl.sl_batch_create([(d, nb, dtype) for d, nb in zip(dev, SIZES)], _mixed_table(sl))
    ncls, cls = sl.sl_batch_info(b)
    assert ncls == 3 and cls[0] == cls[6] and cls[7] != cls[6] and cls[-1] != cls[7]
    first, ns = sl.sl_batch_run(b)
    assert ns > 0
    _check(first, host, [dtype] * len(SIZES))
    for _ in range(3):  # replays are identical (fixed combine order)
        again, _ = sl.sl_batch_run(b)
        assert [(r.sum_u32, r.xor_u64, r.issued_loads, r.fsum) for r in again] == \
               [(r.sum_u32, r.xor_u64, r.issued_loads, r.fsum) for r in first]
    sl.sl_batch_destroy(b)


@pytest.mark.parametrize("cfg", [dict(mech="ldg", k=1, cta=128), dict(mech="ldg", k=16, cta=512),
                                 dict(mech="ldg", k=3, cta=256), dict(mech="cpasync", k=1, cta=128),
                                 dict(mech="cpasync", k=8, cta=512),
                                 dict(mech="tma", cta=128, stage_bytes=4096, stages=3),
                                 dict(mech="tma", cta=512, stage_bytes=65536, stages=2)])
def test_batch_every_mechanism(sl, cfg):
    dts = [wl.U32, wl.F32, wl.BF16, wl.FP8_E4M3]
    sizes = SIZES[:12]
    host, dev, descs, kinds = [], [], [], []
    for j, dt in enumerate(dts):
        h, d = _make(dt, sizes, seed0=300 + 20 * j)
        host += h
        dev += d
        descs += [(x, nb, dt) for x, nb in zip(d, sizes)]
        kinds += [dt] * len(sizes)
    c = dict(cfg)
    mech = c.pop("mech")
    b = sl.sl_batch_create(descs, autotune.plain_table(sl.config(mech, **c)))
    res, _ = sl.sl_batch_run(b)
    _check(res, host, kinds)
    sl.sl_batch_destroy(b)


def test_batch_grid_override_and_small_grid(sl):
    host, dev = _make(wl.F32, SIZES)
    table = [sl.tune_entry(0, 1 << 62, sl.config("ldg", k=2, cta=256, grid=3))]
    b = sl.sl_batch_create([(d, nb, wl.F32) for d, nb in zip(dev, SIZES)], table)
    res, _ = sl.sl_batch_run(b)
    _check(res, host, [wl.F32] * len(SIZES))


def test_batch_errors(sl):
    d = torch.empty(1 << 16, dtype=torch.uint8, device="cuda")
    E = sl.SLError
    cases = [
        ([(d, 1024, wl.U32)], [sl.tune_entry(4096, 8192, sl.config("ldg"))], sl.SL_ERR_ARG),      # no class
        ([(d.data_ptr() + 8, 1024, wl.U32)], autotune.plain_table(), sl.SL_ERR_ALIGN),
        ([(d, 1000, wl.U32)], autotune.plain_table(), sl.SL_ERR_ALIGN),
        ([(d, 1024, 9)], autotune.plain_table(), sl.SL_ERR_ARG),
        ([(d, 1024, wl.U32)], autotune.plain_table(sl.config("ldg", k=5)), sl.SL_ERR_ARG),
        ([(d, 1024, wl.U32)], autotune.plain_table(sl.config("tma", stage_bytes=65536, stages=4)),
         sl.SL_ERR_INFEASIBLE),
        # the batched TMA class kernel runs one ring per CTA
        ([(d, 1024, wl.U32)], autotune.plain_table(sl.config("tma", cta=256, stage_bytes=4096, stages=8, ring="warp")),
         sl.SL_ERR_ARG),
        ([(d, 1024, wl.U32)], autotune.plain_table(sl.config("cpasync", k=2, copies=4, cta=256)), sl.SL_ERR_ARG),
    ]
    for bufs, table, code in cases:
        with pytest.raises(E) as e:
            sl.sl_batch_create(bufs, table)
        assert e.value.status == code, (bufs, e.value)


def test_autotune_small(sl):
    sizes = [64 * KIB * (1 + i % 7) for i in range(40)] + [2 * MIB + 16 * i for i in range(8)] + [20 * MIB, 33 * MIB]
    host, dev = _make(wl.BF16, sizes, seed0=700)
    bufs = [(d, nb, wl.BF16) for d, nb in zip(dev, sizes)]
    table, report = autotune.tune(bufs, repeats=2)
    assert len(table) == 3 and all(r["gbs"] > 0 for r in report)
    b = sl.sl_batch_create(bufs, table)
    res, _ = sl.sl_batch_run(b)
    _check(res, host, [wl.BF16] * len(sizes))


def test_batch_full_size_recipe_f32(sl):
    """The 1,024-buffer, 16 GiB log-uniform workload (float32 payloads) in one
    graph launch: every buffer's uint32 checksum bit-exact, float sums of a
    sample of 48 buffers (spread over the size range) against the oracle."""
    sizes = wl.batch_sizes()
    total = sum(sizes)
    offs = np.cumsum([0] + sizes[:-1])
    host = torch.empty(total, dtype=torch.uint8, pin_memory=True)
    hv = host.numpy()
    # one N(0,1) stream for the whole arena; buffer i is the slice at offs[i]
    wl.payload(wl.F32, total // 4, out=hv.view(np.float32))
    dev = torch.empty(total, dtype=torch.uint8, device="cuda")
    dev.copy_(host)
    base = dev.data_ptr()
    bufs = [(base + int(o), nb, wl.F32) for o, nb in zip(offs, sizes)]
    b = sl.sl_batch_create(bufs, _mixed_table(sl))
    res, _ = sl.sl_batch_run(b)
    threads = os.cpu_count() or 1
    with ThreadPoolExecutor(threads) as ex:
        cks = list(ex.map(lambda i: oracle.checksum(hv[offs[i]:offs[i] + sizes[i]]), range(len(sizes))))
    for r, ck, nb in zip(res, cks, sizes):
        assert (r.sum_u32, r.xor_u64) == ck and r.issued_loads == nb // 16 and r.status == 0
    order = np.argsort(sizes)
    sample = [int(order[i]) for i in np.linspace(0, len(sizes) - 1, 48).astype(int)]
    with ThreadPoolExecutor(threads) as ex:
        refs = list(ex.map(lambda i: oracle.fsum(wl.F32, hv[offs[i]:offs[i] + sizes[i]]), sample))
    for i, (ref, absum) in zip(sample, refs):
        assert _gate(res[i].fsum, ref, absum, sizes[i] // 4), (i, res[i].fsum, ref)
    sl.sl_batch_destroy(b)
    del dev
    torch.cuda.empty_cache()
