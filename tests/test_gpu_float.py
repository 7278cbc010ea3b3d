"""GPU parity of the precision form (FP32 / BF16 / FP8-E4M3 payloads summed
with FP32 Kahan accumulation and an FP64 final combine) against the FP64
oracle, plus bit-exact uint32 checksums of the raw payload words.

Tolerance: |fsum - ref| <= 2e-6 * |ref| (relative to the exact sum).  Where
|ref| is small against the payload's magnitude (|ref| < 1e-3 * sum|x| /
sqrt(n)), the gate is the condition-normalised |fsum - ref| / sum|x| <= 2e-6
instead."""
import math

import numpy as np
import pytest

import oracle
from paper_2608_15764_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 2e-6
DTYPES = [wl.F32, wl.BF16, wl.FP8_E4M3]
NBYTES = (1 << 24) + 16 * 1237


@pytest.fixture(scope="module")
def sl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_15764_gb300 as sl
    sl.load()
    return sl


@pytest.fixture(scope="module")
def payloads(sl):
    out = {}
    for dt in DTYPES:
        n = NBYTES // wl.ELEM_BYTES[dt]
        host = wl.payload(dt, n)
        ref, absum = oracle.fsum(dt, host)
        ck = oracle.checksum(host.view(np.uint8))
        dev = torch.from_numpy(host.view(np.uint8)).cuda()
        out[dt] = (dev, host, ref, absum, ck, n)
    return out


def _gate(got, ref, absum, n):
    err = abs(got - ref)
    if abs(ref) >= 1e-3 * absum / math.sqrt(max(n, 1)):
        return err <= TOL * abs(ref), err / abs(ref)
    return err <= TOL * absum, err / absum


def _check(sl, p, dt, cfg):
    dev, host, ref, absum, ck, n = p
    r = sl.sl_run(dev, dtype=dt, cfg=cfg)
    assert (r.sum_u32, r.xor_u64) == ck
    assert r.issued_loads == NBYTES // 16
    ok, rel = _gate(r.fsum, ref, absum, n)
    assert ok, (r.fsum, ref, rel)
    assert r.fsum_hi == np.float32(r.fsum)
    return r


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("k", [1, 2, 3, 4, 8, 16])
@pytest.mark.parametrize("cta", [128, 512])
def test_ldg_float(sl, payloads, dt, k, cta):
    _check(sl, payloads[dt], dt, sl.config("ldg", k=k, cta=cta))


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("k", [2, 4, 8])
def test_ldg_dynamic_float(sl, payloads, dt, k):
    for _ in range(2):
        _check(sl, payloads[dt], dt, sl.config("ldg", k=k, cta=256, order="dyn"))


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("k", [1, 3, 8])
@pytest.mark.parametrize("order", ["asc", "dyn"])
def test_ldg32_float(sl, payloads, dt, k, order):
    dev, host, ref, absum, ck, n = payloads[dt]
    r = sl.sl_run(dev, dtype=dt, cfg=sl.config("ldg32", k=k, cta=256, order=order))
    assert (r.sum_u32, r.xor_u64) == ck
    assert r.issued_loads == (NBYTES + 31) // 32
    ok, rel = _gate(r.fsum, ref, absum, n)
    assert ok, (r.fsum, ref, rel)


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("g", [1, 5, 12])
def test_ldsts_float(sl, payloads, dt, g):
    _check(sl, payloads[dt], dt, sl.config("ldsts", k=g, cta=256))


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("d,g", [(1, 1), (2, 1), (4, 1), (8, 1), (1, 2), (3, 2), (8, 2), (2, 4), (4, 4), (1, 8), (2, 8)])
def test_cpasync_float(sl, payloads, dt, d, g):
    _check(sl, payloads[dt], dt, sl.config("cpasync", k=d, copies=g, cta=256))


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("d,g", [(1, 1), (4, 1), (2, 4), (2, 8)])
def test_cpasync_dynamic_float(sl, payloads, dt, d, g):
    _check(sl, payloads[dt], dt, sl.config("cpasync", k=d, copies=g, cta=256, order="dyn"))


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("stage,stages", [(4096, 4), (16384, 4), (65536, 3)])
def test_tma_float(sl, payloads, dt, stage, stages):
    _check(sl, payloads[dt], dt, sl.config("tma", cta=256, stage_bytes=stage, stages=stages, order="desc"))


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("stage,stages,cta", [(4096, 8, 256), (4096, 2, 64), (16384, 3, 96), (65536, 2, 32)])
def test_tma_warp_rings_float(sl, payloads, dt, stage, stages, cta):
    _check(sl, payloads[dt], dt, sl.config("tma", cta=cta, stage_bytes=stage, stages=stages, ring="warp"))


@pytest.mark.parametrize("dt", DTYPES)
def test_float_closed_forms(sl, dt):
    """Payloads whose exact sum is known: +v/-v pairs sum to zero; a constant
    payload sums to n*c."""
    n = 1 << 20
    x = wl.payload(wl.F32, n // 2, seed=11)
    pair = np.empty(n, dtype=np.float32)
    pair[0::2] = x
    pair[1::2] = -x
    const = np.full(n, 0.75, dtype=np.float32)
    for vals, want in [(pair, 0.0), (const, 0.75 * n)]:
        if dt == wl.F32:
            p = vals
        elif dt == wl.BF16:
            p = wl.f32_to_bf16(vals)
        else:
            p = wl.f32_to_fp8_e4m3(vals)
        ref, absum = oracle.fsum(dt, p)
        assert ref == want or dt != wl.F32
        dev = torch.from_numpy(p.view(np.uint8)).cuda()
        for cfg in [sl.config("ldg", k=4), sl.config("tma", stage_bytes=16384, stages=4)]:
            r = sl.sl_run(dev, dtype=dt, cfg=cfg)
            ok, rel = _gate(r.fsum, ref, absum, n)
            assert ok, (r.fsum, ref, rel)


@pytest.mark.parametrize("dt", DTYPES)
def test_fp8_sums_exact_per_vector(sl, dt):
    """With every value a small integer, all FP32 partial sums are exact: the
    GPU sum must equal the oracle exactly."""
    rng = np.random.default_rng(3)
    v = rng.integers(-8, 9, size=1 << 20).astype(np.float32)
    p = v if dt == wl.F32 else wl.f32_to_bf16(v) if dt == wl.BF16 else wl.f32_to_fp8_e4m3(v)
    ref, _ = oracle.fsum(dt, p)
    r = sl.sl_run(torch.from_numpy(p.view(np.uint8)).cuda(), dtype=dt, cfg=sl.config("ldg", k=2))
    assert r.fsum == ref
