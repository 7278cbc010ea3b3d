"""Adversarial GPU parity of the precision form against the FP64 oracle.

The N(0,1) payloads of test_gpu_float.py never make a running FP32 sum lose
anything that matters.  These inputs do:

* BF16 vectors in which 2^20 and -2^20 sit next to 2^-5 and 1, in every
  position (a plain FP32 sum of the eight values drops 2^-5 in some orders:
  a 3% error on the whole buffer);
* BF16 / FP32 vectors spread over ~36 binades with a cancelling +-L pair in
  each, so the exact sum is carried by values 2^4 ... 2^36 times smaller than
  the running sums;
* every finite BF16 code (zeros, subnormals, every normal binade up to the
  largest finite value, both signs), in groups whose sums are exact in FP32:
  the GPU sum must equal the oracle's exactly, which pins the device decode of
  every code;
* every finite FP8 E4M3 code, including the subnormals and +-448, alone
  (exact) and repeated with cancelling +-448 pairs (gated).

Each goes through every mechanism (LDG grid-stride and dynamic chunks, 32-byte
loads, cp.async, the matched LDG->STS kernel, TMA rings), the batched form
and the allocation-free entry point.  Gate: |fsum - ref| <= 2e-6 |ref|, or
2e-6 sum|x| where |ref| < 1e-3 sum|x| / sqrt(n); integer checksums and issued
loads bit-exact."""
import math

import numpy as np
import pytest

import oracle
from paper_2608_15764_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 2e-6
NVEC = (1 << 20) + 1237  # 16 MiB + a ragged tail of 1,237 vectors
CONFIGS = [
    ("ldg", dict(k=1, cta=128)),
    ("ldg", dict(k=4, cta=256)),
    ("ldg", dict(k=16, cta=512, order="desc")),
    ("ldg", dict(k=4, cta=256, order="dyn")),
    ("ldg32", dict(k=1, cta=256)),
    ("ldg32", dict(k=6, cta=256, order="dyn")),
    ("cpasync", dict(k=1, cta=256)),
    ("cpasync", dict(k=4, cta=256)),
    ("cpasync", dict(k=8, cta=512)),
    ("cpasync", dict(k=2, copies=4, cta=256)),
    ("cpasync", dict(k=2, copies=8, cta=256, order="dyn")),
    ("ldsts", dict(k=4, cta=256)),
    ("tma", dict(cta=256, stage_bytes=4096, stages=2)),
    ("tma", dict(cta=256, stage_bytes=16384, stages=4, order="desc")),
    ("tma", dict(cta=256, stage_bytes=65536, stages=3)),
    ("tma", dict(cta=256, stage_bytes=4096, stages=8, ring="warp")),
    ("tma", dict(cta=64, stage_bytes=16384, stages=4, ring="warp", order="desc")),
]
IDS = [f"{m}-" + "-".join(f"{k}{v}" for k, v in kw.items()) for m, kw in CONFIGS]


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
        return err <= TOL * abs(ref), err / abs(ref)
    return err <= TOL * absum, err / absum


class Payload:
    def __init__(self, dt, host):
        self.dt = dt
        self.host = np.ascontiguousarray(host)
        self.bytes = self.host.view(np.uint8)
        assert self.bytes.size % 16 == 0
        self.n = self.bytes.size // wl.ELEM_BYTES[dt]
        self.ref, self.absum = oracle.fsum(dt, self.host)
        self.ck = oracle.checksum(self.bytes)
        self.dev = torch.from_numpy(self.bytes).cuda()

    def check(self, r, exact=False, loads=None):
        assert r.status == 0
        assert (r.sum_u32, r.xor_u64) == self.ck
        assert r.issued_loads == (self.bytes.size // 16 if loads is None else loads)
        if exact:
            assert r.fsum == self.ref, (r.fsum, self.ref)
        ok, rel = _gate(r.fsum, self.ref, self.absum, self.n)
        assert ok, (r.fsum, self.ref, rel)


def _loads(mech, nbytes):
    return (nbytes + 31) // 32 if mech == "ldg32" else nbytes // 16


@pytest.fixture(scope="module")
def cancel(sl):
    p = Payload(wl.BF16, wl.bf16_cancel(NVEC))
    # the exact sum is nvec (1 + 2^-5): the oracle must agree before the GPU is asked
    assert p.ref == NVEC * (1 + 2.0 ** -5)
    return p


@pytest.fixture(scope="module")
def wide(sl):
    codes = wl.bf16_wide(NVEC)
    return {wl.BF16: Payload(wl.BF16, codes), wl.F32: Payload(wl.F32, wl.bf16_as_f32_bits(codes))}


@pytest.mark.parametrize("mech,kw", CONFIGS, ids=IDS)
def test_bf16_cancellation_every_mechanism(sl, cancel, mech, kw):
    r = sl.sl_run(cancel.dev, dtype=wl.BF16, cfg=sl.config(mech, **kw))
    cancel.check(r, loads=_loads(mech, cancel.bytes.size))


@pytest.mark.parametrize("dt", [wl.BF16, wl.F32])
@pytest.mark.parametrize("mech,kw", CONFIGS, ids=IDS)
def test_wide_range_every_mechanism(sl, wide, dt, mech, kw):
    p = wide[dt]
    r = sl.sl_run(p.dev, dtype=dt, cfg=sl.config(mech, **kw))
    p.check(r, loads=_loads(mech, p.bytes.size))


def test_adversarial_passes_and_noalloc(sl, cancel, wide):
    """Several passes (the float part adds up P copies) and the allocation-free
    entry point, on the adversarial payloads."""
    for p in (cancel, wide[wl.BF16], wide[wl.F32]):
        r = sl.sl_run(p.dev, dtype=p.dt, cfg=sl.config("ldg", k=8, cta=256, passes=3))
        assert (r.sum_u32, r.xor_u64) == oracle.checksum(p.bytes, passes=3)
        ok, rel = _gate(r.fsum, 3 * p.ref, 3 * p.absum, 3 * p.n)
        assert ok, rel
        out = torch.zeros(sl.RESULT_BYTES, dtype=torch.uint8, device="cuda")
        sl.sl_run_noalloc(p.dev, out, dtype=p.dt, cfg=sl.config("ldg", k=4, cta=256))
        torch.cuda.synchronize()
        p.check(sl.sl_result.from_buffer_copy(out.cpu().numpy().tobytes()))


def _arena(groups, dt):
    """Groups laid out in one device allocation, each in its own 256-byte
    aligned slot, zero-padded to a multiple of 16 bytes."""
    eb = wl.ELEM_BYTES[dt]
    padded = []
    for g in groups:
        b = np.ascontiguousarray(g).view(np.uint8)
        pad = (-b.size) % 16
        padded.append(np.concatenate([b, np.zeros(pad, np.uint8)]) if pad else b)
    offs, o = [], 0
    for b in padded:
        offs.append(o)
        o += (b.size + 255) // 256 * 256
    host = np.zeros(o, np.uint8)
    for off, b in zip(offs, padded):
        host[off:off + b.size] = b
    dev = torch.from_numpy(host).cuda()
    refs = [oracle.fsum(dt, b) for b in padded]
    cks = [oracle.checksum(b) for b in padded]
    assert all(b.size % eb == 0 for b in padded)
    return dev, offs, padded, refs, cks


@pytest.fixture(scope="module")
def bf16_groups(sl):
    return _arena(wl.bf16_code_groups(), wl.BF16)


GROUP_CONFIGS = [("ldg", dict(k=1, cta=128)), ("ldg", dict(k=8, cta=256)), ("ldg32", dict(k=2, cta=128)),
                 ("cpasync", dict(k=2, cta=128)), ("ldsts", dict(k=2, cta=128)),
                 ("tma", dict(cta=128, stage_bytes=4096, stages=2)),
                 ("tma", dict(cta=64, stage_bytes=4096, stages=2, ring="warp"))]


@pytest.mark.parametrize("mech,kw", GROUP_CONFIGS,
                         ids=[m + str(kw.get("k", "")) + kw.get("ring", "") for m, kw in GROUP_CONFIGS])
def test_every_finite_bf16_code_exact(sl, bf16_groups, mech, kw):
    """Each group's sum is exact in FP32 in any order, so the GPU must return
    the oracle's sum exactly: a wrong decode of any code would show."""
    dev, offs, padded, refs, cks = bf16_groups
    base = dev.data_ptr()
    cfg = sl.config(mech, **kw)
    for off, b, (ref, _), ck in zip(offs, padded, refs, cks):
        r = sl.sl_run(base + off, nbytes=b.size, dtype=wl.BF16, cfg=cfg)
        assert (r.sum_u32, r.xor_u64) == ck
        assert r.fsum == ref, (off, b.view(np.uint16)[:4], r.fsum, ref)


def _one_mech_table(sl, mech, **kw):
    return [sl.tune_entry(0, 1 << 62, sl.config(mech, **kw))]


BATCH_TABLES = [("ldg", dict(k=4, cta=256)), ("cpasync", dict(k=4, cta=256)),
                ("tma", dict(cta=256, stage_bytes=16384, stages=4))]


@pytest.mark.parametrize("mech,kw", BATCH_TABLES, ids=[m for m, _ in BATCH_TABLES])
def test_every_finite_bf16_code_batched(sl, bf16_groups, mech, kw):
    """The 1,226 groups as the buffers of one batch: every buffer's sum exact."""
    dev, offs, padded, refs, cks = bf16_groups
    base = dev.data_ptr()
    b = sl.sl_batch_create([(base + o, p.size, wl.BF16) for o, p in zip(offs, padded)],
                           _one_mech_table(sl, mech, **kw))
    for _ in range(2):
        res, _ = sl.sl_batch_run(b)
        for r, (ref, _), ck in zip(res, refs, cks):
            assert r.status == 0 and (r.sum_u32, r.xor_u64) == ck
            assert r.fsum == ref
    sl.sl_batch_destroy(b)


@pytest.mark.parametrize("mech,kw", BATCH_TABLES, ids=[m for m, _ in BATCH_TABLES])
def test_adversarial_batched(sl, cancel, wide, mech, kw):
    """The adversarial payloads cut into uneven buffers of one batch, every
    class mechanism."""
    cuts = [0, 16, 4096 + 48, 200 * 1024, 3 << 20, 9 << 20]
    bufs, exp = [], []
    for p in (cancel, wide[wl.BF16], wide[wl.F32]):
        edges = cuts + [p.bytes.size]
        for lo, hi in zip(edges[:-1], edges[1:]):
            bufs.append((p.dev.data_ptr() + lo, hi - lo, p.dt))
            exp.append((p.dt, p.bytes[lo:hi]))
    b = sl.sl_batch_create(bufs, _one_mech_table(sl, mech, **kw))
    res, _ = sl.sl_batch_run(b)
    for r, (dt, h) in zip(res, exp):
        assert r.status == 0 and (r.sum_u32, r.xor_u64) == oracle.checksum(h)
        assert r.issued_loads == h.size // 16
        ref, absum = oracle.fsum(dt, h)
        ok, rel = _gate(r.fsum, ref, absum, h.size // wl.ELEM_BYTES[dt])
        assert ok, (r.fsum, ref, rel)
    sl.sl_batch_destroy(b)


@pytest.mark.parametrize("mech,kw", CONFIGS, ids=IDS)
def test_every_finite_fp8_code(sl, mech, kw):
    """All 254 finite E4M3 codes: (a) each twice, positive codes only and all
    codes (the sum of all codes is 0): every partial sum is a multiple of 2^-9
    below 2^15, so the sums must be exact; (b) 4,096 seeded shuffles of all
    codes with a cancelling +-448 pair per vector, gated."""
    codes = wl.fp8_finite_codes()
    pos = codes[codes < 0x80]
    cfg = sl.config(mech, **kw)
    for h in (np.tile(pos, 2), np.tile(codes, 2)):
        h = np.concatenate([h, np.zeros((-h.size) % 16, np.uint8)])
        p = Payload(wl.FP8_E4M3, h)
        p.check(sl.sl_run(p.dev, dtype=wl.FP8_E4M3, cfg=cfg), exact=True, loads=_loads(mech, h.size))
    rng = np.random.default_rng(9)
    v = np.concatenate([rng.permutation(np.resize(codes, 16 * 64)) for _ in range(256)]).reshape(-1, 16)
    v[:, 3], v[:, 12] = 0x7E, 0xFE  # +448, -448
    p = Payload(wl.FP8_E4M3, v.reshape(-1))
    p.check(sl.sl_run(p.dev, dtype=wl.FP8_E4M3, cfg=cfg), loads=_loads(mech, p.bytes.size))
