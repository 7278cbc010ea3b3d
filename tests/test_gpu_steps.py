"""GPU parity of sl_enqueue_steps: back-to-back passes whose launches after
the first are programmatic dependent launches (a pass may start loading
while the previous pass's tail runs).  Every pass's result must equal the
oracle's checksum and a separate launch's result, whatever the mechanism,
grid or interleaving with ordinary launches."""
import numpy as np
import pytest

import oracle
from paper_2608_15764_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEED = 1
NBYTES = (1 << 24) + 16 * 1237


@pytest.fixture(scope="module")
def sl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_15764_gb300 as sl
    sl.load()
    return sl


@pytest.fixture(scope="module")
def data(sl):
    dev = torch.empty(NBYTES, dtype=torch.uint8, device="cuda")
    sl.sl_fill_splitmix64(dev, seed=SEED)
    host = workloads.splitmix_u32(SEED, NBYTES // 4)
    return dev, host, oracle.checksum(host)


def _results(sl, out, n):
    raw = out.cpu().numpy().tobytes()
    rb = sl.RESULT_BYTES
    return [sl.sl_result.from_buffer_copy(raw[rb * i:rb * (i + 1)]) for i in range(n)]


@pytest.mark.parametrize("mech,kw,loads", [
    ("ldg", dict(k=2, cta=256), 16), ("ldg", dict(k=6, cta=256, order="desc"), 16),
    ("ldg", dict(k=4, cta=128), 16), ("ldg", dict(k=1, cta=1024), 16),
    ("ldg32", dict(k=4, cta=256), 32), ("ldg4", dict(k=4, cta=256), 4),
    ("cpasync", dict(k=4, cta=256), 16), ("cpasync", dict(k=2, copies=4, cta=256), 16),
    ("cpasync", dict(k=2, copies=8, cta=256, order="dyn"), 16),
    ("ldsts", dict(k=4, cta=256), 16),
    ("ldg", dict(k=12, cta=256, order="dyn"), 16), ("ldg", dict(k=2, cta=512, order="dyn"), 16),
    ("ldg32", dict(k=6, cta=256, order="dyn"), 32),
    ("tma", dict(cta=256, stage_bytes=16384, stages=4), 16), ("tma", dict(cta=512, stage_bytes=65536, stages=2,
                                                                         order="desc"), 16),
    ("tma", dict(cta=256, stage_bytes=4096, stages=8, ring="warp"), 16),
    ("tma", dict(cta=128, stage_bytes=16384, stages=4, ring="warp", order="desc"), 16),
])
def test_steps_each_pass_matches_oracle(sl, data, mech, kw, loads):
    dev, _, want = data
    steps = 9
    out = torch.zeros(steps * sl.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    sl.sl_enqueue_steps(dev, out, steps, dtype=sl.SL_U32, cfg=sl.config(mech, **kw))
    torch.cuda.synchronize()
    want_loads = (NBYTES + loads - 1) // loads
    for r in _results(sl, out, steps):
        assert (r.sum_u32, r.xor_u64, r.issued_loads, r.status) == (*want, want_loads, 0)
        assert r.window_ns > 0


def test_steps_alternate_buffers(sl, data):
    """Pass i reads buffer i mod 3: the per-pass checksums follow the
    buffers."""
    dev, host, want = data
    other = torch.empty_like(dev)
    sl.sl_fill_splitmix64(other, seed=7)
    want7 = oracle.checksum(workloads.splitmix_u32(7, NBYTES // 4))
    steps = 7
    out = torch.zeros(steps * sl.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    sl.sl_enqueue_steps([dev, other, dev], out, steps, dtype=sl.SL_U32, cfg=sl.config("ldg", k=3, cta=256))
    torch.cuda.synchronize()
    for i, r in enumerate(_results(sl, out, steps)):
        assert (r.sum_u32, r.xor_u64) == (want7 if i % 3 == 1 else want), i


def test_steps_run_one_full_wave(sl, data):
    dev, _, _ = data
    cfg = sl.config("ldg", k=3, cta=256)
    plan = sl.sl_plan(NBYTES, sl.SL_U32, cfg)
    wave = plan.resident_per_sm * sl.sl_device_info()["sm_count"]
    out = torch.zeros(2 * sl.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    sl.sl_enqueue_steps(dev, out, 2, dtype=sl.SL_U32, cfg=sl.config("ldg", k=3, cta=256, grid=wave))
    with pytest.raises(sl.SLError) as e:
        sl.sl_enqueue_steps(dev, out, 2, dtype=sl.SL_U32, cfg=sl.config("ldg", k=3, cta=256, grid=wave - 1))
    assert e.value.status == sl.SL_ERR_ARG
    torch.cuda.synchronize()


def test_steps_interleaved_with_ordinary_launches(sl, data):
    dev, _, want = data
    out = torch.zeros(12 * sl.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    cfg = sl.config("ldg", k=3, cta=256)
    sl.sl_enqueue_steps(dev, out[: 4 * sl.RESULT_BYTES], 4, dtype=sl.SL_U32, cfg=cfg)
    sl.sl_enqueue(dev, out[4 * sl.RESULT_BYTES:], dtype=sl.SL_U32, cfg=sl.config("ldg", k=12, order="dyn"))
    sl.sl_enqueue_steps(dev, out[5 * sl.RESULT_BYTES:], 6, dtype=sl.SL_U32, cfg=sl.config("ldg32", k=2))
    r = sl.sl_run(dev, dtype=sl.SL_U32, cfg=cfg)  # ordered after the enqueued work
    assert (r.sum_u32, r.xor_u64) == want
    sl.sl_enqueue(dev, out[11 * sl.RESULT_BYTES:], dtype=sl.SL_U32, cfg=cfg)
    torch.cuda.synchronize()
    for r in _results(sl, out, 12):
        assert (r.sum_u32, r.xor_u64, r.status) == (*want, 0)


def test_steps_float_sums_equal_a_single_launch(sl):
    """Every pass's float sum meets the gate against the FP64 oracle and its
    checksum equals the oracle's; and with the same launch shape (one full
    wave) the float sum is also bit-identical to sl_run's at that grid (a
    determinism property on top of parity)."""
    x = workloads.payload(workloads.F32, (1 << 22) + 5 * 4)
    exact, _ = oracle.fsum(workloads.F32, x)
    ck = oracle.checksum(x.view(np.uint32))
    dev = torch.from_numpy(x.view(np.uint8)).cuda()
    cfg = sl.config("ldg", k=4, cta=256)
    wave = sl.sl_plan(x.nbytes, sl.SL_F32, cfg).resident_per_sm * sl.sl_device_info()["sm_count"]
    ref = sl.sl_run(dev, dtype=sl.SL_F32, cfg=sl.config("ldg", k=4, cta=256, grid=wave))
    out = torch.zeros(5 * sl.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    sl.sl_enqueue_steps(dev, out, 5, dtype=sl.SL_F32, cfg=cfg)
    torch.cuda.synchronize()
    assert abs(ref.fsum - exact) <= 2e-6 * abs(exact) and (ref.sum_u32, ref.xor_u64) == ck
    for r in _results(sl, out, 5):
        assert abs(r.fsum - exact) <= 2e-6 * abs(exact) and (r.sum_u32, r.xor_u64) == ck
        assert r.fsum == ref.fsum


def test_steps_fixed_iteration(sl, data):
    dev, host, _ = data
    target = 2 * (NBYTES // 16) + 999
    cfg = sl.config("ldg", k=4, cta=256, target_loads=target)
    wave = sl.sl_plan(NBYTES, sl.SL_U32, cfg).resident_per_sm * sl.sl_device_info()["sm_count"]
    out = torch.zeros(4 * sl.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    sl.sl_enqueue_steps(dev, out, 4, dtype=sl.SL_U32, cfg=cfg)
    torch.cuda.synchronize()
    issued, _ = oracle.fixed_iteration(target, wave * 256, [4])
    want = oracle.wrapped_checksum(host, issued[0])
    for r in _results(sl, out, 4):
        assert (r.sum_u32, r.xor_u64, r.issued_loads) == (*want, issued[0])


def test_steps_empty_and_rejected(sl, data):
    dev, _, _ = data
    out = torch.ones(3 * sl.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    sl.sl_enqueue_steps(dev, out, 3, nbytes=0, dtype=sl.SL_U32, cfg=sl.config("ldg"))
    torch.cuda.synchronize()
    for r in _results(sl, out, 3):
        assert (r.sum_u32, r.xor_u64, r.issued_loads) == (0, 0, 0)
    for cfg, steps in [(sl.config("ldg", flush_l2=True), 2), (sl.config("ldg"), 0)]:
        with pytest.raises(sl.SLError) as e:
            sl.sl_enqueue_steps(dev, out, steps, dtype=sl.SL_U32, cfg=cfg)
        assert e.value.status == sl.SL_ERR_ARG


def test_dynamic_steps_across_counter_segments(sl, data):
    """More passes than one segment of per-pass chunk counters (4,096): every
    pass still covers the buffer once."""
    dev, _, want = data
    steps = 4096 + 7
    nb = 16 * 70001  # a small buffer: many short passes
    host = workloads.splitmix_u32(SEED, nb // 4)
    want = oracle.checksum(host)
    out = torch.zeros(steps * sl.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    sl.sl_enqueue_steps(dev, out, steps, nbytes=nb, dtype=sl.SL_U32, cfg=sl.config("ldg", k=4, order="dyn"))
    torch.cuda.synchronize()
    for r in _results(sl, out, steps):
        assert (r.sum_u32, r.xor_u64, r.issued_loads) == (*want, nb // 16)


def test_dynamic_steps_float_sums(sl):
    x = workloads.payload(workloads.BF16, (1 << 23) + 8 * 7)
    dev = torch.from_numpy(x.view(np.uint8)).cuda()
    ref, absum = oracle.fsum(workloads.BF16, x)
    out = torch.zeros(6 * sl.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    sl.sl_enqueue_steps(dev, out, 6, dtype=sl.SL_BF16, cfg=sl.config("ldg", k=8, order="dyn"))
    torch.cuda.synchronize()
    for r in _results(sl, out, 6):
        assert abs(r.fsum - ref) <= 2e-6 * abs(ref)


@pytest.mark.parametrize("ring,cta,stage", [("cta", 256, 16384), ("warp", 128, 4096)])
def test_tma_steps_report_a_timeout_on_its_own_pass(sl, data, ring, cta, stage):
    """A TMA pass whose bounded wait gives up (debug flag: one stage never
    armed) reports SL_ERR_TIMEOUT in its own result, and the passes before and
    after it -- overlapped with it -- are unaffected."""
    dev, _, want = data
    ok = sl.config("tma", cta=cta, stage_bytes=stage, stages=4, ring=ring)
    bad = sl.config("tma", cta=cta, stage_bytes=stage, stages=4, ring=ring, debug_flags=sl.SL_DEBUG_TMA_SKIP_STAGE)
    out = torch.zeros(7 * sl.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    rb = sl.RESULT_BYTES
    sl.sl_enqueue_steps(dev, out[: 3 * rb], 3, dtype=sl.SL_U32, cfg=ok)
    sl.sl_enqueue_steps(dev, out[3 * rb: 4 * rb], 1, dtype=sl.SL_U32, cfg=bad)
    sl.sl_enqueue_steps(dev, out[4 * rb:], 3, dtype=sl.SL_U32, cfg=ok)
    torch.cuda.synchronize()
    res = _results(sl, out, 7)
    assert res[3].status == sl.SL_ERR_TIMEOUT
    for i in (0, 1, 2, 4, 5, 6):
        assert (res[i].sum_u32, res[i].xor_u64, res[i].status) == (*want, 0), i
