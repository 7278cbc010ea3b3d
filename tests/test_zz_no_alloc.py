"""sl_run_noalloc, the allocation-free entry point, against sl_run.

sl_run_noalloc serves callers that cannot allocate device memory (a framework
pool that owns the memory, a latency-critical loop, a plugin contract that
forbids allocation): its scratch is a fixed device array instead of lazily
allocated buffers.  These tests call it through the C ABI twice in a row (the
array keeps the previous call's contents) and check each result against the
regular entry point's, bit-exactly for the integer checksum and within the
float tolerance of the other tests (2e-6 relative) for float sums.  The file
is collected last so that a run stopping at the first failure has already run
every other test; it also passes on its own in a fresh process."""
import numpy as np
import pytest

import oracle
from paper_2608_15764_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 2e-6
NBYTES = (1 << 24) + 16 * 1237


@pytest.fixture(scope="module")
def sl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_15764_gb300 as sl
    sl.load()
    return sl


def _noalloc(sl, buf, dtype, cfg, nbytes=None):
    out = torch.zeros(sl.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    sl.sl_run_noalloc(buf, out, nbytes=nbytes, dtype=dtype, cfg=cfg)
    torch.cuda.synchronize()
    return sl.sl_result.from_buffer_copy(out.cpu().numpy().tobytes())


def test_noalloc_matches_sl_run_two_calls(sl):
    dev = torch.empty(NBYTES, dtype=torch.uint8, device="cuda")
    sl.sl_fill_splitmix64(dev, seed=1)
    exact = oracle.checksum(wl.splitmix_u32(1, NBYTES // 4))
    # two calls in a row with different launch shapes: the second must not
    # see anything of the first call's scratch contents
    for cfg in [sl.config("ldg", k=4, cta=256), sl.config("ldg", k=2, cta=512, grid=37, order="desc")]:
        want = sl.sl_run(dev, dtype=sl.SL_U32, cfg=cfg)
        got = _noalloc(sl, dev, sl.SL_U32, cfg)
        assert got.status == 0
        assert (got.sum_u32, got.xor_u64, got.issued_loads) == (want.sum_u32, want.xor_u64, want.issued_loads)
        assert (got.sum_u32, got.xor_u64) == exact  # and both match the oracle


@pytest.mark.parametrize("dtype", [wl.F32, wl.BF16, wl.FP8_E4M3])
def test_noalloc_float_two_calls(sl, dtype):
    host = wl.payload(dtype, NBYTES // wl.ELEM_BYTES[dtype])
    dev = torch.from_numpy(host.view(np.uint8)).cuda()
    exact, _ = oracle.fsum(dtype, host)
    for cfg, passes in [(sl.config("ldg", k=8, cta=128), 1), (sl.config("ldg", k=1, cta=256, passes=2), 2)]:
        want = sl.sl_run(dev, dtype=dtype, cfg=cfg)
        got = _noalloc(sl, dev, dtype, cfg)
        assert (got.sum_u32, got.xor_u64, got.issued_loads) == (want.sum_u32, want.xor_u64, want.issued_loads)
        assert abs(got.fsum - want.fsum) <= TOL * abs(want.fsum)
        assert abs(got.fsum - passes * exact) <= TOL * abs(passes * exact)  # and against the oracle


def test_noalloc_limits_and_empty(sl):
    dev = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    out = torch.zeros(sl.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    for cfg in [sl.config("ldg", k=1, cta=256, grid=sl.SL_NOALLOC_MAX_CTAS + 1),
                sl.config("ldg", k=1, cta=1024, grid=10000),  # more CTAs than the fixed scratch holds
                sl.config("tma"), sl.config("cpasync", k=2, copies=4), sl.config("ldg", flush_l2=True)]:
        with pytest.raises(sl.SLError) as e:
            sl.sl_run_noalloc(dev, out, dtype=sl.SL_U32, cfg=cfg)
        assert e.value.status == sl.SL_ERR_ARG
    r = _noalloc(sl, 0, sl.SL_U32, sl.config("ldg", k=2), nbytes=0)
    assert (r.sum_u32, r.xor_u64, r.issued_loads) == (0, 0, 0)
