"""Timing audit of the offered-ILP axis (replaces the paper's SASS audit,
§3 "Instruments"): a lone warp reading from HBM (L2 flushed before each run)
is latency-bound, so if a thread really keeps its K loads (LDG) or D commit
groups (cp.async) in flight, the time of a fixed-work pass falls about
K-fold; if the loads were serialized behind their consumers it would stay
flat."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NBYTES = 32 << 20


@pytest.fixture(scope="module")
def sl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_15764_gb300 as sl
    sl.load()
    return sl


def _time(sl, buf, cfg):
    ts = []
    for _ in range(3):
        r = sl.sl_run(buf, dtype=sl.SL_U32, cfg=cfg)
        assert r.issued_loads == NBYTES // 16
        ts.append(r.device_ns)
    return min(ts)


@pytest.fixture(scope="module")
def buf(sl):
    b = torch.empty(NBYTES, dtype=torch.uint8, device="cuda")
    sl.sl_fill_splitmix64(b, seed=1)
    return b


def test_lone_warp_ldg_time_scales_with_k(sl, buf):
    ks = [1, 2, 4, 8, 16]
    t = {k: _time(sl, buf, sl.config("ldg", k=k, cta=32, grid=1, flush_l2=True)) for k in ks}
    for k in ks[1:]:
        speedup = t[1] / t[k]
        assert speedup >= 0.5 * k, (k, speedup, t)


def test_lone_warp_cpasync_time_scales_with_depth(sl, buf):
    ds = [1, 2, 4, 8]
    t = {d: _time(sl, buf, sl.config("cpasync", k=d, cta=32, grid=1, flush_l2=True)) for d in ds}
    for d in ds[1:]:
        assert t[1] / t[d] >= 0.5 * d, (d, t)
