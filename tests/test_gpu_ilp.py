"""Timing audit of the offered-ILP axis (replaces the paper's SASS audit,
§3 "Instruments"): a lone warp is latency-bound, so if a thread really keeps
its K loads (LDG) or D commit groups (cp.async) in flight, the time of a
fixed-work pass falls about K-fold.  If the loads were serialized behind their
consumers, the time would stay flat."""
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


@pytest.mark.parametrize("mech,ks", [("ldg", [1, 2, 4, 8, 16]), ("cpasync", [1, 2, 4, 8])])
def test_lone_warp_time_scales_with_offered_ilp(sl, mech, ks):
    buf = torch.empty(NBYTES, dtype=torch.uint8, device="cuda")
    sl.sl_fill_splitmix64(buf, seed=1)
    t = {k: _time(sl, buf, sl.config(mech, k=k, cta=32, grid=1)) for k in ks}
    for k in ks[1:]:
        speedup = t[ks[0]] / t[k]
        assert speedup >= 0.5 * k, (mech, k, speedup, t)
