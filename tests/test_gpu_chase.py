"""The pointer-chase latency probe (paper §4.1 primitive baseline) against the
oracle: after warm + timed steps the final index equals the oracle's walk of
the same chain, at footprints that live in L1, L2 and HBM, with .ca and .cg.
Its latencies must order as the memory hierarchy does."""
import numpy as np
import pytest

import oracle
from paper_2608_15764_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_15764_gb300 as sl
    sl.load()
    return sl


def _chain(n):
    host = wl.chase_chain(n, 64)
    return host, torch.from_numpy(host.view(np.uint8)).cuda()


@pytest.mark.parametrize("footprint", [8 << 10, 4 << 20, 512 << 20])
@pytest.mark.parametrize("ca", [True, False])
def test_chase_final_index_matches_oracle(sl, footprint, ca):
    n = footprint // 64
    host, dev = _chain(n)
    warm, hops = min(n, 1 << 14), 4096
    r = sl.sl_chase(dev, start=0, warm=warm, hops=hops, cache_l1=ca)
    assert r.final_index == oracle.chase(host, 0, warm + hops)
    assert r.hops == hops and r.ns > 0 and r.cycles > 0


def test_latency_ladder_orders(sl):
    lat = {}
    for name, footprint, ca in [("l1", 8 << 10, True), ("l2", 4 << 20, False), ("hbm", 1 << 30, False)]:
        n = footprint // 64
        _, dev = _chain(n)
        lat[name] = sl.sl_chase(dev, warm=min(n, 1 << 14), hops=1 << 13, cache_l1=ca).ns_per_hop
    assert lat["l1"] < lat["l2"] < lat["hbm"], lat


def test_chase_rejects_bad_chain(sl):
    bad = torch.tensor([100, 0], dtype=torch.int32, device="cuda")
    with pytest.raises(sl.SLError) as e:
        sl.sl_chase(bad, hops=4)
    assert e.value.status == sl.SL_ERR_ARG
