"""Parity at the benchmark's full size: the 4 GiB uint32 splitmix64(seed=1)
buffer, filled on the GPU, in every launch configuration the benchmark
measures (its candidate set, from which it times the fastest), checked
bit-exactly against the oracle's checksum of the same words generated on the
host.  Also the 256 MiB LDG cells (K = 1, 2, 4, 8; 256 threads; 4 x SMs)."""
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


@pytest.mark.parametrize("gib", [0.25, 4])
def test_full_size_all_candidates(sl, gib):
    from paper_2608_15764_gb300 import tune
    nbytes = int(gib * (1 << 30))
    dev = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    sl.sl_fill_splitmix64(dev, seed=1)
    want = _oracle_parallel(workloads.splitmix_u32(1, nbytes // 4))
    sms = sl.sl_device_info()["sm_count"]
    points = tune.default_points()
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
