"""Coverage audit (sl_coverage): the coverage instantiations count every load
per 16-byte vector.  Under exact fixed work every vector must be loaded
exactly `passes` times -- no vector skipped, none read twice -- at every
mechanism, shape, traversal and ragged size; under the paper's
fixed-iteration control the counts must follow the wrapped read (the first r
vectors q+1 times, the rest q times, for issued = q*n + r).  The checksums of
the same runs are checked against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2608_15764_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEED = 1
NBYTES = (1 << 24) + 16 * 1237  # an odd number of 16-byte vectors: 32-byte loads end in a half unit

CONFIGS = [
    ("ldg", dict(k=1, cta=128)), ("ldg", dict(k=3, cta=256)), ("ldg", dict(k=8, cta=512, order="desc")),
    ("ldg", dict(k=16, cta=256, grid=7)), ("ldg", dict(k=2, cta=256, order="dyn")),
    ("ldg", dict(k=12, cta=512, order="dyn")),
    ("ldg32", dict(k=1, cta=256)), ("ldg32", dict(k=3, cta=256, order="desc")), ("ldg32", dict(k=8, cta=256)),
    ("ldg32", dict(k=3, cta=256, order="dyn")), ("ldg32", dict(k=8, cta=256, order="dyn")),
    ("cpasync", dict(k=1, cta=256)), ("cpasync", dict(k=4, cta=128)), ("cpasync", dict(k=16, cta=256)),
    ("cpasync", dict(k=2, copies=4, cta=256)), ("cpasync", dict(k=3, copies=2, cta=128, order="desc")),
    ("cpasync", dict(k=4, cta=256, order="dyn")), ("cpasync", dict(k=2, copies=4, cta=128, order="dyn")),
    ("ldsts", dict(k=1, cta=256)), ("ldsts", dict(k=16, cta=256)),
    ("tma", dict(cta=256, stage_bytes=16384, stages=4)), ("tma", dict(cta=128, stage_bytes=4096, stages=2,
                                                                      order="desc")),
    ("tma", dict(cta=256, stage_bytes=4096, stages=8, ring="warp")),
    ("tma", dict(cta=64, stage_bytes=16384, stages=4, ring="warp", order="desc")),
]


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
    counts = torch.empty(NBYTES // 16, dtype=torch.int32, device="cuda")
    return dev, host, counts


def _counts(counts, n):
    return counts[:n].cpu().numpy()


@pytest.mark.parametrize("mech,kw", CONFIGS)
@pytest.mark.parametrize("passes", [1, 3])
def test_every_vector_read_exactly_passes_times(sl, data, mech, kw, passes):
    dev, host, counts = data
    r = sl.sl_coverage(dev, counts, cfg=sl.config(mech, passes=passes, **kw))
    c = _counts(counts, NBYTES // 16)
    assert c.min() == passes and c.max() == passes, (np.flatnonzero(c != passes)[:8], c.min(), c.max())
    s, x = oracle.checksum(host)
    assert (r.sum_u32, r.xor_u64) == ((passes * s) % (1 << 32), x if passes % 2 else 0)


@pytest.mark.parametrize("nvec", [1, 2, 33, 4096 + 5, 65536 * 2 + 3])
@pytest.mark.parametrize("mech,kw", [("ldg", dict(k=16, cta=256)), ("ldg", dict(k=12, cta=256, order="dyn")),
                                     ("ldg32", dict(k=8, cta=256, order="dyn")), ("cpasync", dict(k=16, cta=256)),
                                     ("tma", dict(cta=256, stage_bytes=4096, stages=3)),
                                     ("tma", dict(cta=256, stage_bytes=4096, stages=8, ring="warp"))])
def test_small_and_ragged_coverage(sl, data, nvec, mech, kw):
    dev, host, counts = data
    counts.fill_(-1)
    r = sl.sl_coverage(dev, counts, nbytes=16 * nvec, cfg=sl.config(mech, **kw))
    c = counts.cpu().numpy()
    assert (c[:nvec] == 1).all()
    assert (c[nvec:] == -1).all()  # nothing beyond the buffer is counted (or zeroed)
    assert (r.sum_u32, r.xor_u64) == oracle.checksum(host[: 4 * nvec])


@pytest.mark.parametrize("k,cta", [(2, 256), (8, 256), (2, 1024), (8, 1024)])
@pytest.mark.parametrize("order", ["asc", "desc"])
def test_fixed_iteration_coverage_follows_the_wrap(sl, data, k, cta, order):
    dev, host, counts = data
    n = NBYTES // 16
    target = 2 * n + 54321
    r = sl.sl_coverage(dev, counts, cfg=sl.config("ldg", k=k, cta=cta, grid=152, order=order, target_loads=target))
    issued, _ = oracle.fixed_iteration(target, 152 * cta, [k])
    q, rem = divmod(issued[0], n)
    c = _counts(counts, n)
    assert (c[:rem] == q + 1).all() and (c[rem:] == q).all()
    assert r.issued_loads == issued[0]
    assert (r.sum_u32, r.xor_u64) == oracle.wrapped_checksum(host, issued[0])


def test_coverage_rejects_shapes_without_instantiation(sl, data):
    dev, _, counts = data
    for mech, kw in [("ldg", dict(k=5)), ("ldg", dict(k=3, cop=1)), ("ldg4", dict(k=1)), ("cpasync", dict(k=3)),
                     ("ldg32", dict(k=2)), ("ldg", dict(k=2, target_loads=1 << 24, cta=512))]:
        with pytest.raises(sl.SLError) as e:
            sl.sl_coverage(dev, counts, cfg=sl.config(mech, **kw))
        assert e.value.status == sl.SL_ERR_ARG, (mech, kw)
