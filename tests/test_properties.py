"""Property-based checks of the host logic (hypothesis; skipped where it is
not installed): the batch-size recipe, the regime rule, the fixed-iteration
arithmetic and its wrapped-read checksum, and the point catalogue."""
import math

import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
from hypothesis import given, settings  # noqa: E402

import oracle  # noqa: E402
from oracle import brute  # noqa: E402
from paper_2608_15764_gb300 import sweep, tune  # noqa: E402
from paper_2608_15764_gb300 import workloads as wl  # noqa: E402


@settings(max_examples=25, deadline=None)
@given(seed=st.integers(0, 2**63), n=st.integers(1, 300), per=st.integers(1, 64))
def test_batch_sizes_hit_the_total_within_bounds(seed, n, per):
    lo, hi, align = 64 << 10, 256 << 20, 4096
    total = n * per * (1 << 20)
    total = min(max(total, n * lo), n * hi) // align * align
    s = wl.batch_sizes(n=n, total=total, seed=seed)
    assert len(s) == n and sum(s) == total
    assert all(lo <= v <= hi and v % align == 0 for v in s)


@settings(max_examples=200, deadline=None)
@given(st.lists(st.floats(1.0, 1e4), min_size=4, max_size=16))
def test_regime_rule_is_a_partition(values):
    c = sweep.regime(values)
    mx = max(values)
    tail_ok = all(v >= 0.95 * mx for v in values[-3:])
    if tail_ok:
        assert c == "saturating"
    elif values.index(mx) < len(values) - 3 and values[-1] < 0.95 * mx:
        assert c == "peak-decline"
    else:
        assert c == "rising-censored"
    # scaling every value leaves the class unchanged
    assert sweep.regime([3.0 * v for v in values]) == c


@settings(max_examples=100, deadline=None)
@given(target=st.integers(0, 2**40), threads=st.integers(1, 1 << 20),
       ks=st.lists(st.sampled_from([1, 2, 3, 4, 6, 8, 12, 16]), min_size=1, max_size=6))
def test_fixed_iteration_arithmetic(target, threads, ks):
    issued, mm = oracle.fixed_iteration(target, threads, ks)
    for k, v in zip(ks, issued):
        assert v == (target // (threads * k)) * threads * k
        assert target - threads * k < v <= target
    assert 0.0 <= mm <= 1.0
    assert (mm == 0.0) == (len(set(issued)) == 1)


@settings(max_examples=60, deadline=None)
@given(nvec=st.integers(0, 40), nloads=st.integers(0, 200), seed=st.integers(0, 2**32 - 1))
def test_wrapped_checksum_matches_brute_force(nvec, nloads, seed):
    b = np.random.default_rng(seed).integers(0, 256, size=16 * nvec, dtype=np.uint8)
    assert oracle.wrapped_checksum(b, nloads) == brute.wrapped_checksum(b.tobytes(), nloads)


@settings(max_examples=60, deadline=None)
@given(st.sampled_from(tune.default_points()), st.integers(16, 1 << 34))
def test_point_catalogue(p, nbytes):
    nbytes = nbytes // 16 * 16
    q = tune.parse_point(p.spec())
    assert q.label() == p.label() or p.cop  # cop is not in the dynamic/32-byte specs
    assert p.loads(nbytes) in (nbytes // 16, (nbytes + 31) // 32)
    assert p.overlapped
    assert p.offered > 0 and math.isfinite(p.offered)
