"""GPU parity of the two-co-resident-stream probe (paper §4.4) against the CPU
oracle: each stream's checksum and issued-load count are those of its own
buffer (stream B's over its passes), bit-exactly, at every warp split, K and
ragged size; timing fields are consistent."""
import pytest

import oracle
from paper_2608_15764_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NB_A = (1 << 22) + 16 * 77      # ragged for every stream width
NB_B = (1 << 23) + 16 * 1237


@pytest.fixture(scope="module")
def sl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_15764_gb300 as sl
    sl.load()
    return sl


@pytest.fixture(scope="module")
def bufs(sl):
    a = torch.empty(NB_A, dtype=torch.uint8, device="cuda")
    b = torch.empty(NB_B, dtype=torch.uint8, device="cuda")
    sl.sl_fill_splitmix64(a, seed=21)
    sl.sl_fill_splitmix64(b, seed=22)
    ha = workloads.splitmix_u32(21, NB_A // 4)
    hb = workloads.splitmix_u32(22, NB_B // 4)
    return a, b, oracle.checksum(ha), hb


@pytest.mark.parametrize("wa,wb", [(1, 0), (1, 1), (1, 16), (2, 16), (4, 8), (8, 4), (16, 16), (31, 1), (32, 0)])
@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_two_streams_parity(sl, bufs, wa, wb, k):
    a, b, ca, hb = bufs
    passes = 3
    r = sl.sl_twostream(a, b if wb else None, warps_a=wa, warps_b=wb, k=k, passes_b=passes)
    assert (r.sum_u32[0], r.xor_u64[0]) == ca
    assert r.issued_loads[0] == oracle.issued_loads(NB_A, 1)
    if wb:
        assert (r.sum_u32[1], r.xor_u64[1]) == oracle.checksum(hb, passes)
        assert r.issued_loads[1] == oracle.issued_loads(NB_B, passes)
        assert r.window_ns[1] > 0
    else:
        assert (r.sum_u32[1], r.xor_u64[1], r.issued_loads[1], r.window_ns[1]) == (0, 0, 0, 0)
        assert r.b_covers_a == 1
    assert r.cta == 32 * (wa + wb)
    assert r.grid == torch.cuda.get_device_properties(0).multi_processor_count
    assert 0 < r.window_ns[0] <= r.device_ns + 50_000
    assert r.device_ns > 0


@pytest.mark.parametrize("nvec_a,nvec_b", [(1, 1), (31, 33), (257, 4096 + 5), (40_000, 3)])
def test_two_streams_small_and_ragged(sl, bufs, nvec_a, nvec_b):
    a, b, _, _ = bufs
    ha = workloads.splitmix_u32(21, 4 * nvec_a)
    hb = workloads.splitmix_u32(22, 4 * nvec_b)
    r = sl.sl_twostream(a, b, warps_a=3, warps_b=5, k=2, passes_b=2, nbytes_a=16 * nvec_a, nbytes_b=16 * nvec_b)
    assert (r.sum_u32[0], r.xor_u64[0]) == oracle.checksum(ha)
    assert (r.sum_u32[1], r.xor_u64[1]) == oracle.checksum(hb, 2)
    assert (r.issued_loads[0], r.issued_loads[1]) == (nvec_a, 2 * nvec_b)


def test_heavy_b_covers_a(sl, bufs):
    """With B re-reading its buffer many times and A small, every B warp is
    still loading when A finishes, and B's window spans A's."""
    a, b, _, _ = bufs
    r = sl.sl_twostream(a, b, warps_a=1, warps_b=16, k=2, passes_b=256)
    assert r.b_covers_a == 1
    assert r.b_first_end_ns >= r.window_ns[0]
    assert r.window_ns[1] >= r.window_ns[0]


def test_back_to_back_calls_agree(sl, bufs):
    a, b, ca, hb = bufs
    cb = oracle.checksum(hb)
    rs = [sl.sl_twostream(a, b, warps_a=4, warps_b=4, k=4, passes_b=1) for _ in range(3)]
    for r in rs:
        assert (r.sum_u32[0], r.xor_u64[0], r.sum_u32[1], r.xor_u64[1]) == (*ca, *cb)


def test_two_stream_argument_errors(sl, bufs):
    a, b, _, _ = bufs
    E = sl.SLError
    cases = [
        (dict(warps_a=0, warps_b=1), sl.SL_ERR_ARG),
        (dict(warps_a=1, warps_b=-1), sl.SL_ERR_ARG),
        (dict(warps_a=16, warps_b=17), sl.SL_ERR_ARG),
        (dict(warps_a=1, warps_b=1, k=3), sl.SL_ERR_ARG),
        (dict(warps_a=1, warps_b=1, passes_b=-2), sl.SL_ERR_ARG),
        (dict(warps_a=1, warps_b=1, nbytes_a=1000), sl.SL_ERR_ALIGN),
        (dict(warps_a=1, warps_b=1, nbytes_a=0), sl.SL_ERR_ARG),
    ]
    for kw, code in cases:
        with pytest.raises(E) as e:
            sl.sl_twostream(a, b, **kw)
        assert e.value.status == code, kw
    with pytest.raises(E) as e:
        sl.sl_twostream(a.data_ptr() + 8, b, warps_a=1, warps_b=1, nbytes_a=1024)
    assert e.value.status == sl.SL_ERR_ALIGN
    with pytest.raises(E) as e:
        sl.sl_twostream(a, None, warps_a=1, warps_b=2)
    assert e.value.status == sl.SL_ERR_ARG
    r = sl.sl_twostream(a, None, warps_a=2, warps_b=0, k=1)
    assert r.issued_loads[0] == NB_A // 16
