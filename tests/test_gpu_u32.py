"""GPU parity of the uint32 streaming checksum against the CPU oracle, through
the C ABI: every mechanism and launch shape must give the oracle's checksum
bit-exactly, and issued loads must equal passes*bytes/16 (zero mismatch)."""
import numpy as np
import pytest

import oracle
from paper_2608_15764_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEED = 1
# several tiles of every shape plus a ragged tail (not a multiple of any tile)
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
    """Device buffer filled on the GPU, and the oracle's checksum of the same
    words generated on the host."""
    dev = torch.empty(NBYTES, dtype=torch.uint8, device="cuda")
    sl.sl_fill_splitmix64(dev, seed=SEED)
    host = workloads.splitmix_u32(SEED, NBYTES // 4)
    return dev, host, oracle.checksum(host)


def _check(sl, dev, nbytes, want, cfg, passes=1):
    r = sl.sl_run(dev, nbytes=nbytes, dtype=sl.SL_U32, cfg=cfg)
    assert r.status == 0
    assert (r.sum_u32, r.xor_u64) == want
    assert r.issued_loads == oracle.issued_loads(nbytes, passes)
    return r


def test_device_fill_matches_host_generator(sl, data):
    dev, host, _ = data
    got = dev.view(torch.int32).cpu().numpy().view(np.uint32)
    assert np.array_equal(got, host)


@pytest.mark.parametrize("k", list(range(1, 17)))
@pytest.mark.parametrize("order", ["asc", "desc"])
def test_ldg_every_k(sl, data, k, order):
    dev, _, want = data
    _check(sl, dev, NBYTES, want, sl.config("ldg", k=k, cta=256, order=order))


@pytest.mark.parametrize("cta", [32, 128, 512, 1024])
@pytest.mark.parametrize("k", [1, 3, 8])
@pytest.mark.parametrize("cop", [0, 1, 2])
def test_ldg_cta_and_cop(sl, data, cta, k, cop):
    dev, _, want = data
    _check(sl, dev, NBYTES, want, sl.config("ldg", k=k, cta=cta, cop=cop))


@pytest.mark.parametrize("grid", [1, 7, 152, 10007])
def test_ldg_grids(sl, data, grid):
    dev, _, want = data
    r = _check(sl, dev, NBYTES, want, sl.config("ldg", k=4, cta=128, grid=grid))
    assert r.grid == grid


@pytest.mark.parametrize("d", list(range(1, 9)))
@pytest.mark.parametrize("cta", [128, 256, 1024])
@pytest.mark.parametrize("order", ["asc", "desc"])
def test_cpasync_every_depth(sl, data, d, cta, order):
    dev, _, want = data
    _check(sl, dev, NBYTES, want, sl.config("cpasync", k=d, cta=cta, order=order))


@pytest.mark.parametrize("g", list(range(1, 17)))
@pytest.mark.parametrize("cta", [32, 256])
def test_ldsts_and_deep_cpasync(sl, data, g, cta):
    """The matched ld.global -> st.shared kernel (paper §4.3) at every offered
    group count, and cp.async at the same depths (up to 16)."""
    dev, _, want = data
    _check(sl, dev, NBYTES, want, sl.config("ldsts", k=g, cta=cta))
    _check(sl, dev, NBYTES, want, sl.config("cpasync", k=g, cta=cta, order="desc"))


CP_GROUPS = [(d, g) for g in (2, 4, 8) for d in range(1, 16 // g + 1)]


@pytest.mark.parametrize("d,g", CP_GROUPS)
@pytest.mark.parametrize("cta", [32, 256, 512])
@pytest.mark.parametrize("order", ["asc", "desc"])
def test_cpasync_copies_per_group(sl, data, d, g, cta, order):
    """cp.async with G copies per commit group and D groups in flight: the
    ring holds D*G slots per thread and a tile is cta*D*G vectors."""
    dev, _, want = data
    r = _check(sl, dev, NBYTES, want, sl.config("cpasync", k=d, copies=g, cta=cta, order=order))
    assert r.smem_bytes == d * g * cta * 16


CP_DYN = [(1, 1), (2, 1), (3, 1), (4, 1), (6, 1), (8, 1), (2, 2), (1, 4), (2, 4), (1, 8), (2, 8)]


@pytest.mark.parametrize("d,g", CP_DYN)
@pytest.mark.parametrize("cta", [32, 128, 256, 512])
def test_cpasync_dynamic_chunks(sl, data, d, g, cta):
    """cp.async under the SL_DYN traversal: CTAs claim ~1 MiB chunks, the
    refills cross from one chunk into the next; every instantiated D x G."""
    dev, _, want = data
    _check(sl, dev, NBYTES, want, sl.config("cpasync", k=d, copies=g, cta=cta, order="dyn"))


@pytest.mark.parametrize("grid", [1, 7, 152, 3000])
@pytest.mark.parametrize("passes", [1, 2, 3])
def test_cpasync_dynamic_grids_and_passes(sl, data, grid, passes):
    dev, _, (s, x) = data
    want = ((passes * s) % (1 << 32), x if passes % 2 else 0)
    _check(sl, dev, NBYTES, want, sl.config("cpasync", k=4, cta=256, grid=grid, order="dyn", passes=passes),
           passes=passes)


def test_cpasync_dynamic_needs_an_instantiation(sl, data):
    dev, _, _ = data
    for kw in (dict(k=5), dict(k=4, copies=2), dict(k=16)):
        with pytest.raises(sl.SLError) as e:
            sl.sl_run(dev, nbytes=1024, dtype=sl.SL_U32, cfg=sl.config("cpasync", order="dyn", **kw))
        assert e.value.status == sl.SL_ERR_ARG
    with pytest.raises(sl.SLError) as e:
        sl.sl_run(dev, nbytes=1024, dtype=sl.SL_U32, cfg=sl.config("ldsts", k=4, order="dyn"))
    assert e.value.status == sl.SL_ERR_ARG


@pytest.mark.parametrize("stage", [4096, 16384, 65536])
@pytest.mark.parametrize("stages", [2, 3, 4, 8])
@pytest.mark.parametrize("order", ["asc", "desc"])
def test_tma_ring(sl, data, stage, stages, order):
    dev, _, want = data
    cfg = sl.config("tma", cta=256, stage_bytes=stage, stages=stages, order=order)
    if stage * stages > 227 * 1024:
        with pytest.raises(sl.SLError) as e:
            sl.sl_run(dev, dtype=sl.SL_U32, cfg=cfg)
        assert e.value.status == sl.SL_ERR_INFEASIBLE
        return
    _check(sl, dev, NBYTES, want, cfg)


@pytest.mark.parametrize("cta", [32, 128, 992])
@pytest.mark.parametrize("grid", [1, 3, 0])
def test_tma_shapes(sl, data, cta, grid):
    dev, _, want = data
    _check(sl, dev, NBYTES, want, sl.config("tma", cta=cta, grid=grid, stage_bytes=16384, stages=4))


@pytest.mark.parametrize("stage", [4096, 16384, 65536])
@pytest.mark.parametrize("stages", [2, 3, 4, 8])
@pytest.mark.parametrize("order", ["asc", "desc"])
def test_tma_warp_rings(sl, data, stage, stages, order):
    """The CTA's TMA stages dealt to its warps: one, two and all stages per
    warp."""
    dev, _, want = data
    for cta in sorted({32 * stages, 32 * max(1, stages // 2) if stages % 2 == 0 else 32 * stages, 32}):
        cfg = sl.config("tma", cta=cta, stage_bytes=stage, stages=stages, order=order, ring="warp")
        try:
            sl.sl_plan(NBYTES, sl.SL_U32, cfg)
        except sl.SLError as e:
            # only a ring too large for one CTA's shared memory is refused
            assert e.status == sl.SL_ERR_INFEASIBLE and stages * (stage + 8) > 200 * 1024
            continue
        r = _check(sl, dev, NBYTES, want, cfg)
        assert r.cta == cta


@pytest.mark.parametrize("cta,grid,stages", [(32, 1, 2), (96, 3, 6), (256, 0, 8), (64, 10007, 4), (128, 0, 8)])
def test_tma_warp_ring_shapes(sl, data, cta, grid, stages):
    dev, _, want = data
    r = _check(sl, dev, NBYTES, want, sl.config("tma", cta=cta, grid=grid, stage_bytes=4096, stages=stages,
                                                ring="warp"))
    assert r.grid == (grid or r.grid)


def test_tma_warp_ring_chunk_count_limit(sl):
    """The per-warp ring counts chunks in 32 bits up to total + stages x grid:
    a launch whose chunk count is within that margin of 2^32 is refused for
    SL_RING_WARP (SL_ERR_ARG) and planned for SL_RING_CTA.  Planning only."""
    nbytes = 1 << 20                      # 256 chunks of 4 KiB
    passes = ((1 << 32) - 1024) // 256    # total = 2^32 - 1024 chunks
    warp = sl.config("tma", cta=256, stage_bytes=4096, stages=8, ring="warp", grid=608, passes=passes)
    with pytest.raises(sl.SLError) as e:
        sl.sl_plan(nbytes, sl.SL_U32, warp)
    assert e.value.status == sl.SL_ERR_ARG
    ok = sl.sl_plan(nbytes, sl.SL_U32, sl.config("tma", cta=256, stage_bytes=4096, stages=8, grid=608, passes=passes))
    assert ok.grid == 608
    fewer = sl.sl_plan(nbytes, sl.SL_U32, sl.config("tma", cta=256, stage_bytes=4096, stages=8, ring="warp", grid=608,
                                                    passes=passes - 32))
    assert fewer.grid == 608


def test_tma_warp_ring_needs_warps_dividing_stages(sl, data):
    dev, _, _ = data
    with pytest.raises(sl.SLError) as e:
        sl.sl_run(dev, dtype=sl.SL_U32, cfg=sl.config("tma", cta=96, stage_bytes=4096, stages=4, ring="warp"))
    assert e.value.status == sl.SL_ERR_ARG


@pytest.mark.parametrize("mech,kw", [("ldg", {"k": 2}), ("ldg", {"k": 13}), ("cpasync", {"k": 3}),
                                     ("cpasync", {"k": 3, "copies": 2}), ("cpasync", {"k": 2, "copies": 8}),
                                     ("tma", {"stage_bytes": 4096, "stages": 3}),
                                     ("tma", {"stage_bytes": 4096, "stages": 8, "ring": "warp"})])
@pytest.mark.parametrize("passes", [2, 3])
def test_passes_closed_form(sl, data, mech, kw, passes):
    dev, _, (s, x) = data
    want = ((passes * s) % (1 << 32), x if passes % 2 else 0)
    _check(sl, dev, NBYTES, want, sl.config(mech, cta=256, passes=passes, **kw), passes=passes)


@pytest.mark.parametrize("nvec", [0, 1, 2, 3, 31, 33, 255, 257, 4096 + 5])
@pytest.mark.parametrize("mech,kw", [("ldg", {"k": 1}), ("ldg", {"k": 16}), ("cpasync", {"k": 8}),
                                     ("cpasync", {"k": 1, "copies": 8}), ("cpasync", {"k": 5, "copies": 2}),
                                     ("cpasync", {"k": 3, "order": "dyn"}),
                                     ("cpasync", {"k": 2, "copies": 8, "order": "dyn"}),
                                     ("tma", {"stage_bytes": 4096, "stages": 2}),
                                     ("tma", {"stage_bytes": 4096, "stages": 8, "ring": "warp"}),
                                     ("tma", {"stage_bytes": 65536, "stages": 2, "ring": "warp", "cta": 32})])
def test_small_and_ragged(sl, data, nvec, mech, kw):
    dev, host, _ = data
    nbytes = 16 * nvec
    want = oracle.checksum(host[: nbytes // 4])
    _check(sl, dev, nbytes, want, sl.config(mech, **{"cta": 256, **kw}))


@pytest.mark.parametrize("k", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("cta", [128, 256, 512, 1024])
@pytest.mark.parametrize("order", ["asc", "desc"])
def test_ldg4_every_shape(sl, data, k, cta, order):
    """4-byte plain loads (paper §4.1's K1 streaming row and its K sweep): the
    same checksum; issued loads count 4-byte loads."""
    dev, _, want = data
    r = sl.sl_run(dev, nbytes=NBYTES, dtype=sl.SL_U32, cfg=sl.config("ldg4", k=k, cta=cta, order=order))
    assert (r.sum_u32, r.xor_u64) == want
    assert r.issued_loads == NBYTES // 4


@pytest.mark.parametrize("nvec", [0, 1, 2, 3, 31, 33, 255, 257, 4096 + 5])
@pytest.mark.parametrize("k", [1, 16])
def test_ldg4_small_ragged_and_passes(sl, data, nvec, k):
    dev, host, _ = data
    nbytes = 16 * nvec
    s, x = oracle.checksum(host[: nbytes // 4])
    for passes in (1, 3):
        r = sl.sl_run(dev, nbytes=nbytes, dtype=sl.SL_U32,
                      cfg=sl.config("ldg4", k=k, cta=128, grid=7, passes=passes))
        assert (r.sum_u32, r.xor_u64) == ((passes * s) % (1 << 32), x if passes % 2 else 0)
        assert r.issued_loads == passes * nbytes // 4


@pytest.mark.parametrize("mech,k", [("cpasync", 1), ("cpasync", 4), ("cpasync", 16), ("ldsts", 4), ("ldsts", 16)])
@pytest.mark.parametrize("skew", [1, 2, 4, 7])
def test_smem_skew_keeps_results(sl, data, mech, k, skew):
    """The ring-alignment experiment knob moves the shared-memory slots only."""
    dev, _, want = data
    r = sl.sl_run(dev, nbytes=NBYTES, dtype=sl.SL_U32,
                  cfg=sl.config(mech, k=k, cta=256, debug_flags=sl.SL_DEBUG_SMEM_SKEW(skew)))
    assert (r.sum_u32, r.xor_u64, r.issued_loads) == (*want, NBYTES // 16)
    assert r.smem_bytes == k * 256 * 16 + 128


@pytest.mark.parametrize("skew", [1, 7])
def test_smem_skew_with_copies_per_group(sl, data, skew):
    dev, _, want = data
    r = sl.sl_run(dev, nbytes=NBYTES, dtype=sl.SL_U32,
                  cfg=sl.config("cpasync", k=2, copies=4, cta=256, debug_flags=sl.SL_DEBUG_SMEM_SKEW(skew)))
    assert (r.sum_u32, r.xor_u64, r.issued_loads) == (*want, NBYTES // 16)
    assert r.smem_bytes == 2 * 4 * 256 * 16 + 128


def test_ldg4_rejects_other_forms(sl, data):
    dev, _, _ = data
    for kw, dtype, code in [(dict(k=3), sl.SL_U32, sl.SL_ERR_ARG), (dict(k=1, cta=32), sl.SL_U32, sl.SL_ERR_ARG),
                            (dict(k=1), sl.SL_F32, sl.SL_ERR_ARG), (dict(k=1, cop=1), sl.SL_U32, sl.SL_ERR_ARG),
                            (dict(k=1, order="dyn"), sl.SL_U32, sl.SL_ERR_ARG)]:
        with pytest.raises(sl.SLError) as e:
            sl.sl_run(dev, nbytes=1024, dtype=dtype, cfg=sl.config("ldg4", **kw))
        assert e.value.status == code, kw


def _ldg32_loads(nbytes, passes=1):
    return passes * ((nbytes + 31) // 32)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 6, 8])
@pytest.mark.parametrize("cta", [128, 256, 512])
@pytest.mark.parametrize("order", ["asc", "desc", "dyn"])
def test_ldg32_every_shape(sl, data, k, cta, order):
    """32-byte loads (ld.global.v8): the same checksum at every K, CTA size
    and traversal; the buffer ends in a half unit (an odd number of 16-byte
    vectors), which one thread reads with a 16-byte load."""
    dev, _, want = data
    assert (NBYTES // 16) % 2 == 1
    for _ in range(2 if order == "dyn" else 1):
        r = sl.sl_run(dev, nbytes=NBYTES, dtype=sl.SL_U32, cfg=sl.config("ldg32", k=k, cta=cta, order=order))
        assert (r.sum_u32, r.xor_u64) == want
        assert r.issued_loads == _ldg32_loads(NBYTES)


@pytest.mark.parametrize("nvec", [0, 1, 2, 3, 31, 33, 255, 257, 4096 + 5, 65536 * 3 + 1])
@pytest.mark.parametrize("k", [1, 8])
@pytest.mark.parametrize("order", ["asc", "dyn"])
def test_ldg32_small_ragged_and_passes(sl, data, nvec, k, order):
    dev, host, _ = data
    nbytes = 16 * nvec
    s, x = oracle.checksum(host[: nbytes // 4])
    for passes in (1, 3):
        r = sl.sl_run(dev, nbytes=nbytes, dtype=sl.SL_U32,
                      cfg=sl.config("ldg32", k=k, cta=128, grid=7, passes=passes, order=order))
        assert (r.sum_u32, r.xor_u64) == ((passes * s) % (1 << 32), x if passes % 2 else 0)
        assert r.issued_loads == _ldg32_loads(nbytes, passes)


def test_ldg32_needs_32_byte_alignment(sl, data):
    dev, host, _ = data
    with pytest.raises(sl.SLError) as e:
        sl.sl_run(dev.data_ptr() + 16, nbytes=4096, dtype=sl.SL_U32, cfg=sl.config("ldg32", k=2))
    assert e.value.status == sl.SL_ERR_ALIGN
    r = sl.sl_run(dev.data_ptr() + 32, nbytes=4096 + 16, dtype=sl.SL_U32, cfg=sl.config("ldg32", k=2))
    assert (r.sum_u32, r.xor_u64) == oracle.checksum(host[8: 8 + (4096 + 16) // 4])
    for kw in (dict(k=5), dict(k=16), dict(k=2, cta=1024), dict(k=2, cop=1)):
        with pytest.raises(sl.SLError) as e:
            sl.sl_run(dev, nbytes=4096, dtype=sl.SL_U32, cfg=sl.config("ldg32", **kw))
        assert e.value.status == sl.SL_ERR_ARG, kw


@pytest.mark.parametrize("k", [1, 2, 3, 4, 6, 8, 12, 16])
@pytest.mark.parametrize("cta", [128, 256, 512])
def test_ldg_dynamic_chunks(sl, data, k, cta):
    """SL_DYN: CTAs claim ~1 MiB contiguous chunks from a counter; the counter
    is reset by the last CTA, so back-to-back launches all cover the buffer
    exactly once."""
    dev, _, want = data
    for grid in (0, 5):
        for _ in range(2):
            r = _check(sl, dev, NBYTES, want, sl.config("ldg", k=k, cta=cta, grid=grid, order="dyn"))
    _check(sl, dev, NBYTES, ((3 * want[0]) % (1 << 32), want[1]),
           sl.config("ldg", k=k, cta=cta, order="dyn", passes=3), passes=3)


@pytest.mark.parametrize("nvec", [0, 1, 33, 4096 + 5, 65536, 65536 + 17, 3 * 65536 + 1])
def test_ldg_dynamic_ragged(sl, data, nvec):
    dev, host, _ = data
    nbytes = 16 * nvec
    _check(sl, dev, nbytes, oracle.checksum(host[: nbytes // 4]), sl.config("ldg", k=4, cta=256, order="dyn"))


def test_dynamic_rejected_outside_its_kernels(sl, data):
    """SL_DYN runs on the LDG, 32-byte LDG and cp.async kernels only."""
    dev, _, _ = data
    for cfg in [sl.config("tma", order="dyn"), sl.config("ldsts", order="dyn"), sl.config("cpasync", k=5, order="dyn"),
                sl.config("ldg", k=5, order="dyn"), sl.config("ldg", k=2, cop=1, order="dyn")]:
        with pytest.raises(sl.SLError) as e:
            sl.sl_run(dev, dtype=sl.SL_U32, cfg=cfg)
        assert e.value.status == sl.SL_ERR_ARG


def test_empty_buffer(sl):
    r = sl.sl_run(0, nbytes=0, dtype=sl.SL_U32, cfg=sl.config("ldg", k=2))
    assert (r.sum_u32, r.xor_u64, r.issued_loads, r.grid) == (0, 0, 0, 0)


def test_offset_views(sl, data):
    """A buffer that starts 16 bytes into the allocation (aligned, not at a
    tile boundary of anything)."""
    dev, host, _ = data
    nbytes = NBYTES - 64
    want = oracle.checksum(host[4: 4 + nbytes // 4])
    for cfg in [sl.config("ldg", k=4), sl.config("cpasync", k=2), sl.config("cpasync", k=3, copies=4),
                sl.config("tma", stage_bytes=16384, stages=4)]:
        r = sl.sl_run(dev.data_ptr() + 16, nbytes=nbytes, dtype=sl.SL_U32, cfg=cfg)
        assert (r.sum_u32, r.xor_u64) == want


def test_argument_errors(sl, data):
    dev, _, _ = data
    E = sl.SLError
    cases = [
        (dict(buf=dev.data_ptr() + 8, nbytes=1024, cfg=sl.config("ldg")), sl.SL_ERR_ALIGN),
        (dict(buf=dev, nbytes=1000, cfg=sl.config("ldg")), sl.SL_ERR_ALIGN),
        (dict(buf=dev, nbytes=1024, cfg=sl.config("ldg", k=0)), sl.SL_ERR_ARG),
        (dict(buf=dev, nbytes=1024, cfg=sl.config("ldg", k=17)), sl.SL_ERR_ARG),
        (dict(buf=dev, nbytes=1024, cfg=sl.config("ldg", cta=100)), sl.SL_ERR_ARG),
        (dict(buf=dev, nbytes=1024, cfg=sl.config("ldg", cta=64)), sl.SL_ERR_ARG),
        (dict(buf=dev, nbytes=1024, cfg=sl.config("cpasync", k=17)), sl.SL_ERR_ARG),
        (dict(buf=dev, nbytes=1024, cfg=sl.config("ldsts", k=0)), sl.SL_ERR_ARG),
        (dict(buf=dev, nbytes=1024, cfg=sl.config("cpasync", k=2, copies=3)), sl.SL_ERR_ARG),
        (dict(buf=dev, nbytes=1024, cfg=sl.config("cpasync", k=2, copies=16)), sl.SL_ERR_ARG),
        (dict(buf=dev, nbytes=1024, cfg=sl.config("cpasync", k=2, copies=-1)), sl.SL_ERR_ARG),
        (dict(buf=dev, nbytes=1024, cfg=sl.config("cpasync", k=3, copies=8)), sl.SL_ERR_ARG),
        (dict(buf=dev, nbytes=1024, cfg=sl.config("cpasync", k=9, copies=2)), sl.SL_ERR_ARG),
        (dict(buf=dev, nbytes=1024, cfg=sl.config("ldg", k=2, copies=2)), sl.SL_ERR_ARG),
        (dict(buf=dev, nbytes=1024, cfg=sl.config("ldsts", k=2, copies=2)), sl.SL_ERR_ARG),
        (dict(buf=dev, nbytes=1024, cfg=sl.config("cpasync", k=4, copies=4, cta=1024)), sl.SL_ERR_INFEASIBLE),
        (dict(buf=dev, nbytes=1024, cfg=sl.config("tma", stage_bytes=8192)), sl.SL_ERR_INFEASIBLE),
        (dict(buf=dev, nbytes=1024, cfg=sl.config("tma", stages=1)), sl.SL_ERR_ARG),
        (dict(buf=dev, nbytes=1024, cfg=sl.config("tma", stage_bytes=65536, stages=4)), sl.SL_ERR_INFEASIBLE),
        (dict(buf=dev, nbytes=1024, cfg=sl.config("ldg", k=16, cta=1024)), sl.SL_ERR_INFEASIBLE),
        (dict(buf=dev, nbytes=1024, cfg=sl.config("ldg", passes=-1)), sl.SL_ERR_ARG),
        (dict(buf=dev, nbytes=1024, cfg=sl.config(7)), sl.SL_ERR_ARG),
        (dict(buf=0, nbytes=1024, cfg=sl.config("ldg")), sl.SL_ERR_ARG),
    ]
    for kw, code in cases:
        with pytest.raises(E) as e:
            sl.sl_run(kw["buf"], nbytes=kw["nbytes"], dtype=sl.SL_U32, cfg=kw["cfg"])
        assert e.value.status == code, (kw, e.value)
        assert sl.sl_last_error()
    with pytest.raises(E) as e:
        sl.sl_run(dev, nbytes=1024, dtype=9, cfg=sl.config("ldg"))
    assert e.value.status == sl.SL_ERR_ARG
    # the context is still fine afterwards
    r = sl.sl_run(dev, nbytes=1024, dtype=sl.SL_U32, cfg=sl.config("ldg"))
    assert r.issued_loads == 64


def test_sweep_orders_agree(sl, data):
    dev, _, want = data
    cells = [sl.config("ldg", k=k) for k in (1, 2, 4, 8)] + [sl.config("tma", stage_bytes=65536, stages=4)]
    asc = sl.sl_sweep(dev, cells, dtype=sl.SL_U32, repeats=2, warmup=1, sweep_order="asc")
    desc = sl.sl_sweep(dev, cells, dtype=sl.SL_U32, repeats=2, warmup=1, sweep_order="desc")
    for rows in (asc, desc):
        for row in rows[:4]:
            for r in row:
                assert r.status == 0 and (r.sum_u32, r.xor_u64) == want and r.device_ns > 0
        assert all(r.status == sl.SL_ERR_INFEASIBLE for r in rows[4])


def test_enqueue_many_on_one_stream(sl, data):
    dev, _, want = data
    n = 40
    rb = sl.RESULT_BYTES
    out = torch.zeros(rb * n, dtype=torch.uint8, device="cuda")
    cfgs = [sl.config("ldg", k=1 + i % 16) if i % 3 == 0 else
            sl.config("cpasync", k=1 + i % 8) if i % 3 == 1 else
            sl.config("tma", stage_bytes=4096 << (2 * (i % 2)), stages=2 + i % 5) for i in range(n)]
    for i, c in enumerate(cfgs):
        sl.sl_enqueue(dev, out[rb * i:], dtype=sl.SL_U32, cfg=c)
    torch.cuda.synchronize()
    raw = out.cpu().numpy().tobytes()
    for i in range(n):
        r = sl.sl_result.from_buffer_copy(raw[rb * i: rb * (i + 1)])
        assert (r.sum_u32, r.xor_u64, r.status) == (*want, 0)
        assert r.issued_loads == NBYTES // 16


@pytest.mark.parametrize("mech,kw", [("ldg", {"k": 4}), ("tma", {"stage_bytes": 16384, "stages": 4}),
                                     ("ldg", {"k": 4, "order": "dyn"}),
                                     ("ldg", {"k": 8, "order": "dyn", "host_direct": True}),
                                     ("ldg", {"k": 3, "host_direct": True}),
                                     ("tma", {"stage_bytes": 65536, "stages": 3, "host_direct": True}),
                                     ("cpasync", {"k": 4, "host_direct": True})])
def test_run_host_matches(sl, data, mech, kw):
    _, host, want = data
    pinned = torch.from_numpy(host.view(np.uint8)).pin_memory()
    r = sl.sl_run_host(pinned, dtype=sl.SL_U32, cfg=sl.config(mech, **kw))
    assert (r.sum_u32, r.xor_u64) == want and r.issued_loads == NBYTES // 16
    # pageable numpy memory works too
    r = sl.sl_run_host(host, dtype=sl.SL_U32, cfg=sl.config(mech, **kw))
    assert (r.sum_u32, r.xor_u64) == want


def test_device_info(sl):
    info = sl.sl_device_info()
    assert info["sm_count"] > 0 and info["l2_bytes"] > 0
    assert (info["cc_major"], info["cc_minor"]) == (10, 3)
