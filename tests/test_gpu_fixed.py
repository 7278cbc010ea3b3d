"""GPU parity of the paper's fixed-iteration control (SL_LDG with
target_loads > 0): every thread runs floor(target / (threads*K)) iterations of
K 16-byte loads that wrap around the buffer.  The issued-load counter must
equal the oracle's fixed-iteration arithmetic, and the checksum must equal the
oracle's literal wrapped read, bit-exactly.  At the paper's primary cell
(132 CTAs x 1,024 threads, 16,785 MiB issued) the GPU's own counters
reproduce the printed 0.024576% mismatch."""
import json
import os

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
    return dev, workloads.splitmix_u32(SEED, NBYTES // 4)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 8, 16])
@pytest.mark.parametrize("cta,grid", [(256, 7), (256, 608), (1024, 152)])
@pytest.mark.parametrize("order", ["asc", "desc"])
def test_fixed_iteration_wraps(sl, data, k, cta, grid, order):
    dev, host = data
    nvec = NBYTES // 16
    target = 3 * nvec + 12345  # wraps three times and a bit
    try:
        r = sl.sl_run(dev, dtype=sl.SL_U32, cfg=sl.config("ldg", k=k, cta=cta, grid=grid, order=order,
                                                          target_loads=target))
    except sl.SLError as e:  # K=16 at 1,024 threads does not fit the register file
        assert (k, cta) == (16, 1024) and e.status == sl.SL_ERR_INFEASIBLE
        return
    issued, _ = oracle.fixed_iteration(target, grid * cta, [k])
    assert r.issued_loads == issued[0]
    assert (r.sum_u32, r.xor_u64) == oracle.wrapped_checksum(host, issued[0])


def test_fixed_iteration_below_one_wrap(sl, data):
    dev, host = data
    target = 1000 * 256 * 4 + 77
    r = sl.sl_run(dev, dtype=sl.SL_U32, cfg=sl.config("ldg", k=4, cta=256, grid=1000, target_loads=target))
    assert r.issued_loads == 1000 * 256 * 4
    assert (r.sum_u32, r.xor_u64) == oracle.checksum(host[: 4 * 1000 * 256 * 4])


def test_fixed_iteration_zero_iterations(sl, data):
    dev, _ = data
    r = sl.sl_run(dev, dtype=sl.SL_U32, cfg=sl.config("ldg", k=8, cta=256, grid=608, target_loads=1000))
    assert (r.sum_u32, r.xor_u64, r.issued_loads, r.grid) == (0, 0, 0, 0)


def test_paper_primary_cell_mismatch_on_gpu(sl, golden_dir):
    """The paper's primary-cell arithmetic (§3, §4.2) run by the kernel: 132
    CTAs of 32 warps, K = 1, 2, 4, 8, a 16,785 MiB issued volume wrapping over
    a 256 MiB buffer.  Issued loads come from the GPU's own counters."""
    g = json.load(open(os.path.join(golden_dir, "paper_fixed_work.json")))
    cta = g["warps_per_cta"] * 32
    target = g["issued_volume_mib"] * (1 << 20) // g["bytes_per_load"]
    nbytes = 256 << 20
    dev = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    sl.sl_fill_splitmix64(dev, seed=SEED)
    host = workloads.splitmix_u32(SEED, nbytes // 4)
    got = []
    want_ck = {}
    for k in g["ks"]:
        r = sl.sl_run(dev, dtype=sl.SL_U32, cfg=sl.config("ldg", k=k, cta=cta, grid=g["ctas"], target_loads=target))
        got.append(r.issued_loads)
        if r.issued_loads not in want_ck:
            want_ck[r.issued_loads] = oracle.wrapped_checksum(host, r.issued_loads)
        assert (r.sum_u32, r.xor_u64) == want_ck[r.issued_loads], k
    issued, mm = oracle.fixed_iteration(target, g["ctas"] * cta, g["ks"])
    assert got == issued
    gpu_mm = (max(got) - min(got)) / max(got)
    assert round(100 * gpu_mm, 6) == pytest.approx(g["max_mismatch_pct"], abs=5e-7)
    del dev
    torch.cuda.empty_cache()


def test_fixed_iteration_argument_errors(sl, data):
    dev, _ = data
    E = sl.SLError
    t = 1 << 24
    cases = [
        (dict(buf=dev, dtype=sl.SL_U32, cfg=sl.config("cpasync", k=2, target_loads=t)), sl.SL_ERR_ARG),
        (dict(buf=dev, dtype=sl.SL_U32, cfg=sl.config("ldg", k=2, order="dyn", target_loads=t)), sl.SL_ERR_ARG),
        (dict(buf=dev, dtype=sl.SL_F32, cfg=sl.config("ldg", k=2, target_loads=t)), sl.SL_ERR_ARG),
        (dict(buf=dev, dtype=sl.SL_U32, cfg=sl.config("ldg", k=2, passes=2, target_loads=t)), sl.SL_ERR_ARG),
        (dict(buf=dev, dtype=sl.SL_U32, cfg=sl.config("ldg", k=2, cop=1, target_loads=t)), sl.SL_ERR_ARG),
        (dict(buf=dev, dtype=sl.SL_U32, cfg=sl.config("ldg", k=5, target_loads=t)), sl.SL_ERR_ARG),
        (dict(buf=dev, dtype=sl.SL_U32, cfg=sl.config("ldg", k=2, cta=128, target_loads=t)), sl.SL_ERR_ARG),
        (dict(buf=dev, nbytes=16 * 511, dtype=sl.SL_U32, cfg=sl.config("ldg", k=2, target_loads=t)),
         sl.SL_ERR_ARG),
    ]
    for kw, code in cases:
        with pytest.raises(E) as e:
            sl.sl_run(**kw)
        assert e.value.status == code, kw
    host = torch.zeros(4096, dtype=torch.uint8).numpy()
    with pytest.raises(E) as e:
        sl.sl_run_host(host, dtype=sl.SL_U32, cfg=sl.config("ldg", k=2, target_loads=t))
    assert e.value.status == sl.SL_ERR_ARG
