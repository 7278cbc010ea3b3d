"""The benchmark's single-GPU sections at small sizes: the allocation sweep,
the precision form and the batched form run end to end (device fill or host
payloads, every mechanism they time, the oracle beside them) and report
parity, so a regression in them shows in the test run and not only in the
benchmark."""
import os
import sys
import types

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def bench():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import bench as b
    import paper_2608_15764_gb300 as sl
    sl.load()
    return b


def _args(**kw):
    base = dict(steps=3, warmup=1, alloc_gib="0.015625,0.0625", prec_gib=0.0625, batch_gib=1.0,
                dtypes="f32,bf16,fp8")
    base.update(kw)
    return types.SimpleNamespace(**base)


def test_allocation_sweep_section(bench):
    import paper_2608_15764_gb300 as sl
    sec = bench.alloc_section(_args(), sl.sl_device_info())
    assert sec["parity"] and len(sec["sizes"]) == 2
    for row in sec["sizes"]:
        for order in ("asc", "desc"):
            assert row[order]["parity"] and set(row[order]["gbs"]) == set(bench.ALLOC_K)


def test_precision_section(bench):
    sec = bench.prec_section(_args())
    assert sec["parity"] and sec["max_gated_err"] <= 2e-6
    assert [p["payload"] for p in sec["per_payload"]] == ["f32", "bf16", "fp8", "bf16-cancel"]
    for p in sec["per_payload"]:
        assert len(p["points"]) == len(bench.PREC_CELLS)
        assert all(q["checksum_ok"] for q in p["points"])


def test_batched_section(bench):
    import paper_2608_15764_gb300 as sl
    sec = bench.batch_section(_args(), sl.sl_device_info())
    assert sec["parity"]
    for p in sec["per_dtype"]:
        assert p["checksums_match_oracle"] and p["baselines_match_oracle"]
        assert p["fsum_max_gated_err_sample48"] <= 2e-6
        assert p["batched_gbs"] > 0 and p["per_buffer_gbs"] > 0 and p["per_buffer_tuned_graph_gbs"] > 0
