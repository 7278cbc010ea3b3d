"""Host-side pieces of bench.py that need no GPU: the oracle's prefix
checksums of the allocation sweep (against whole-buffer checksums) and the
tile count behind the tuned per-buffer grids."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402
from paper_2608_15764_gb300 import workloads  # noqa: E402


def test_prefix_checksums_match_whole_buffers():
    piece = 16 << 20
    sizes = [piece, 3 * piece]
    cks, gbs, sec = bench.oracle_prefix_checksums(1, sizes, threads=4)
    assert gbs > 0 and sec > 0
    for s in sizes:
        assert cks[s] == oracle.checksum(workloads.splitmix_u32(1, s // 4))
    with pytest.raises(AssertionError):
        bench.oracle_prefix_checksums(1, [piece + 16], threads=2)


def test_tiles_per_mechanism():
    import paper_2608_15764_gb300 as sl
    assert bench._tiles(sl.config("ldg", k=4, cta=256), 16 * 1024) == 1
    assert bench._tiles(sl.config("ldg", k=4, cta=256), 16 * 1025) == 2
    assert bench._tiles(sl.config("cpasync", k=2, cta=128), 16 * 256 * 3) == 3
    assert bench._tiles(sl.config("tma", stage_bytes=16384, stages=4), 16384 * 5 + 16) == 6


def test_kernel_hash_ignores_comments_only():
    """Counters stay attached to the kernels' code: comment and layout edits
    keep the hash, any code edit changes it."""
    from paper_2608_15764_gb300 import build
    a = "int f(int x) {\n    return x + 1;  // one\n}\n"
    b = "/* the same\n   function */\nint f(int x)\n{ return x + 1; }\n"
    c = "int f(int x) {\n    return x + 2;  // one\n}\n"
    assert build._code_only(a) == build._code_only(b)
    assert build._code_only(a) != build._code_only(c)
    assert len(build.kernel_source_hash()) == 16


def test_alloc_counters_match_the_sweep_sizes():
    """The committed single-pass allocation counters cover every size of the
    benchmark's allocation sweep at both K endpoints, for the current kernels."""
    import bench
    sizes = [int(g * (1 << 30)) for g in (0.5, 1, 2, 4, 8, 16, 20)]
    r = bench._alloc_counters(sizes)
    if r.get("note") == "kernels changed since the counters were taken":
        pytest.skip("the allocation counters were taken on another version of the kernels' code")
    assert "note" not in r, r
    assert sorted(int(b) for b in r["per_size"]) == sizes
    for per_k in r["per_size"].values():
        assert set(per_k) == {"k2", "k8"}
        for v in per_k.values():
            assert abs(v["dram_read_over_bytes"] - 1) < 1e-3 and abs(v["l2_read_hit_derived"]) < 1e-3


def test_traffic_counters_name_catalogue_points():
    """profiles/traffic.json: every captured point is a point of the benchmark's
    catalogue (its label is what bench.py looks up), with DRAM reads within
    0.1% of the bytes, and the benchmark's usual choices are among them."""
    import json
    from paper_2608_15764_gb300 import tune
    from paper_2608_15764_gb300.build import kernel_source_hash
    doc = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    if doc["kernel_source_hash"] != kernel_source_hash():
        pytest.skip("the traffic counters were taken on another version of the kernels' code")
    labels = {p.label() for p in tune.default_points()}
    assert set(doc["points"]) <= labels
    for e in doc["points"].values():
        assert abs(e["dram_read"] / e["bytes"] - 1) < 1e-3
        assert tune.parse_point(e["spec"]).label() in doc["points"]
    for spec in ("ldgdyn:4:512", "ldgdyn:4:256", "ldgdyn:2:512", "ldg32dyn:2:256"):
        assert tune.parse_point(spec).label() in doc["points"]


def test_counter_files_from_other_kernels_are_not_reported(tmp_path, monkeypatch):
    """Counters taken on another version of the kernels' code are reported as
    such (a note, no numbers), and a missing file is noted too."""
    import json
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._alloc_counters([1 << 30]) == {"note": "no profiles/alloc_counters.json"}
    assert bench._traffic("ldg K=4 cta=512 cop=0 dyn", 4 << 30) == (None, "no profiles/traffic.json")
    (tmp_path / "profiles" / "alloc_counters.json").write_text(json.dumps({"kernel_source_hash": "0", "rows": []}))
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"kernel_source_hash": "0", "points": {}}))
    assert bench._alloc_counters([1 << 30]) == {"note": "kernels changed since the counters were taken"}
    assert bench._traffic("ldg K=4 cta=512 cop=0 dyn", 4 << 30)[0] is None
