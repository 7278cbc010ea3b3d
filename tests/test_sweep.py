"""Host logic of the collection harness (no GPU): the endpoint-change formula
against the paper's printed table, the cell grids of each configuration, and
the resume keys."""
import json
import os

import pytest

from paper_2608_15764_gb300 import sweep


def test_decline_matches_paper_table1(golden_dir):
    """The printed bandwidths are rounded to 0.1 GB/s and the change to 0.1%,
    so the formula must land inside the interval those roundings allow (the
    first row, 3111.0 -> 1989.5 printed as -36.1%, is -36.05% from the rounded
    inputs).  A wrong formula (another denominator, a sign flip) misses it by
    whole percents."""
    g = json.load(open(os.path.join(golden_dir, "paper_table1.json")))
    for row in g["rows"]:
        k2, k8 = row["k2_gbs"], row["k8_gbs"]
        lo = sweep.decline(k2 + 0.05, k8 - 0.05)
        hi = sweep.decline(k2 - 0.05, k8 + 0.05)
        assert lo - 0.05 <= row["change_pct"] <= hi + 0.05, row["arm"]
        assert abs(sweep.decline(k2, k8) - row["change_pct"]) < 0.06, row["arm"]
    assert sweep.decline(100.0, 50.0) == -50.0 and sweep.decline(50.0, 100.0) == 100.0


def test_cell_grids():
    sms = 152
    c1 = list(sweep._cells("c1", sms))
    assert [c["k"] for c in c1] == [1, 2, 4, 8] and all(c["grid"] == 4 * sms and c["gib"] == 0.25 for c in c1)
    c2 = list(sweep._cells("c2", sms))
    assert len(c2) == 3 * 8 * 8
    assert {c["grid"] for c in c2} == {r * sms for r in range(1, 9)}
    assert {c["k"] for c in c2} == {1, 2, 3, 4, 6, 8, 12, 16}
    c3 = list(sweep._cells("c3", sms))
    assert sum(c["mech"] == "ldg" and not c.get("trav") for c in c3) == 16
    assert sum(c["mech"] == "ldg" and c.get("trav") == 2 for c in c3) == 8
    assert sum(c["mech"] == "cpasync" for c in c3) == 8
    assert sum(c["mech"] == "tma" and c.get("ring", "cta") == "cta" for c in c3) == 21 + 7
    # the stages dealt to the warps: one per warp at every count, two per warp at even counts
    assert sum(c["mech"] == "tma" and c.get("ring") == "warp" for c in c3) == 3 * (7 + 4)
    assert all(c["stages"] % (c["cta"] // 32) == 0 for c in c3 if c.get("ring") == "warp")
    c4 = list(sweep._cells("c4", sms))
    assert sorted({c["gib"] for c in c4}) == [0.5, 1, 2, 4, 8, 16, 20]
    prim = list(sweep._cells("primary", sms))
    assert all(c["cta"] == 1024 and c["grid"] == sms for c in prim)  # 132 x 32 warps on H100 -> 152 x 32 here


def test_resume_keys_distinguish_order():
    c = next(sweep._cells("c1", 152))
    assert sweep._key(c, "asc") != sweep._key(c, "desc")
    assert json.loads(sweep._key(c, "asc"))["order"] == "asc"


def test_summarize_endpoint_change():
    rows = [{"config": "c1", "mech": "ldg", "status": 0, "gib": 1, "cta": 256, "grid": 608, "order": "asc",
             "k": k, "gbs_median": v} for k, v in [(2, 3058.8), (8, 1988.7)]]
    s = sweep.summarize(rows)
    assert s == [{"config": "c1", "gib": 1, "cta": 256, "grid": 608, "order": "asc", "k2": 3058.8,
                  "k8": 1988.7, "change_pct": -34.98}]


def test_cp_ratio_pairs_mechanisms():
    rows = [{"config": "cpratio", "status": 0, "warps_per_sm": 1, "k": 16, "order": "asc", "mech": m, "gbs_median": v}
            for m, v in (("cpasync", 290.0), ("ldsts", 100.0))]
    assert sweep.cp_ratio(rows) == [{"warps_per_sm": 1, "groups": 16, "order": "asc", "cpasync_gbs": 290.0,
                                     "ldsts_gbs": 100.0, "ratio": 2.9}]
    cells = list(sweep._cells("cpratio", 152))
    assert len(cells) == 2 * 6 * 2 and {c["cta"] for c in cells} == {32, 256}


def test_regime_rule():
    assert sweep.regime([1, 2, 3, 10, 9.9, 9.8]) == "saturating"
    assert sweep.regime([1, 10, 9, 8, 7, 6]) == "peak-decline"
    assert sweep.regime([1, 2, 3, 4, 5, 6]) == "rising-censored"
    # the paper's H100 primary cell (K=2 peak, -35% at K=8) is a peak-decline
    assert sweep.regime([2000, 3059, 2700, 2300, 2100, 1989]) == "peak-decline"
    # a maximum inside the tail that the last cell falls from is not a decline yet
    assert sweep.regime([1, 2, 3, 10, 5, 9]) == "rising-censored"
    with pytest.raises(ValueError):
        sweep.regime([1, 2, 3])


def test_regime_map_groups_curves():
    rows = [{"config": "c2", "status": 0, "cta": 256, "resident_req": 4, "order": "asc", "k": k, "gbs_median": v}
            for k, v in zip((1, 2, 3, 4, 6, 8), (10, 20, 30, 40, 39.5, 39))]
    assert sweep.regime_map(rows) == {(16, 256, 4, "asc"): "saturating"}
    wide = [dict(r, config="c2w", mech="ldg32") for r in rows]
    falling = [dict(r, config="c2w", mech="ldg4", gbs_median=100 - r["k"]) for r in rows]
    assert sweep.regime_map(rows + wide + falling) == {(16, 256, 4, "asc"): "saturating",
                                                        (32, 256, 4, "asc"): "saturating",
                                                        (4, 256, 4, "asc"): "peak-decline"}


def test_fixed_mismatch_summary():
    """The GPU-counter form of the paper's §4.2 mismatch: issued loads per K
    from the fixed-iteration cells, largest relative spread across K."""
    threads, target = 132 * 1024, 16785 * (1 << 20) // 16
    rows = []
    for k in (1, 2, 4, 8):
        issued = target // (threads * k) * threads * k
        rows.append({"config": "fixedit", "target_loads": target, "status": 0, "issued": issued, "gib": 0.5,
                     "grid": 132, "order": "asc", "k": k})
    (s,) = sweep.fixed_mismatch(rows)
    assert s["max_mismatch_pct"] == 0.024576
    assert s["issued"]["1"] == s["issued"]["2"] == 8138 * threads


def test_tune_points_specs_loads_and_choice():
    """Host logic of the point catalogue: specs round-trip, config overrides,
    per-width load counts, overlap eligibility and the two choice rules."""
    from paper_2608_15764_gb300 import SL_DYN, SL_LDG32, tune
    pts = tune.default_points()
    for p in pts:
        q = tune.parse_point(p.spec())
        assert (q.mech, q.k, q.cta, q.order, q.stage_bytes, q.stages, q.ring, q.copies) == \
            (p.mech, p.k, p.cta, p.order, p.stage_bytes, p.stages, p.ring, p.copies), p.spec()
    # the catalogue: LDG K 1-16, cp.async D 1-8, TMA 4/16/64 KiB x 2-8 in both ring layouts, every
    # per-warp point with a warp count dividing its stage count
    from paper_2608_15764_gb300 import SL_CPASYNC, SL_LDG, SL_RING_WARP, SL_TMA
    assert sorted(q.k for q in pts if q.mech == SL_LDG and q.order == 0 and q.cop == 0) == list(range(1, 17))
    assert sorted(q.k for q in pts if q.mech == SL_CPASYNC and q.copies == 1 and q.order == 0) == list(range(1, 9))
    assert {(q.k, q.copies) for q in pts if q.mech == SL_CPASYNC and q.copies > 1 and q.order == 0} == \
        {(1, 2), (2, 2), (1, 4), (2, 4), (1, 8)}
    assert {(q.k, q.copies) for q in pts if q.mech == SL_CPASYNC and q.order == SL_DYN} == set(tune.CP_DYN_POINTS)
    d = tune.parse_point("cpasyncdyn:2:256:8")
    assert (d.order, d.spec(), d.label(), d.cfg().order) == (SL_DYN, "cpasyncdyn:2:256:8", "cpasync D=2 G=8 cta=256 dyn",
                                                             SL_DYN)
    assert tune.parse_point("cpasyncdyn:4:256").spec() == "cpasyncdyn:4:256"
    g = tune.parse_point("cpasync:2:256:4")
    assert (g.k, g.copies, g.offered, g.spec()) == (2, 4, 2 * 4 * 256 * 16, "cpasync:2:256:4")
    assert g.cfg().copies == 4 and g.label() == "cpasync D=2 G=4 cta=256" and g.as_dict()["copies"] == 4
    for ring in (0, SL_RING_WARP):
        got = {(q.stage_bytes, q.stages) for q in pts if q.mech == SL_TMA and q.ring == ring}
        assert got == {(s, n) for s in (4096, 16384, 65536) for n in range(2, 9)}
    assert all(q.stages % (q.cta // 32) == 0 for q in pts if q.mech == SL_TMA and q.ring == SL_RING_WARP)
    w = tune.parse_point("tmaw:4096:8")
    assert (w.ring, w.cta, w.offered) == (SL_RING_WARP, 256, 8 * 4096) and "per-warp" in w.label()
    p = tune.parse_point("ldg32dyn:6:256")
    assert p.mech == SL_LDG32 and p.order == SL_DYN and p.overlapped
    assert p.cfg(grid=0).grid == 0 and p.cfg().order == SL_DYN and p.cfg(order="asc").order == 0
    assert p.loads(4096 + 16) == 129 and tune.parse_point("ldg:2:256").loads(4096 + 16) == 257
    assert tune.parse_point("ldg:3:256").overlapped and tune.parse_point("tma:16384:2:256").overlapped
    a, b, c = tune.parse_point("ldg:2:256"), tune.parse_point("ldg:8:256"), tune.parse_point("tma:65536:2:256")
    a.gbs, b.gbs, c.gbs = [7000.0], [7300.0], [7310.0]
    a.step_gbs, b.step_gbs, c.step_gbs = [7500.0], [7400.0], []
    assert tune.choose([a, b, c]) is b          # within 0.5% of the best: fewer bytes in flight
    assert tune.choose([a, b, c], steps=True) is a


def test_counter_capture_configs_stay_small():
    """Every counter-capture configuration for multi-pass metric sets is one or
    two launches on at most 2 GiB (the capture-size rule); ncu-alloc1, the
    one that reaches 20 GiB, is for single-pass metric sets and runs one
    launch per cell."""
    from paper_2608_15764_gb300 import sweep
    sms = 152
    for cfg, kw in [("ncu-primary", {}), ("ncu-fixed", {}), ("ncu-cpskew", {}), ("ncu-point", {"point": "ldgdyn:2:512"}),
                    ("ncu-point", {"point": "tmaw:4096:8:256"}), ("ncu-point", {"point": "tma:65536:2:256"})]:
        cells = list(sweep._cells(cfg, sms, **kw))
        assert 1 <= len(cells) <= 2 and all(c["gib"] <= 2 for c in cells), cfg
    w = list(sweep._cells("ncu-point", sms, point="tmaw:4096:8:256"))[0]
    assert (w["mech"], w["ring"], w["stages"], w["cta"]) == ("tma", "warp", 8, 256)
    with pytest.raises(ValueError):
        list(sweep._cells("ncu-alloc", sms))
    a = list(sweep._cells("ncu-alloc1", sms, gib=20))
    assert [(c["gib"], c["k"]) for c in a] == [(g, k) for g in sweep.ALLOC_GIB for k in (2, 8)]
    assert len(list(sweep._cells("ncu-alloc1", sms))) == 4  # default --gib 1: 512 MiB and 1 GiB
    c2 = list(sweep._cells("ncu-c2", sms))
    assert len(c2) == 4 * 6 and all(c["gib"] == 4 and c["cta"] * c["resident_req"] == 1024 for c in c2)


def test_traffic_writer_reads_single_launch_captures(tmp_path):
    """The ncu CSV reader and the traffic writer: base units, one launch per
    capture, labels matching the benchmark's point labels."""
    from paper_2608_15764_gb300 import sweep, tune
    hdr = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
           '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"')

    def row(i, metric, unit, value):
        return (f'"{i}","1","python","h","void sl::k_ldg_dyn<4, 256, 0, 0>(sl::KArgs)","1","7","(256, 1, 1)",'
                f'"(912, 1, 1)","0","10.3","","{metric}","{unit}","{value}"')

    good = tmp_path / "good.csv"
    good.write_text("\n".join(["==PROF== Connected", hdr, row(0, "dram__bytes_read.sum", "byte", "1,073,770,000"),
                               row(0, "dram__bytes_write.sum", "byte", "2,964,736")]) + "\n")
    out = tmp_path / "traffic.json"
    doc = sweep.write_traffic([f"ldgdyn:4:256={good}"], str(out))
    e = doc["points"][tune.parse_point("ldgdyn:4:256").label()]
    assert e["dram_read"] == 1073770000 and e["dram_bytes_per_launch"] == 1073770000 + 2964736
    assert json.load(open(out))["kernel_source_hash"] == doc["kernel_source_hash"]
    scaled = tmp_path / "scaled.csv"
    scaled.write_text("\n".join([hdr, row(0, "dram__bytes_read.sum", "Gbyte", "1.07"),
                                 row(0, "dram__bytes_write.sum", "Mbyte", "2.9")]) + "\n")
    with pytest.raises(ValueError):
        sweep.write_traffic([f"ldgdyn:4:256={scaled}"], str(out))
    two = tmp_path / "two.csv"
    two.write_text("\n".join([hdr, row(0, "dram__bytes_read.sum", "byte", "1"), row(0, "dram__bytes_write.sum", "byte", "1"),
                              row(1, "dram__bytes_read.sum", "byte", "1"), row(1, "dram__bytes_write.sum", "byte", "1")]))
    with pytest.raises(ValueError):
        sweep.write_traffic([f"ldgdyn:4:256={two}"], str(out))


def test_alloc_counter_table_pairs_launches_with_cells(tmp_path):
    """The allocation sweep's single-pass counters: launch i of each capture is
    cell i (K = 2 and 8 per size, ascending); the derived L2 read hit rate is
    1 - DRAM read bytes / (32 x L1-to-L2 read sectors)."""
    from paper_2608_15764_gb300 import sweep
    hdr = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
           '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"')

    def row(i, metric, unit, value):
        return (f'"{i}","1","python","h","void sl::k_ldg<2, 256, 0, 0, 0>(sl::KArgs)","1","7","(256, 1, 1)",'
                f'"(608, 1, 1)","0","10.3","","{metric}","{unit}","{value}"')

    cells = [(g, k) for g in (0.5, 1) for k in (2, 8)]
    dram, l2 = [hdr], [hdr]
    for i, (g, k) in enumerate(cells):
        nbytes = int(g * (1 << 30))
        dram += [row(i, "dram__bytes_read.sum", "byte", nbytes - 32 * 10 * (i + 1)),
                 row(i, "dram__bytes_write.sum", "byte", 3000000)]
        l2 += [row(i, "lts__t_sectors_srcunit_tex_op_read.sum", "sector", nbytes // 32),
               row(i, "lts__t_sectors.sum", "sector", nbytes // 32 * 3 // 2)]
    (tmp_path / "d.csv").write_text("\n".join(dram) + "\n")
    (tmp_path / "l.csv").write_text("\n".join(l2) + "\n")
    rows = sweep.counter_table("ncu-alloc1", str(tmp_path / "d.csv"), str(tmp_path / "l.csv"), gib=1)
    assert [(r["gib"], r["k"]) for r in rows] == cells
    r = rows[3]
    assert r["bytes"] == 1 << 30 and r["dram_read"] == (1 << 30) - 1280
    assert r["l2_read_hit_derived"] == pytest.approx(1280 / (1 << 30), rel=1e-3)
    with pytest.raises(ValueError):  # a capture with a launch missing
        sweep.counter_table("ncu-alloc1", str(tmp_path / "d.csv"), str(tmp_path / "l.csv"), gib=2)
    with pytest.raises(ValueError):  # not a single-pass configuration
        sweep.counter_table("c1", str(tmp_path / "d.csv"), str(tmp_path / "l.csv"))
