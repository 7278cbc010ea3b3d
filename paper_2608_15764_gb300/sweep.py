"""Collection harness: the paper's sweeps on GB300, one JSONL row per cell.

Paper §3 "Fixed-work control": every K sweep runs ascending and reversed, with
total issued logical loads matched across K (here exactly bytes/16 per pass).
§3 "Hardware counters": the warm-up launch is excluded.  §3 "Timing,
residency, statistics": the unit is the launch, per-cell medians with
min-max, and a residency screen flags any HBM cell above the datasheet.

Configurations (buffers of uint32 words from splitmix64(seed=1), filled on the
GPU and checked against the first cell's checksum):

  c1   256 MiB; LDG K in {1,2,4,8}; 256 threads; grid 4 x SMs.
  c2   4 GiB; LDG K in {1,2,3,4,6,8,12,16} x CTA {128,256,512} x resident
       CTAs per SM r = 1..8 (grid = r x SMs; a cell is infeasible when the
       occupancy API allows fewer than r) x sweep order {asc, desc}.
  c3   4 GiB; same bytes through LDG K 1..16 (grid-stride tiles, and the
       dynamic contiguous-chunk traversal for K in {1,2,3,4,6,8,12,16}),
       cp.async D 1..8 and TMA stage {4,16,64} KiB x stages 2..8 in both ring
       layouts (one ring per CTA read by 256 consumer threads, and by 128 for
       4 KiB stages; the stages dealt to the warps, one per warp and, for even
       stage counts, two); cells over the shared-memory limit are recorded as
       infeasible.
  c4   allocations 512 MiB, 1, 2, 4, 8, 16, 20 GiB; LDG K in {1,2,4,8,16}.
  cpratio  paper §4.3: cp.async against the matched ld.global -> st.shared
       kernel at equal offered groups G in {1,2,4,8,12,16} (cp.async depth D =
       G; G loads staged through shared memory), at 1 and 8 warps per SM (one
       CTA per SM), on 1 GiB.
  cpgroups  cp.async with G in {1,2,4,8} 16-byte copies per commit group
       and D groups in flight (D*G <= 16): every cell at 256 threads on
       4 GiB, one warp (32 threads, one CTA) on 32 MiB, and the eleven
       dynamic-chunk instantiations at 256 threads on 4 GiB.
  ladder  paper §4.1: pointer-chase latency versus footprint, .ca / .cg.
  l2   the L2-targeted backend (paper §4.2 "L2-targeted control"): 16, 32
       and 64 MiB buffers (below the 129 MB L2) read 4 GiB / size passes per
       launch, LDG K in {1,2,3,4,6,8,12,16} at 256 threads x 4 x SMs and
       K in {1,2,4,8} at the primary shape; cells legitimately exceed the
       HBM datasheet.
  ilp  one CTA of one warp (32 threads) on a 32 MiB buffer: time versus K
       (LDG) and D (cp.async).  With all K loads in flight, a lone warp is
       latency-bound and its time falls about K-fold at fixed work.
  primary  the paper's primary cell shape (§4.2: one CTA of 32 warps per SM,
       .cg, 16-byte loads), K in {1,2,4,8}, on 4 GiB.
  ncu-point  one launch (no warm-up) of the point --point (tune.parse_point
       notation) on a --gib buffer (default 1 GiB): the small case of every
       counter capture, one kernel per ncu invocation.
  c2w  the residency grid of c2 at the other two load widths: 4-byte loads
       (K in {1,2,4,8,16}) and 32-byte loads (K in {1,2,3,4,6,8}); with c2
       it gives the paper's regime map over warps x width.
  cpskew  cp.async D in {1,2,4,8} and the matched LDG->STS kernel (G=4) at 256
       threads, and cp.async D=4 at 64/128/512/1024 threads, with the
       shared-memory ring 0, 16, 32 or 64 bytes past a 128-byte boundary
       (SL_DEBUG_SMEM_SKEW), 1 GiB: the destination alignment's effect.
  c2fixed  the residency grid (CTA 256/512 x 1-8 resident CTAs/SM x K) under
       the paper's fixed-iteration control: 4 GiB of loads wrapping over a
       2 GiB allocation; regime map as for c2.
  fixedit  the paper's own fixed-iteration control (§3, §4.2): the primary
       cell shape (1,024-thread CTAs, .cg, 16 B) issuing 16,785 MiB of loads
       that wrap around a 512 MiB, 2, 4, 8 or 20 GiB allocation, at 132 CTAs
       (the paper's H100) and one CTA per GB300 SM, K in {1,2,4,8}; reports
       the issued counts (mismatch across K) and GB/s of the issued bytes.
  ncu-fixed  one launch per cell of the fixed-iteration control at 132 CTAs,
       K = 2 and 8, on a 2 GiB allocation (two launches).
  ncu-alloc1  the allocation sweep's K = 2 and 8 endpoints at 512 MiB ...
       --gib GiB, one launch each, for single-pass counter captures (DRAM
       bytes; L1-to-L2 read sectors); --counter-table turns two such
       captures into the per-cell table.
  ncu-c2  the residency grid's K sweep (K <= 8) at 1,024 threads per SM (CTA
       128 x 8, 256 x 4, 512 x 2 and 1,024 x 1) on 4 GiB, one launch each, for
       the same single-pass captures.
  ncu-cpskew  cp.async D=4 at 256 threads with its shared-memory ring on a
       128-byte boundary and 16 bytes past one, 1 GiB (two launches).
  k1gate  paper §4.1's streaming-read qualification row: 4-byte plain loads
       (SL_LDG4) at K = 1 (the gate) and K up to 16, CTA 256 and 1024, on
       4 GiB, beside 16-byte LDG at K = 1, 2, 4.
  launches  paper §4.2 repeatability: the primary cell shape, K in {1,2,4,8},
       as --repeats independent launches (each a sweep over K); per-launch
       paired K=2 -> 8 change and the per-K spread across launches.
  two  paper §4.4: two co-resident plain-load streams in one CTA per SM,
       stream A = 1/2/4/8/16 warps, stream B = 0..16 warps, K = 1, 2, 4;
       displacement of A's bandwidth by B.
  ncu-primary  the primary cell shape (1,024 threads, one CTA per SM), K = 2
       and 8 (the paper's endpoints), 1 GiB, one launch each: the paper's
       counter audit (two launches).

Counter captures stay small: one kernel, one to three launches, at most a
few GiB on the device (every ncu-* configuration above).  Counters at larger
allocations are not captured; the kernels' own issued-load counts give the
bytes read at every size.

    python -m paper_2608_15764_gb300.sweep --config c2 --out runs.jsonl [--repeats 10]

A rerun with the same --out skips cells already recorded (resume after an
interrupted run).

    python -m paper_2608_15764_gb300.sweep --traffic SPEC=CSV [SPEC=CSV ...] --traffic-out FILE

writes the DRAM bytes per launch of each point (SPEC in tune.parse_point
notation) from `ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum
--print-units base --csv` logs of single-launch `ncu-point` captures, with
the kernel-source hash they were taken on; bench.py reads it for the
roofline's traffic.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys
import time

DATASHEET_GBS = 8000.0


def decline(bw_k2: float, bw_k8: float) -> float:
    """Endpoint change from K=2 to K=8 in percent (paper §4.2 tables: negative
    for a decline)."""
    return 100.0 * (bw_k8 - bw_k2) / bw_k2


def _cells(config: str, sms: int, point: str | None = None, gib: float = 1.0):
    """Yield (cell_key, cell dict) in ascending order."""
    if config == "c1":
        for k in (1, 2, 4, 8):
            yield dict(mech="ldg", k=k, cta=256, grid=4 * sms, gib=0.25)
    elif config == "c2":
        for cta in (128, 256, 512):
            for r in range(1, 9):
                for k in (1, 2, 3, 4, 6, 8, 12, 16):
                    yield dict(mech="ldg", k=k, cta=cta, grid=r * sms, resident_req=r, gib=4)
    elif config == "cpskew":
        # destination alignment of the shared-memory ring: 0 = 128-byte
        # aligned, n = n x 16 bytes past a 128-byte boundary
        for skew in (0, 1, 2, 4):
            for d in (1, 2, 4, 8):
                yield dict(mech="cpasync", k=d, cta=256, grid=0, skew=skew, gib=1)
            yield dict(mech="ldsts", k=4, cta=256, grid=0, skew=skew, gib=1)
            for cta in (64, 128, 512, 1024):
                yield dict(mech="cpasync", k=4, cta=cta, grid=0, skew=skew, gib=1)
    elif config == "c2fixed":
        # the residency grid under the paper's fixed-iteration control: 4 GiB
        # of 16-byte loads wrapping over a 2 GiB allocation
        target = (4 << 30) // 16
        for cta in (256, 512):
            for r in range(1, 9):
                for k in (1, 2, 3, 4, 6, 8, 12, 16):
                    yield dict(mech="ldg", k=k, cta=cta, grid=r * sms, resident_req=r, target_loads=target, gib=2)
    elif config == "fixedit":
        # paper §3 / §4.2: the primary cell under the paper's own fixed-iteration
        # control (16,785 MiB of 16-byte loads, wrapping over the allocation),
        # at the paper's 132 CTAs and at GB300's SM count
        target = 16785 * (1 << 20) // 16
        for gib in (0.5, 2, 4, 8, 20):
            for grid in (132, sms):
                for k in (1, 2, 4, 8):
                    yield dict(mech="ldg", k=k, cta=1024, grid=grid, target_loads=target, gib=gib)
    elif config == "ncu-fixed":
        # counters of the fixed-iteration control at K = 2 and 8, 132 CTAs, on
        # a 2 GiB allocation (two launches)
        target = 16785 * (1 << 20) // 16
        for k in (2, 8):
            yield dict(mech="ldg", k=k, cta=1024, grid=132, target_loads=target, gib=2)
    elif config == "c2w":
        for cta in (128, 256, 512):
            for r in range(1, 9):
                for k in (1, 2, 4, 8, 16):
                    yield dict(mech="ldg4", k=k, cta=cta, grid=r * sms, resident_req=r, gib=4)
                for k in (1, 2, 3, 4, 6, 8):
                    yield dict(mech="ldg32", k=k, cta=cta, grid=r * sms, resident_req=r, gib=4)
    elif config == "c3":
        for k in range(1, 17):
            yield dict(mech="ldg", k=k, cta=256, grid=0, gib=4)
        for k in (1, 2, 3, 4, 6, 8, 12, 16):
            yield dict(mech="ldg", k=k, cta=256, grid=0, trav=2, gib=4)
        for trav in (0, 2):
            for k in (1, 2, 3, 4, 6, 8):
                yield dict(mech="ldg32", k=k, cta=256, grid=0, trav=trav, gib=4)
        for d in range(1, 9):
            yield dict(mech="cpasync", k=d, cta=256, grid=0, gib=4)
        for sb in (4096, 16384, 65536):
            for n in range(2, 9):
                yield dict(mech="tma", stage_bytes=sb, stages=n, cta=256, grid=0, gib=4)
        for n in range(2, 9):  # 4 KiB stages read by 128 consumer threads (two vectors per lane)
            yield dict(mech="tma", stage_bytes=4096, stages=n, cta=128, grid=0, gib=4)
        for sb in (4096, 16384, 65536):
            for n in range(2, 9):
                for cta in ([32 * n, 16 * n] if n % 2 == 0 else [32 * n]):
                    yield dict(mech="tma", stage_bytes=sb, stages=n, cta=cta, ring="warp", grid=0, gib=4)
    elif config == "c4":
        for gib in ALLOC_GIB:
            for k in (1, 2, 4, 8, 16):
                yield dict(mech="ldg", k=k, cta=256, grid=4 * sms, gib=gib)
    elif config == "ilp":
        for k in (1, 2, 4, 8, 16):
            yield dict(mech="ldg", k=k, cta=32, grid=1, gib=1 / 32)
        for d in (1, 2, 4, 8):
            yield dict(mech="cpasync", k=d, cta=32, grid=1, gib=1 / 32)
    elif config == "cpgroups":
        # cp.async with G copies per commit group and D groups in flight: the
        # whole grid at 4 GiB (D*G*16 bytes in flight per thread), and a lone
        # warp, whose time shows the offered concurrency directly
        for g in (1, 2, 4, 8):
            for d in range(1, 16 // g + 1):
                yield dict(mech="cpasync", k=d, copies=g, cta=256, grid=0, gib=4)
        for g in (1, 2, 4, 8):
            for d in (1, 2, 4, 8, 16):
                if d * g <= 16:
                    yield dict(mech="cpasync", k=d, copies=g, cta=32, grid=1, gib=1 / 32)
        # the dynamic-chunk traversal's instantiations at 256 threads
        for d, g in ((1, 1), (2, 1), (3, 1), (4, 1), (6, 1), (8, 1), (2, 2), (1, 4), (2, 4), (1, 8), (2, 8)):
            yield dict(mech="cpasync", k=d, copies=g, cta=256, grid=0, trav=2, gib=4)
    elif config == "primary":
        for k in (1, 2, 4, 8):
            yield dict(mech="ldg", k=k, cta=1024, grid=sms, gib=4)
    elif config == "cpratio":
        for warps in (1, 8):
            for g in (1, 2, 4, 8, 12, 16):
                for mech in ("cpasync", "ldsts"):
                    yield dict(mech=mech, k=g, cta=32 * warps, grid=sms, gib=1, warps_per_sm=warps)
    elif config == "l2":
        for mib in (16, 32, 64):
            passes = (4 << 30) // (mib << 20)  # 4 GiB issued at every size
            for k in (1, 2, 3, 4, 6, 8, 12, 16):
                yield dict(mech="ldg", k=k, cta=256, grid=4 * sms, gib=mib / 1024, passes=passes)
            for k in (1, 2, 4, 8):
                yield dict(mech="ldg", k=k, cta=1024, grid=sms, gib=mib / 1024, passes=passes)
    elif config == "k1gate":
        for cta in (256, 1024):
            for k in (1, 2, 4, 8, 16):
                yield dict(mech="ldg4", k=k, cta=cta, grid=0, gib=4)
            for k in (1, 2, 4):
                yield dict(mech="ldg", k=k, cta=cta, grid=0, gib=4)
    elif config == "ncu-point":
        # one launch of one point: the small case of a counter capture
        from .tune import MECH_NAMES, parse_point
        if not point:
            raise ValueError("ncu-point needs --point")
        p = parse_point(point)
        if p.mech == 2:
            yield dict(mech="tma", stage_bytes=p.stage_bytes, stages=p.stages, cta=p.cta, grid=0, gib=gib,
                       ring="warp" if p.ring else "cta")
        else:
            cell = dict(mech=MECH_NAMES[p.mech], k=p.k, cta=p.cta, grid=0, cop=p.cop, trav=p.order, gib=gib)
            if p.copies != 1:
                cell["copies"] = p.copies
            yield cell
    elif config == "ncu-alloc1":
        # the allocation sweep's K = 2 and 8 endpoints, one launch each, at the
        # sizes up to --gib; captured only with metric sets that ncu collects
        # in a single pass (no device-memory save and restore between
        # passes), the only kind taken on full-size buffers
        for g in ALLOC_GIB:
            if g <= gib:
                for k in (2, 8):
                    yield dict(mech="ldg", k=k, cta=256, grid=4 * sms, gib=g)
    elif config == "ncu-c2":
        # the residency grid's K sweep at 1,024 threads per SM (CTA 128 x 8,
        # 256 x 4, 512 x 2 resident CTAs, and the paper's primary 1,024 x 1) on
        # 4 GiB, one launch per cell: for single-pass counter captures, as
        # ncu-alloc1
        # (K = 12 and 16 need more than 64 registers per thread, so they never
        # run at 1,024 threads per SM)
        for cta, r in ((128, 8), (256, 4), (512, 2), (1024, 1)):
            for k in (1, 2, 3, 4, 6, 8):
                yield dict(mech="ldg", k=k, cta=cta, grid=r * sms, resident_req=r, gib=4)
    elif config == "ncu-cpskew":
        for skew in (0, 1):
            yield dict(mech="cpasync", k=4, cta=256, grid=0, skew=skew, gib=1)
    elif config == "ncu-primary":
        # the paper's primary cell shape (one 1,024-thread CTA per SM) on 1 GiB:
        # its counter audit (§4.2) at the endpoints K = 2 and 8
        for k in (2, 8):
            yield dict(mech="ldg", k=k, cta=1024, grid=sms, gib=1)
    else:
        raise ValueError(config)


ALLOC_GIB = (0.5, 1, 2, 4, 8, 16, 20)


def counter_table(config: str, dram_csv: str, l2_csv: str, gib: float = 20.0) -> list[dict]:
    """Rows of a single-pass counter configuration (ncu-alloc1, ncu-c2) run
    twice under ncu, once for dram__bytes_read.sum / dram__bytes_write.sum and
    once for lts__t_sectors_srcunit_tex_op_read.sum / lts__t_sectors.sum (each
    set takes one pass; together they take more).  Launch i of a capture is
    cell i of the configuration (cells that are infeasible on the device
    launch nothing: capture on a GPU where every cell runs).  The L2 hit rate
    of the kernel's reads is derived as 1 - DRAM read bytes / (32 x L1-to-L2
    read sectors): the share of requested sectors that needed no DRAM read
    (the per-request hit and miss counters take three passes)."""
    if config not in ("ncu-alloc1", "ncu-c2"):
        raise ValueError(f"{config} is not a single-pass counter configuration")
    cells = [c for c in _cells(config, 1, gib=gib)]
    per = {}
    for path in (dram_csv, l2_csv):
        for r in read_ncu_csv(path):
            if r["unit"] not in ("byte", "sector", ""):
                raise ValueError(f"{path}: {r['metric']} in {r['unit']}; capture with --print-units base")
            per.setdefault(path, {}).setdefault(r["id"], {})[r["metric"]] = r["value"]
    ids = {path: sorted(v) for path, v in per.items()}
    for path in (dram_csv, l2_csv):
        if len(ids.get(path, [])) != len(cells):
            raise ValueError(f"{path}: {len(ids.get(path, []))} launches for {len(cells)} cells")
    rows = []
    for i, c in enumerate(cells):
        d = per[dram_csv][ids[dram_csv][i]]
        l2 = per[l2_csv][ids[l2_csv][i]]
        nbytes = int(c["gib"] * (1 << 30)) // 16 * 16
        req = 32.0 * l2["lts__t_sectors_srcunit_tex_op_read.sum"]
        rows.append({"gib": c["gib"], "k": c["k"], "cta": c["cta"], "resident": c.get("resident_req"), "bytes": nbytes,
                     "dram_read": d["dram__bytes_read.sum"], "dram_write": d["dram__bytes_write.sum"],
                     "dram_read_over_bytes": round(d["dram__bytes_read.sum"] / nbytes, 7),
                     "l1_l2_read_sectors": l2["lts__t_sectors_srcunit_tex_op_read.sum"],
                     "l2_sectors": l2["lts__t_sectors.sum"],
                     "l2_read_hit_derived": float(f"{1.0 - d['dram__bytes_read.sum'] / req:.4g}") if req else None})
    return rows


def _expected_loads(mech: str, nbytes: int, passes: int) -> int:
    """Loads a launch issues under exact fixed work: 16-byte loads, 4-byte
    loads (ldg4), or 32-byte loads plus one 16-byte load for a final half
    unit (ldg32)."""
    if mech == "ldg4":
        return passes * (nbytes // 4)
    if mech == "ldg32":
        return passes * ((nbytes + 31) // 32)
    return passes * (nbytes // 16)


def _key(cell: dict, order: str) -> str:
    return json.dumps({**cell, "order": order}, sort_keys=True)


def run(config: str, out: str | None, repeats: int = 10, orders=("asc", "desc"), verbose: bool = True,
        warmup: int = 1, point: str | None = None, gib: float = 1.0, dtype: str = "u32"):
    import torch

    import paper_2608_15764_gb300 as sl

    sl.load()
    info = sl.sl_device_info()
    sms = info["sm_count"]
    dt = sl.DTYPES[dtype]
    done = set()
    if out and os.path.exists(out):
        for line in open(out):
            try:
                row = json.loads(line)
            except ValueError:
                continue
            if row.get("config") == config and "key" in row:
                done.add(row["key"])
    cells = list(_cells(config, sms, point=point, gib=gib))
    rows = []
    by_size = {}
    for c in cells:
        by_size.setdefault(c["gib"], []).append(c)
    for gib, group in by_size.items():
        nbytes = int(gib * (1 << 30)) // 16 * 16
        buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        sl.sl_fill_splitmix64(buf, seed=1)
        torch.cuda.synchronize()
        ref = None
        for order in orders:
            todo = [c for c in group if _key(c, order) not in done]
            if not todo:
                continue
            seq = todo if order == "asc" else list(reversed(todo))
            cfgs, keep = [], []
            for c in seq:
                passes = c.get("passes", 1)
                kw = dict(cta=c["cta"], grid=c["grid"], passes=passes, target_loads=c.get("target_loads", 0),
                          debug_flags=sl.SL_DEBUG_SMEM_SKEW(c.get("skew", 0)))
                if c["mech"] == "tma":
                    cfg = sl.config("tma", stage_bytes=c["stage_bytes"], stages=c["stages"], ring=c.get("ring", "cta"),
                                    **kw)
                else:
                    cfg = sl.config(c["mech"], k=c["k"], cop=c.get("cop", 0), order=c.get("trav", 0),
                                    copies=c.get("copies", 1), **kw)
                status, resident = 0, 0
                try:
                    plan = sl.sl_plan(nbytes, dt, cfg)
                    resident = plan.resident_per_sm
                    if c.get("resident_req") and resident < c["resident_req"]:
                        status = sl.SL_ERR_INFEASIBLE
                except sl.SLError as e:
                    status = e.status
                row = {"config": config, "key": _key(c, order), "order": order, "bytes": nbytes, **c,
                       "status": status, "resident_per_sm": resident}
                if status:
                    rows.append(row)
                    _emit(out, row, verbose)
                    continue
                cfgs.append(cfg)
                keep.append(row)
            if not cfgs:
                continue
            # one sweep call per order: the cells run back to back in `seq` order
            res = sl.sl_sweep(buf, cfgs, dtype=dt, repeats=repeats, warmup=warmup, sweep_order="asc")
            for row, rr in zip(keep, res):
                ok = [r for r in rr if r.status == 0]
                fixed = row.get("target_loads", 0) > 0
                if fixed:  # the paper's fixed-iteration control: bytes = 16 x loads issued
                    tk = row["grid"] * row["cta"] * row["k"]
                    want_loads = row["target_loads"] // tk * tk
                    vol = 16 * want_loads
                else:
                    want_loads = _expected_loads(row["mech"], nbytes, row.get("passes", 1))
                    vol = nbytes * row.get("passes", 1)  # bytes issued per launch
                gbs = [vol / r.device_ns for r in ok if r.device_ns]
                wgbs = [vol / r.window_ns for r in ok if r.window_ns]
                cks = {(r.sum_u32, r.xor_u64) for r in ok}
                if ref is None and cks and not fixed:
                    ref = next(iter(cks))
                row.update(
                    status=0 if len(ok) == len(rr) else rr[0].status,
                    grid_used=rr[0].grid,
                    gbs_median=round(statistics.median(gbs), 2) if gbs else None,
                    gbs_min=round(min(gbs), 2) if gbs else None,
                    gbs_max=round(max(gbs), 2) if gbs else None,
                    gbs=[round(v, 2) for v in gbs],
                    window_gbs_median=round(statistics.median(wgbs), 2) if wgbs else None,
                    issued=ok[0].issued_loads if ok else None,
                    issued_ok=all(r.issued_loads == want_loads for r in ok),
                    checksum_ok=(len(cks) == 1) if fixed else (cks == {ref}),
                    above_datasheet=bool(gbs and max(gbs) > DATASHEET_GBS),
                    frac_of_datasheet=round(statistics.median(gbs) / DATASHEET_GBS, 4) if gbs else None,
                )
                rows.append(row)
                _emit(out, row, verbose)
        del buf
        torch.cuda.empty_cache()
    return rows


def _emit(out, row, verbose):
    if out:
        with open(out, "a") as f:
            f.write(json.dumps(row) + "\n")
    if verbose:
        c = {k: row.get(k) for k in ("mech", "k", "stage_bytes", "stages", "cta", "grid", "gib", "order")}
        print(json.dumps({**{k: v for k, v in c.items() if v is not None}, "status": row["status"],
                          "gbs": row.get("gbs_median"), "res": row.get("resident_per_sm")}), flush=True)


LADDER_FOOTPRINTS = [1 << e for e in range(13, 31)] + [24 << 20, 48 << 20, 96 << 20, 192 << 20]


def run_ladder(out: str | None, verbose: bool = True):
    """Paper §4.1 latency ladder: unloaded pointer-chase latency on one SM
    versus footprint (8 KiB .. 1 GiB, one element per 64 bytes, one random
    cycle through every element), .ca and .cg.  Before each chase the L2 is
    flushed; chains of up to 4 Mi elements (256 MiB) are first walked once in
    full (untimed), so the timed steps revisit lines that the footprint lets
    the caches keep; longer chains are not warmed.  32,768 steps are timed.
    The .ca and .cg walks of a chain must end on the same index (the chase
    itself is checked against the oracle by the test suite)."""
    import numpy as np
    import torch

    import paper_2608_15764_gb300 as sl
    from . import workloads as wl

    sl.load()
    rows = []
    for fp in sorted(LADDER_FOOTPRINTS):
        n = fp // 64
        host = wl.chase_chain(n, 64)
        dev = torch.from_numpy(host.view(np.uint8)).cuda()
        warm, hops = (n if n <= (1 << 22) else 0), 1 << 15
        finals = set()
        for ca in (True, False):
            sl.sl_flush_l2()
            torch.cuda.synchronize()
            r = sl.sl_chase(dev, warm=warm, hops=hops, cache_l1=ca)
            finals.add(r.final_index)
            row = {"config": "ladder", "footprint": fp, "cop": "ca" if ca else "cg", "ns_per_hop": round(r.ns_per_hop, 2),
                   "cycles_per_hop": round(r.cycles_per_hop, 1), "final_index": r.final_index,
                   "ca_cg_agree": len(finals) == 1}
            rows.append(row)
            if out:
                with open(out, "a") as f:
                    f.write(json.dumps(row) + "\n")
            if verbose:
                print(json.dumps(row), flush=True)
        del dev
    return rows


def run_launches(out: str | None, launches: int = 10, gib: float = 4.0, verbose: bool = True):
    """Paper §4.2 "Repeatability": the primary cell shape (one 1,024-thread
    CTA per SM, .cg, 16-byte loads) on a 4 GiB buffer, run as `launches`
    independent launches, each a sweep over K = 1, 2, 4, 8 (one timed run per
    K after one warm-up run).  Per launch: GB/s per K and the paired K=2 -> 8
    change; overall: the per-K spread across launches and the range of the
    paired changes."""
    import torch

    import paper_2608_15764_gb300 as sl

    sl.load()
    sms = sl.sl_device_info()["sm_count"]
    nbytes = int(gib * (1 << 30)) // 16 * 16
    buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    sl.sl_fill_splitmix64(buf, seed=1)
    ks = (1, 2, 4, 8)
    cfgs = [sl.config("ldg", k=k, cta=1024, grid=sms) for k in ks]
    per = []
    cks = set()
    for li in range(launches):
        res = sl.sl_sweep(buf, cfgs, dtype=sl.SL_U32, repeats=1, warmup=1)
        gbs = {k: nbytes / row[0].device_ns for k, row in zip(ks, res)}
        cks |= {(row[0].sum_u32, row[0].xor_u64, row[0].issued_loads) for row in res}
        row = {"config": "launches", "launch": li, "gbs": {str(k): round(v, 2) for k, v in gbs.items()},
               "paired_change_pct": round(decline(gbs[2], gbs[8]), 3)}
        per.append(row)
        if out:
            with open(out, "a") as f:
                f.write(json.dumps(row) + "\n")
        if verbose:
            print(json.dumps(row), flush=True)
    spread = {}
    for k in ks:
        v = [r["gbs"][str(k)] for r in per]
        med = statistics.median(v)
        spread[str(k)] = {"median": round(med, 2), "spread_pct": round(100.0 * (max(v) - min(v)) / med, 3)}
    changes = [r["paired_change_pct"] for r in per]
    summary = {"config": "launches", "launches": launches, "per_k": spread,
               "paired_change_pct": {"min": min(changes), "median": statistics.median(changes), "max": max(changes)},
               "checksums_consistent": len(cks) == 1}
    if out:
        with open(out, "a") as f:
            f.write(json.dumps(summary) + "\n")
    if verbose:
        print(json.dumps(summary), flush=True)
    return per, summary


TWO_WARPS = (1, 2, 4, 8, 16)
TWO_B_WARPS = (0, 1, 2, 4, 8, 16)


def run_two(out: str | None, repeats: int = 3, ks=(1, 2, 4), a_gib: float = 1.0, b_gib: float = 2.0,
            verbose: bool = True):
    """Paper §4.4: two co-resident plain-load streams in one CTA per SM.
    Stream A (A warps) reads a 1 GiB buffer once; stream B (B warps) re-reads
    a 2 GiB buffer for as many passes as it takes to keep loading until A's
    last warp is done (start from the pass count of the previous B width,
    double until sl_twostream reports b_covers_a).  A's bandwidth = bytes / A's
    %globaltimer window (median of `repeats`); displacement = 1 - A(B) / A(0).
    Checksums: A's must agree across every cell, B's must follow the
    closed form of its pass count from a single-pass read of B's buffer."""
    import torch

    import paper_2608_15764_gb300 as sl

    sl.load()
    nb_a = int(a_gib * (1 << 30)) // 16 * 16
    nb_b = int(b_gib * (1 << 30)) // 16 * 16
    a = torch.empty(nb_a, dtype=torch.uint8, device="cuda")
    b = torch.empty(nb_b, dtype=torch.uint8, device="cuda")
    sl.sl_fill_splitmix64(a, seed=21)
    sl.sl_fill_splitmix64(b, seed=22)
    r1 = sl.sl_run(b, dtype=sl.SL_U32, cfg=sl.config("ldg", k=4))
    sb, xb = r1.sum_u32, r1.xor_u64
    ref_a = None
    rows = []
    for k in ks:
        for wa in TWO_WARPS:
            solo_gbs, prev_passes = None, 1
            for wb in TWO_B_WARPS:
                if wa + wb > 32:
                    continue
                passes, pmax = 1, 1
                if wb:
                    tiles_b = -(-(nb_b // 16) // (32 * wb * k))
                    pmax = ((1 << 32) - 4096) // tiles_b  # the kernel counts tiles in 32 bits
                    passes = min(pmax, prev_passes)
                gbs, bgbs, cover, ck_ok = [], [], True, True
                for _ in range(repeats):
                    for _try in range(6):
                        r = sl.sl_twostream(a, b if wb else None, warps_a=wa, warps_b=wb, k=k, passes_b=passes)
                        if r.b_covers_a or passes >= pmax:
                            break
                        passes = min(pmax, 2 * passes)
                    cover = cover and bool(r.b_covers_a)
                    ca = (r.sum_u32[0], r.xor_u64[0])
                    ref_a = ref_a or ca
                    ck_ok = ck_ok and ca == ref_a and r.issued_loads[0] == nb_a // 16
                    if wb:
                        ck_ok = ck_ok and (r.sum_u32[1], r.xor_u64[1]) == ((passes * sb) % (1 << 32),
                                                                             xb if passes % 2 else 0)
                        bgbs.append(passes * nb_b / r.window_ns[1])
                    gbs.append(nb_a / r.window_ns[0])
                med = statistics.median(gbs)
                if wb == 0:
                    solo_gbs = med
                prev_passes = passes
                row = {"config": "two", "k": k, "warps_a": wa, "warps_b": wb, "a_gbs": round(med, 2),
                       "a_gbs_all": [round(v, 2) for v in gbs],
                       "displacement_pct": round(100.0 * (1.0 - med / solo_gbs), 2),
                       "b_gbs": round(statistics.median(bgbs), 2) if bgbs else None, "passes_b": passes,
                       "b_covers_a": cover, "checksum_ok": ck_ok}
                rows.append(row)
                if out:
                    with open(out, "a") as f:
                        f.write(json.dumps(row) + "\n")
                if verbose:
                    print(json.dumps(row), flush=True)
    return rows


def regime(values, frac: float = 0.95, tail: int = 3) -> str:
    """Class of a response curve (values in ascending offered load), by the
    paper's 95%-plateau rule with a three-cell tail (§3, §4.2 "Prevalence";
    read as: saturating if every tail cell is within 95% of the maximum;
    peak-decline if the maximum lies before the tail and the last cell is below
    95% of it; rising-censored otherwise)."""
    v = list(values)
    if len(v) < tail + 1:
        raise ValueError("curve too short")
    top = max(v)
    if all(x >= frac * top for x in v[-tail:]):
        return "saturating"
    if v.index(top) < len(v) - tail and v[-1] < frac * top:
        return "peak-decline"
    return "rising-censored"


WIDTH_BYTES = {"ldg": 16, "ldg4": 4, "ldg32": 32}


def regime_map(rows):
    """Regime of every plain-load K curve of the residency grid (configs c2
    and c2w): one curve per (load width in bytes, CTA, resident CTAs per SM,
    order) over the K values present."""
    curves = {}
    for r in rows:
        if r.get("config") not in ("c2", "c2w", "c2fixed") or r.get("status") or r.get("gbs_median") is None:
            continue
        key = (WIDTH_BYTES[r.get("mech", "ldg")], r["cta"], r["resident_req"], r["order"])
        if r.get("config") == "c2fixed":
            key = ("fixed",) + key
        curves.setdefault(key, {})[r["k"]] = r["gbs_median"]
    out = {}
    for key, byk in sorted(curves.items()):
        ks = sorted(byk)
        if len(ks) >= 4:
            out[key] = regime([byk[k] for k in ks])
    return out


def cp_ratio(rows):
    """cp.async / matched-plain-load bandwidth ratio per (warps per SM, G,
    order) -- the quantity of paper §4.3."""
    by = {}
    for r in rows:
        if r.get("config") != "cpratio" or r.get("status") or r.get("gbs_median") is None:
            continue
        by.setdefault((r["warps_per_sm"], r["k"], r["order"]), {})[r["mech"]] = r["gbs_median"]
    return [{"warps_per_sm": w, "groups": g, "order": o, "cpasync_gbs": d["cpasync"], "ldsts_gbs": d["ldsts"],
             "ratio": round(d["cpasync"] / d["ldsts"], 3)}
            for (w, g, o), d in sorted(by.items()) if "cpasync" in d and "ldsts" in d]


def fixed_mismatch(rows):
    """Paper §4.2 "Exact-work accounting" under the fixed-iteration control:
    per (allocation, grid, order) the issued loads at each K (from the
    launches' own counters) and the largest relative mismatch across K."""
    groups = {}
    for r in rows:
        if r.get("target_loads") and not r.get("status") and r.get("issued") is not None:
            groups.setdefault((r["gib"], r["grid"], r["order"]), {})[r["k"]] = r["issued"]
    out = []
    for (gib, grid, order), byk in sorted(groups.items()):
        hi, lo = max(byk.values()), min(byk.values())
        out.append({"gib": gib, "grid": grid, "order": order, "issued": {str(k): v for k, v in sorted(byk.items())},
                    "max_mismatch_pct": round(100.0 * (hi - lo) / hi, 6) if hi else 0.0})
    return out


def summarize(rows):
    """K=2 -> K=8 endpoint change per (config group, order) where both exist."""
    out = []
    groups = {}
    for r in rows:
        if r.get("mech") != "ldg" or r.get("status") or r.get("gbs_median") is None:
            continue
        g = (r["config"], r["gib"], r["cta"], r["grid"], r["order"])
        groups.setdefault(g, {})[r["k"]] = r["gbs_median"]
    for g, byk in sorted(groups.items()):
        if 2 in byk and 8 in byk:
            out.append({"config": g[0], "gib": g[1], "cta": g[2], "grid": g[3], "order": g[4],
                        "k2": byk[2], "k8": byk[8], "change_pct": round(decline(byk[2], byk[8]), 2)})
    return out


def read_ncu_csv(path: str) -> list[dict]:
    """Rows of an `ncu --csv --log-file` metrics log: one dict per (launch,
    metric) with the kernel name, metric name, unit and value (thousands
    separators removed)."""
    import csv
    with open(path) as f:
        lines = f.read().splitlines()
    start = next(i for i, l in enumerate(lines) if l.startswith('"ID"'))
    rows = []
    for r in csv.DictReader(lines[start:]):
        v = r.get("Metric Value", "").replace(",", "")
        try:
            val = float(v)
        except ValueError:
            continue
        rows.append({"id": int(r["ID"]), "kernel": r["Kernel Name"], "metric": r["Metric Name"],
                     "unit": r.get("Metric Unit", ""), "value": val})
    return rows


def write_traffic(pairs: list[str], out: str, gib: float = 1.0) -> dict:
    """profiles/traffic.json from single-launch captures: pairs 'SPEC=CSV'."""
    from .build import kernel_source_hash
    from .tune import parse_point
    points = {}
    for pair in pairs:
        spec, path = pair.split("=", 1)
        rows = read_ncu_csv(path)
        ids = sorted({r["id"] for r in rows})
        if len(ids) != 1:
            raise ValueError(f"{path}: expected one captured launch, found {len(ids)}")
        m = {r["metric"]: r for r in rows}
        for name in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            if m[name]["unit"] not in ("byte", "bytes", "B"):
                raise ValueError(f"{path}: {name} in {m[name]['unit']!r}; capture with --print-units base")
        rd, wr = m["dram__bytes_read.sum"]["value"], m["dram__bytes_write.sum"]["value"]
        points[parse_point(spec).label()] = {
            "spec": spec, "kernel": m["dram__bytes_read.sum"]["kernel"], "bytes": int(gib * (1 << 30)),
            "dram_read": int(rd), "dram_write": int(wr), "dram_bytes_per_launch": int(rd + wr)}
    doc = {"kernel_source_hash": kernel_source_hash(),
           "command": f"for each point: python -m paper_2608_15764_gb300.sweep --config ncu-point --point SPEC "
                      f"--gib {gib:g} --repeats 1 > plain.log && ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum "
                      "--print-units base --clock-control none -k regex:\"k_(ldg|tma|cpasync)\" -c 1 --csv "
                      "--log-file SPEC.csv python -m paper_2608_15764_gb300.sweep --config ncu-point --point SPEC "
                      f"--gib {gib:g} --repeats 1 (single-pass metrics)",
           "note": f"DRAM bytes per launch on a {gib:g} GiB buffer, one captured launch per point; bench.py scales "
                   "them to its buffer by bytes read (a factor of 1 when the sizes match)",
           "points": points}
    with open(out, "w") as f:
        json.dump(doc, f, indent=1)
    return doc


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--traffic", nargs="+", default=None, metavar="SPEC=CSV",
                    help="write --traffic-out from single-launch ncu-point captures instead of running a sweep")
    ap.add_argument("--traffic-out", default=os.path.join("profiles", "traffic.json"))
    ap.add_argument("--counter-table", nargs=2, default=None, metavar=("DRAM_CSV", "L2_CSV"),
                    help="print the per-cell table of two single-pass captures of --config (ncu-alloc1 with "
                         "sizes up to --gib, or ncu-c2) instead of running a sweep")
    ap.add_argument("--counter-out", default=None,
                    help="with --counter-table: also write the table with the kernel code hash as JSON "
                         "(profiles/alloc_counters.json is read by bench.py's allocation sweep)")
    ap.add_argument("--config", required=False,
                    choices=["c1", "c2", "c2w", "c2fixed", "fixedit", "cpskew", "cpgroups", "c3", "c4", "ilp", "primary",
                             "ncu-point", "ncu-primary", "ncu-fixed", "ncu-cpskew", "ncu-alloc1", "ncu-c2", "l2", "cpratio",
                             "ladder",
                             "k1gate", "two",
                             "launches"])
    ap.add_argument("--out", default=None)
    ap.add_argument("--repeats", type=int, default=10)
    ap.add_argument("--orders", default="asc,desc")
    ap.add_argument("--point", default=None, help="ncu-point: the point, e.g. ldgdyn:2:512 or tmaw:4096:8:256")
    ap.add_argument("--gib", type=float, default=1.0, help="ncu-point: buffer size in GiB")
    ap.add_argument("--dtype", default="u32", choices=["u32", "f32", "bf16", "fp8"],
                    help="fold of every cell (the buffer holds splitmix64 bits whatever the dtype: for float "
                         "dtypes only timing and counters mean anything, the float sums do not)")
    a = ap.parse_args(argv)
    if a.counter_table:
        rows = counter_table(a.config, a.counter_table[0], a.counter_table[1], gib=a.gib)
        for row in rows:
            print(json.dumps(row), flush=True)
        if a.counter_out:
            from .build import kernel_source_hash
            doc = {"kernel_source_hash": kernel_source_hash(), "config": a.config, "gib": a.gib,
                   "command": f"python -m paper_2608_15764_gb300.sweep --repeats 1 --config {a.config} --gib {a.gib:g} "
                              "under ncu twice: --metrics dram__bytes_read.sum,dram__bytes_write.sum and --metrics "
                              "lts__t_sectors_srcunit_tex_op_read.sum,lts__t_sectors.sum (--print-units base "
                              "--clock-control none -k regex:k_ldg --csv), both single-pass",
                   "rows": rows}
            with open(a.counter_out, "w") as f:
                json.dump(doc, f, indent=1)
        return 0
    if a.traffic:
        doc = write_traffic(a.traffic, a.traffic_out, gib=a.gib)
        print(json.dumps({"traffic_points": len(doc["points"]), "out": a.traffic_out}), flush=True)
        return 0
    if not a.config:
        ap.error("--config is required")
    t0 = time.time()
    if a.config == "launches":
        run_launches(a.out, launches=a.repeats)
        print(json.dumps({"config": a.config, "seconds": round(time.time() - t0, 1)}), flush=True)
        return 0
    if a.config == "two":
        rows = run_two(a.out, repeats=min(a.repeats, 5))
        print(json.dumps({"config": a.config, "cells": len(rows), "seconds": round(time.time() - t0, 1)}), flush=True)
        return 0
    if a.config == "ladder":
        rows = run_ladder(a.out)
        print(json.dumps({"config": a.config, "cells": len(rows), "seconds": round(time.time() - t0, 1)}), flush=True)
        return 0
    ncu = a.config.startswith("ncu")
    orders = ("asc",) if ncu else tuple(a.orders.split(","))
    rows = run(a.config, a.out, repeats=a.repeats, orders=orders, warmup=0 if ncu else 1, point=a.point, gib=a.gib,
               dtype=a.dtype)
    for s in summarize(rows):
        print(json.dumps({"summary": s}), flush=True)
    for s in cp_ratio(rows):
        print(json.dumps({"cp_ratio": s}), flush=True)
    if a.config == "fixedit":
        for s in fixed_mismatch(rows):
            print(json.dumps({"fixed_iteration": s}), flush=True)
    if a.config in ("c2", "c2w", "c2fixed"):
        rm = regime_map(rows)
        counts = {c: sum(1 for v in rm.values() if v == c) for c in ("saturating", "peak-decline", "rising-censored")}
        print(json.dumps({"regime_counts": counts, "curves": len(rm)}), flush=True)
    print(json.dumps({"config": a.config, "cells": len(rows), "seconds": round(time.time() - t0, 1)}), flush=True)


if __name__ == "__main__":
    sys.exit(main())
