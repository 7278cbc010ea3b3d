#!/usr/bin/env python3
"""Benchmark of the streaming global-load path on GB300.

Workload: a 4 GiB buffer of uint32 words from splitmix64(seed=1) (larger than
the 129 MB L2, so no flush is needed between steps).  Before timing, the
K-response curves of the mechanisms (LDG K at 16 and 32 bytes, grid-stride and
dynamic chunks; cp.async D; TMA stage x stages) are measured on the same
buffer as single launches, then every point's throughput over 16 back-to-back
passes, and the fastest point for back-to-back passes is chosen
(tune.choose(steps=True)).  One step = one checksum pass over the whole
buffer with that point: one load kernel, whose last CTA to finish combines
the per-CTA partials into the result.  Passes of grid-stride points run as
programmatic dependent launches (``sl_enqueue_steps``: a pass starts loading
while the previous pass's tail runs); other points use one ``sl_enqueue`` per
pass.

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

Prints one JSON line (rank 0).  N > 1 (torchrun): every rank streams its own
4 GiB buffer on its own GPU (weak scaling, no data-path collective); the
barrier and the max over ranks of the timed interval use torch.distributed.

``--impl reference`` times the CPU oracle (``oracle/``) on the host cores over
the same workload instead; it is the deliberately slow baseline arm.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "attained HBM GB/s vs offered ILP K per mechanism (LDG/cp.async/TMA); % of peak"
WORKLOAD = "4 GiB uint32 splitmix64(seed=1) buffer, single-pass streaming checksum (u32 sum + u64 xor)"
DATASHEET_GBS = 8000.0
FALLBACK_HBM_GBS = 6800.0


def _args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--gib", type=float, default=4.0, help="buffer size in GiB (default 4)")
    ap.add_argument("--curve-repeats", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=1.5,
                    help="wall-clock seconds of the CPU-oracle sample (all cores)")
    ap.add_argument("--out", default=None, help="also append the JSON line (and curves) to this file")
    ap.add_argument("--workload", choices=["stream", "batch", "prec"], default="stream",
                    help="stream: the 4 GiB K-response workload (default); batch: the 1,024-buffer batched form; "
                         "prec: the precision form (float payloads through every mechanism)")
    ap.add_argument("--prec-gib", type=float, default=1.0, help="prec workload payload size per dtype")
    ap.add_argument("--dtypes", default="f32,bf16,fp8", help="batch workload payload dtypes")
    ap.add_argument("--batch-gib", type=float, default=16.0, help="batch workload total per dtype")
    ap.add_argument("--choice", default=None,
                    help="skip the curves and time this point, e.g. 'ldg:6:256:0' (mech:K:cta:cop), "
                         "'cpasync:5:256' or 'tma:16384:2:256' (tma:stage_bytes:stages:cta)")
    return ap.parse_args(argv)


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi SM clocks / throttle reasons sampled every 200 ms."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for name, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_hash() -> str:
    """Hash of the kernel sources: DRAM-traffic counters taken on another
    version of the kernels are not reported."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2608_15764_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(csrc)):
        if name.startswith("k_") or name.endswith(".cuh") or name == "sl_internal.h":
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def _traffic(label: str, nbytes: int):
    """DRAM bytes per launch of the timed kernel from profiles/traffic.json
    (captured on a smaller buffer; DRAM traffic of this streaming kernel grows
    in proportion to the bytes read, so it is scaled to nbytes), or None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        tj = json.load(open(path))
    except Exception:
        return None, "no profiles/traffic.json"
    if tj.get("kernel_source_hash") != kernel_source_hash():
        return None, "kernels changed since the counters were taken"
    e = tj.get("points", {}).get(label)
    if not e:
        return None, f"no capture for {label}"
    return round(e["dram_bytes_per_launch"] * nbytes / e["bytes"]), \
        f"scaled from a {e['bytes'] >> 20} MiB capture ({tj.get('command', '')})"


def host_buffer(nbytes: int, pinned: bool):
    """Host copy of the workload, from the shared input generator."""
    import torch
    from paper_2608_15764_gb300 import workloads
    t = torch.empty(nbytes, dtype=torch.uint8, pin_memory=pinned)
    w = t.numpy().view("uint32")
    workloads.splitmix_u32(1, w.size, out=w)
    return t


def _roofline_simple(achieved: float, note: str) -> dict:
    """The HBM roofline object for a workload line without per-kernel DRAM
    counters (traffic null)."""
    peak, kind = _peaks()
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4),
            "peak_kind": f"{kind} copy (MEASURED_PEAKS.json hbm_gbs)" if kind == "measured" else "fallback",
            "traffic": None, "traffic_note": "no DRAM counters taken for this workload", "note": note}


def cpu_oracle(words, seconds: float):
    """Time the CPU oracle on all host cores over repeated full passes of the
    workload (each pass split into one contiguous range per thread; the
    per-range checksums combine exactly).  Returns (checksum, GB/s, threads,
    passes, seconds)."""
    import oracle
    threads = os.cpu_count() or 1
    n = words.size
    per = (n // threads) // 4 * 4
    cuts = [i * per for i in range(threads)] + [n]

    def one_pass():
        with ThreadPoolExecutor(max_workers=threads) as ex:
            parts = list(ex.map(lambda i: oracle.checksum(words[cuts[i]:cuts[i + 1]]), range(threads)))
        return oracle.combine(parts)

    ck = one_pass()  # warm (page-in)
    t0 = time.perf_counter()
    passes = 0
    while True:
        assert one_pass() == ck
        passes += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return ck, passes * words.nbytes / el / 1e9, threads, passes, el


def run_reference(a):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    nbytes = int(a.gib * (1 << 30)) // 16 * 16
    host = host_buffer(nbytes, pinned=False)
    words = host.numpy().view("uint32")
    import oracle
    ck, _, threads, _, _ = cpu_oracle(words, 0.0)
    times = []
    for i in range(a.warmup + a.steps):
        t0 = time.perf_counter()
        _, gbs, threads, passes, el = cpu_oracle(words, 0.0)
        if i >= a.warmup:
            times.append(el)
    total = sum(times)
    value = a.steps * nbytes / total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 2), "unit": "GB/s",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": round(1e3 * total / a.steps, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "bytes": nbytes, "l2": "n/a (host)"},
        "cpu_baseline": {"value": round(value, 2), "unit": "GB/s", "cores": threads, "kind": "oracle",
                         "sample": f"one full pass over the {nbytes >> 20} MiB host buffer per step, "
                                   f"split over {threads} threads"},
        "e2e": {"value": round(value, 2), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "checksum": {"sum_u32": ck[0], "xor_u64": ck[1]},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(a):
    import torch
    import paper_2608_15764_gb300 as sl
    from paper_2608_15764_gb300 import replicas, tune

    rank, world, local = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the streaming-load path has no CPU fallback)")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist = None
    sl.load()
    info = sl.sl_device_info()
    nbytes = int(a.gib * (1 << 30)) // 16 * 16
    buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    sl.sl_fill_splitmix64(buf, seed=1)
    # a second resident copy: back-to-back passes alternate between the two,
    # so no pass can find the previous pass's lines in L2
    buf2 = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    sl.sl_fill_splitmix64(buf2, seed=1)
    bufs = [buf, buf2]
    torch.cuda.synchronize()

    # ---- K-response curves and the choice (rank 0 decides, all ranks follow)
    points = tune.default_points()
    if a.choice:
        points = [tune.parse_point(a.choice)]
    # single-launch curves (the paper's K response), then the throughput of
    # back-to-back passes of every point, which picks the timed configuration
    if rank == 0 and a.choice:
        tune.measure(buf, nbytes, points, repeats=1, warmup=1)
        tune.measure_steps(bufs, nbytes, points, steps=8, repeats=1)
        choice = [0]
    elif rank == 0:
        tune.measure(buf, nbytes, points, repeats=a.curve_repeats, warmup=1)
        tune.measure_steps(bufs, nbytes, points, steps=16, repeats=a.curve_repeats)
        best = tune.choose(points, steps=True)
        choice = [points.index(best)]
    else:
        choice = [0]
    best = points[replicas.broadcast_choice(choice[0], dist)]
    cfg = best.cfg()

    # ---- timed steps: one pass per step.  Where the point allows it the
    # passes are programmatic dependent launches (sl_enqueue_steps: a pass
    # starts loading while the previous pass's tail runs), else one
    # sl_enqueue per pass.
    dev_out = torch.zeros((a.warmup + a.steps) * sl.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    rb = sl.RESULT_BYTES
    if best.overlapped:
        cfg = best.cfg(grid=0)  # one full wave of CTAs per pass
        sl.sl_enqueue_steps(bufs, dev_out, a.warmup, dtype=sl.SL_U32, cfg=cfg)
    else:
        for i in range(a.warmup):
            sl.sl_enqueue(bufs[i % 2], dev_out[rb * i:], dtype=sl.SL_U32, cfg=cfg)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(info["device"])
    if rank == 0:
        clocks.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps + 1)]
    ev[0].record(stream)
    if best.overlapped:
        sl.sl_enqueue_steps(bufs, dev_out[rb * a.warmup:], a.steps, dtype=sl.SL_U32, cfg=cfg)
        ev[a.steps].record(stream)
    else:
        for i in range(a.steps):
            sl.sl_enqueue(bufs[i % 2], dev_out[rb * (a.warmup + i):], dtype=sl.SL_U32, cfg=cfg)
            ev[i + 1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop() if rank == 0 else None
    total_ms = ev[0].elapsed_time(ev[a.steps])
    step_ms = ([total_ms / a.steps] * a.steps if best.overlapped
               else [ev[i].elapsed_time(ev[i + 1]) for i in range(a.steps)])
    total_ms = replicas.max_over_ranks(total_ms, dist, device="cuda")
    value = replicas.job_gbs(nbytes, a.steps, world, total_ms)

    # results of every timed step must agree, and so must the ranks (each
    # streams an identical buffer)
    raw = dev_out.cpu().numpy().tobytes()
    res = [sl.sl_result.from_buffer_copy(raw[rb * i:rb * (i + 1)]) for i in range(a.warmup + a.steps)]
    ck = {(r.sum_u32, r.xor_u64, r.issued_loads, r.status) for r in res}
    consistent = len(ck) == 1 and res[0].issued_loads == best.loads(nbytes) and res[0].status == 0
    per_rank = replicas.gather_results(res[-1].sum_u32, res[-1].xor_u64, res[-1].issued_loads, dist, device="cuda")
    ranks_agree = len(set(per_rank)) == 1

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    # ---- end to end through the public host-buffer entry point
    # Staged: 256 MiB copies to device staging overlapped with the kernel on
    # the previous chunk.  Direct: one kernel reads the pinned host buffer in
    # place over the CPU-GPU link (longer latency: more bytes in flight).  The
    # faster measured mode is reported.
    host = host_buffer(nbytes, pinned=True)
    e2e_cands = [("staged", best.label(), cfg)]
    for label, pt in [("direct", "ldgdyn:16:256"), ("direct", "ldgdyn:8:512"), ("direct", "ldgdyn:12:256"),
                      ("direct", "tma:65536:3:256"), ("direct", "tma:16384:8:512")]:
        p = tune.parse_point(pt)
        e2e_cands.append((label, p.label(), p.cfg(host_direct=True)))
    e2e_all = []
    for mode, label, c in e2e_cands:
        try:
            sl.sl_run_host(host, dtype=sl.SL_U32, cfg=c)  # warm (staging allocation, page mapping)
        except sl.SLError as e:
            e2e_all.append({"mode": mode, "point": label, "status": e.status})
            continue
        ts = []
        for _ in range(a.e2e_steps):
            t0 = time.perf_counter()
            r_ = sl.sl_run_host(host, dtype=sl.SL_U32, cfg=c)
            ts.append(time.perf_counter() - t0)
        e2e_all.append({"mode": mode, "point": label, "gbs": round(nbytes * len(ts) / sum(ts) / 1e9, 2),
                        "result": r_})
    ok = [e for e in e2e_all if "gbs" in e]
    e2e_best = max(ok, key=lambda e: e["gbs"])
    e2e_value = e2e_best["gbs"]
    rh = e2e_best["result"]
    e2e_host_ok = all((e["result"].sum_u32, e["result"].xor_u64) == (rh.sum_u32, rh.xor_u64) for e in ok)

    # ---- CPU oracle on the host cores (bounded sample) and parity
    words = host.numpy().view("uint32")
    oc, cpu_gbs, threads, passes, el = cpu_oracle(words, a.cpu_seconds)
    parity = (res[0].sum_u32, res[0].xor_u64) == oc and (rh.sum_u32, rh.xor_u64) == oc and e2e_host_ok

    peak, peak_kind = _peaks()
    kern_ms = statistics.mean(step_ms)
    achieved = nbytes / (kern_ms * 1e6)
    traffic, traffic_note = _traffic(best.label(), nbytes)
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": round(total_ms / a.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "bytes": nbytes, "choice": best.label(), "choice_spec": best.spec(),
                   "launch": "programmatic dependent launches (sl_enqueue_steps)" if best.overlapped
                   else "one sl_enqueue per step",
                   "grid": best.resident * info["sm_count"] if best.overlapped else best.grid_used,
                   "resident_per_sm": best.resident,
                   "l2": "inputs larger than L2 (4 GiB vs 129 MB), two resident copies read alternately by "
                         "consecutive steps: no flush between steps",
                   "parallelism": f"replicas x{world} (one buffer per GPU)"},
        "frac_of_datasheet": round(value / world / DATASHEET_GBS, 4),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_kind": f"{peak_kind} copy (MEASURED_PEAKS.json hbm_gbs)"
                     if peak_kind == "measured" else "fallback", "traffic": traffic,
                     "traffic_note": traffic_note,
                     "note": ("mean interval per pass of the overlapped launches (programmatic dependent "
                              "launches, one kernel per pass, CUDA events around the timed passes)"
                              if best.overlapped else
                              "per-step CUDA-event time of the load kernel, including its last-CTA combine")},
        "cpu_baseline": {"value": round(cpu_gbs, 2), "unit": "GB/s", "cores": threads, "kind": "oracle",
                         "sample": f"{passes} full passes over the {nbytes >> 20} MiB host buffer "
                                   f"({el:.1f} s wall, {threads} threads)"},
        "e2e": {"value": round(e2e_value, 2), "unit": "GB/s", "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": sl.RESULT_BYTES,
                "api": f"sl_run_host, pinned host buffer, {e2e_best['mode']} mode, {e2e_best['point']}",
                "modes": [{k: v for k, v in e.items() if k != "result"} for e in e2e_all]},
        "gpu_launches": a.steps,
        "clocks": clk,
        "parity": {"oracle_match": bool(parity), "steps_consistent": bool(consistent),
                   "ranks_agree": bool(ranks_agree)},
        "curves": [p.as_dict() for p in points],
        "device": {k: info[k] for k in ("name", "sm_count", "l2_bytes", "cc_major", "cc_minor")},
    }
    print(json.dumps(line), flush=True)
    if a.out:
        with open(a.out, "a") as f:
            f.write(json.dumps(line) + "\n")
    if dist:
        dist.destroy_process_group()
    return 0 if parity and consistent else 3


BATCH_METRIC = "aggregate GB/s, 1,024 uneven buffers in one autotuned CUDA-graph launch vs per-buffer launches"


def run_batch(a):
    """Batched precision form: for each payload dtype, 1,024 buffers with
    log-uniform sizes in 64 KiB - 256 MiB adding up to 16 GiB (N(0,1) payloads,
    FP8 scaled by 8), placed back to back in one device arena.  The autotuner
    picks mechanism / K / CTA per size class from measured curves; the batch
    (one graph launch) is timed against 1,024 per-buffer sl_enqueue launches
    (LDG K=2, 256 threads, 4 x SMs) queued on one stream with one final sync.
    Every buffer's uint32 checksum is checked against the oracle, and the
    float sums of 48 buffers spread over the size range."""
    import numpy as np
    import torch

    import oracle
    import paper_2608_15764_gb300 as sl
    from paper_2608_15764_gb300 import autotune
    from paper_2608_15764_gb300 import workloads as wl

    rank, world, local = _dist()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    sl.load()
    info = sl.sl_device_info()
    sizes = wl.batch_sizes(total=int(a.batch_gib * (1 << 30)))
    total = sum(sizes)
    offs = np.cumsum([0] + sizes[:-1])
    names = {"f32": wl.F32, "bf16": wl.BF16, "fp8": wl.FP8_E4M3, "u32": wl.U32}
    per, cpu_gbs = [], []
    threads = os.cpu_count() or 1
    host = torch.empty(total, dtype=torch.uint8, pin_memory=True)
    hv = host.numpy()
    dev = torch.empty(total, dtype=torch.uint8, device="cuda")
    base = dev.data_ptr()
    for name in a.dtypes.split(","):
        dt = names[name]
        t0 = time.perf_counter()
        if dt == wl.U32:
            wl.splitmix_u32(5, total // 4, out=hv.view(np.uint32))
        else:
            wl.payload(dt, total // wl.ELEM_BYTES[dt], out=hv.view(wl.NP_DTYPE[dt]))
        gen_s = time.perf_counter() - t0
        dev.copy_(host)
        torch.cuda.synchronize()
        bufs = [(base + int(o), nb, dt) for o, nb in zip(offs, sizes)]
        table, report = autotune.tune(bufs, repeats=3)
        b = sl.sl_batch_create(bufs, table)
        for _ in range(a.warmup):
            sl.sl_batch_run(b, results=False)
        ts = [sl.sl_batch_run(b, results=False)[1] for _ in range(a.steps)]
        res, _ = sl.sl_batch_run(b)
        batch_gbs = total * len(ts) / sum(ts)
        # per-buffer launches on one stream, one final sync
        cfg = sl.config("ldg", k=2, cta=256, grid=4 * info["sm_count"])
        out = torch.zeros(len(sizes) * sl.RESULT_BYTES, dtype=torch.uint8, device="cuda")
        stream = torch.cuda.current_stream()
        plain_ms = []
        for rep in range(a.warmup + a.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for i, (p, nb, _) in enumerate(bufs):
                sl.sl_enqueue(p, out[i * sl.RESULT_BYTES:], nbytes=nb, dtype=dt, cfg=cfg)
            e1.record(stream)
            torch.cuda.synchronize()
            if rep >= a.warmup:
                plain_ms.append(e0.elapsed_time(e1))
        plain_gbs = total * len(plain_ms) / (sum(plain_ms) * 1e6)
        raw = out.cpu().numpy().tobytes()
        plain = [sl.sl_result.from_buffer_copy(raw[i * sl.RESULT_BYTES:(i + 1) * sl.RESULT_BYTES])
                 for i in range(len(sizes))]
        # cpu_baseline leg: the oracle's checksum of every buffer on all host
        # cores, timed; its results are also the parity reference
        t0 = time.perf_counter()
        with ThreadPoolExecutor(threads) as ex:
            cks = list(ex.map(lambda i: oracle.checksum(hv[offs[i]:offs[i] + sizes[i]]), range(len(sizes))))
        cpu_gbs.append(total / (time.perf_counter() - t0) / 1e9)
        ck_ok = all((r.sum_u32, r.xor_u64, r.issued_loads) == (*ck, nb // 16) for r, ck, nb in zip(res, cks, sizes))
        ck_ok = ck_ok and all((r.sum_u32, r.xor_u64) == ck for r, ck in zip(plain, cks))
        worst = None
        if dt != wl.U32:
            # gate per buffer: relative to |exact sum|, or to sum|x| when the
            # exact sum is small against the payload (|ref| < 1e-3 sum|x| / sqrt(n))
            order = np.argsort(sizes)
            sample = [int(order[i]) for i in np.linspace(0, len(sizes) - 1, 48).astype(int)]
            with ThreadPoolExecutor(threads) as ex:
                refs = list(ex.map(lambda i: oracle.fsum(dt, hv[offs[i]:offs[i] + sizes[i]]), sample))
            errs = []
            for i, (ref, absum) in zip(sample, refs):
                nel = sizes[i] // wl.ELEM_BYTES[dt]
                small = abs(ref) < 1e-3 * absum / max(nel, 1) ** 0.5
                errs.append(abs(res[i].fsum - ref) / (absum if small else abs(ref)))
            worst = max(errs)
        sl.sl_batch_destroy(b)
        per.append({"dtype": name, "bytes": total, "batched_gbs": round(batch_gbs, 1),
                    "batched_ms": round(statistics.median(ts) / 1e6, 4), "per_buffer_gbs": round(plain_gbs, 1),
                    "per_buffer_ms": round(statistics.median(plain_ms), 4),
                    "speedup": round(batch_gbs / plain_gbs, 3), "frac_of_datasheet": round(batch_gbs / DATASHEET_GBS, 4),
                    "checksums_match_oracle": bool(ck_ok), "fsum_max_gated_err_sample48": worst,
                    "host_generation_s": round(gen_s, 1),
                    "tuning": [{k: r[k] for k in ("class", "buffers", "bytes", "choice", "gbs")} for r in report]})
    all_bytes = sum(p["bytes"] for p in per)
    value = all_bytes / sum(p["bytes"] / p["batched_gbs"] for p in per)
    line = {"metric": BATCH_METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": 1, "steps": a.steps,
            "warmup": a.warmup, "higher_is_better": True, "data": "synthetic", "dtype": a.dtypes,
            "config": {"workload": f"1,024 buffers, log-uniform 64 KiB-256 MiB, {a.batch_gib:g} GiB per dtype "
                                   "(N(0,1), FP8 x8), one device arena",
                       "l2": "inputs larger than L2; each buffer read once per launch"},
            "cpu_baseline": {"value": round(len(cpu_gbs) / sum(1.0 / v for v in cpu_gbs), 2), "unit": "GB/s",
                             "cores": threads, "kind": "oracle",
                             "sample": "the oracle's uint32 checksum of all 1,024 buffers per dtype, "
                                       "buffers spread over the host threads"},
            "roofline": _roofline_simple(value, "aggregate bytes of all buffers / CUDA-event time of the graph "
                                                "launch (all class kernels and the combine)"),
            "per_dtype": per,
            "parity": all(p["checksums_match_oracle"] for p in per) and
            all(p["fsum_max_gated_err_sample48"] is None or p["fsum_max_gated_err_sample48"] <= 2e-6 for p in per)}
    print(json.dumps(line), flush=True)
    if a.out:
        with open(a.out, "a") as f:
            f.write(json.dumps(line) + "\n")
    return 0 if line["parity"] else 3


PREC_METRIC = "attained GB/s of the compensated FP32 sum (FP64 final combine) per payload dtype and mechanism"
PREC_CELLS = ([dict(mech="ldg", k=k, cta=256) for k in (1, 2, 4, 8, 16)] +
              [dict(mech="ldg", k=k, cta=256, order="dyn") for k in (2, 4, 8)] +
              [dict(mech="cpasync", k=d, cta=256) for d in (2, 4, 6)] +
              [dict(mech="tma", stage_bytes=sb, stages=n, cta=256) for sb, n in ((16384, 2), (16384, 4), (65536, 2))])


def run_prec(a):
    """Precision form: N(0,1) payloads of --prec-gib GiB (float32, bfloat16,
    FP8-E4M3 x8; inputs larger than L2) through every point of PREC_CELLS,
    `steps` timed launches each.  cpu_baseline leg: the oracle's FP64
    Neumaier sum of the same payload on all host cores (one contiguous range
    per thread, range sums added with math.fsum), timed; it is also the
    reference for the error of every GPU sum, reported relative to |sum| and
    normalised by sum|x|.  value = the harmonic mean over dtypes of each
    dtype's fastest point."""
    import math

    import numpy as np
    import torch

    import oracle
    import paper_2608_15764_gb300 as sl
    from paper_2608_15764_gb300 import workloads as wl

    rank, world, local = _dist()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    sl.load()
    nbytes = int(a.prec_gib * (1 << 30)) // 16 * 16
    threads = os.cpu_count() or 1
    per, cpu = [], []
    worst_all = 0.0
    clocks = ClockSampler(local)
    for dt in (wl.F32, wl.BF16, wl.FP8_E4M3):
        name = {wl.F32: "f32", wl.BF16: "bf16", wl.FP8_E4M3: "fp8"}[dt]
        n = nbytes // wl.ELEM_BYTES[dt]
        host = wl.payload(dt, n)
        hb = host.view(np.uint8)
        cut = [i * (n // threads) // 16 * 16 for i in range(threads)] + [n]
        t0 = time.perf_counter()
        with ThreadPoolExecutor(threads) as ex:
            parts = list(ex.map(lambda i: oracle.fsum(dt, host[cut[i]:cut[i + 1]]), range(threads)))
        cpu_s = time.perf_counter() - t0
        cpu.append(nbytes / cpu_s / 1e9)
        ref = math.fsum(p[0] for p in parts)
        absum = math.fsum(p[1] for p in parts)
        dev = torch.from_numpy(hb).cuda()
        cfgs = [sl.config(c["mech"], **{k: v for k, v in c.items() if k != "mech"}) for c in PREC_CELLS]
        clocks.start()
        res = sl.sl_sweep(dev, cfgs, dtype=dt, repeats=a.steps, warmup=a.warmup)
        clk = clocks.stop()
        points = []
        for c, rr in zip(PREC_CELLS, res):
            gbs = [nbytes / r.device_ns for r in rr if r.status == 0 and r.device_ns]
            fs = [r.fsum for r in rr]
            err = max(abs(f - ref) for f in fs)
            small = abs(ref) < 1e-3 * absum / max(n, 1) ** 0.5
            gated = err / (absum if small else abs(ref))
            worst_all = max(worst_all, gated)
            points.append({**c, "gbs_median": round(statistics.median(gbs), 1) if gbs else None,
                           "rel_err": err / abs(ref), "err_over_abs_sum": err / absum, "gated_err": gated,
                           "deterministic": len(set(fs)) == 1})
        best = max(points, key=lambda p: p["gbs_median"] or 0)
        per.append({"dtype": name, "bytes": nbytes, "ref_fsum": ref, "abs_sum": absum, "best": best,
                    "points": points, "clocks": clk, "oracle_gbs": round(cpu[-1], 2)})
        del dev
        torch.cuda.empty_cache()
    value = len(per) / sum(1.0 / p["best"]["gbs_median"] for p in per)
    line = {"metric": PREC_METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": 1, "steps": a.steps,
            "warmup": a.warmup, "higher_is_better": True, "data": "synthetic", "dtype": "f32,bf16,fp8",
            "config": {"workload": f"{a.prec_gib:g} GiB N(0,1) payload per dtype (FP8 x8), one launch per step",
                       "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": round(len(cpu) / sum(1.0 / v for v in cpu), 2), "unit": "GB/s",
                             "cores": threads, "kind": "oracle",
                             "sample": "one FP64 Neumaier pass over each full payload, split over the host threads"},
            "roofline": _roofline_simple(value, "harmonic mean over dtypes of the fastest point's bytes / "
                                                "CUDA-event time of one launch"),
            "per_dtype": per, "max_gated_err": worst_all, "parity": worst_all <= 2e-6}
    print(json.dumps(line), flush=True)
    if a.out:
        with open(a.out, "a") as f:
            f.write(json.dumps(line) + "\n")
    return 0 if line["parity"] else 3


def main(argv=None):
    a = _args(argv)
    if a.impl == "reference":
        return run_reference(a)
    if a.workload == "batch":
        return run_batch(a)
    if a.workload == "prec":
        return run_prec(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
