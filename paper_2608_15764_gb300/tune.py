"""Response-curve measurement and configuration choice.

A curve is attained GB/s per offered-concurrency point of one mechanism
(LDG: K; cp.async: depth D; TMA: stage size x stages) on one buffer.  The
choice rule picks the point with the highest median GB/s; points within
``tie_frac`` of the best count as ties, broken towards the smaller offered
load (fewer loads in flight), then LDG before cp.async before TMA.

Infeasible points (shared memory, registers, occupancy) are recorded with
their status instead of being silently shrunk.
"""
from __future__ import annotations

import statistics
from dataclasses import dataclass, field

from . import (SL_ASC, SL_CPASYNC, SL_LDG, SL_LDG32, SL_OK, SL_RING_CTA, SL_RING_WARP, SL_TMA, SL_U32, SLError,
               config, sl_plan, sl_sweep)

MECH_NAMES = {SL_LDG: "ldg", SL_CPASYNC: "cpasync", SL_TMA: "tma", SL_LDG32: "ldg32"}


@dataclass
class Point:
    mech: int
    k: int = 0            # K (LDG) or D (cp.async)
    cta: int = 256
    grid: int = 0
    stage_bytes: int = 0  # TMA
    stages: int = 0       # TMA
    ring: int = SL_RING_CTA  # TMA: one ring per CTA or per warp
    copies: int = 1       # cp.async: 16-byte copies per commit group (G)
    cop: int = 0
    order: int = 0        # SL_ASC, or SL_DYN (dynamic contiguous chunks, LDG)
    gbs: list = field(default_factory=list)  # per repeat
    step_gbs: list = field(default_factory=list)  # back-to-back passes, per repeat
    window_gbs: list = field(default_factory=list)
    status: int = SL_OK
    resident: int = 0
    grid_used: int = 0
    results: set = field(default_factory=set)  # distinct (sum_u32, xor_u64, issued_loads, status) seen

    def cfg(self, **kw):
        """The point's sl_config; keyword arguments override its fields."""
        if self.mech == SL_TMA:
            base = dict(cta=self.cta, grid=self.grid, stage_bytes=self.stage_bytes, stages=self.stages,
                        ring=self.ring)
        else:
            base = dict(k=self.k, cta=self.cta, grid=self.grid, cop=self.cop)
            if self.copies != 1:
                base["copies"] = self.copies
            if self.order:
                base["order"] = self.order
        base.update(kw)
        return config(self.mech, **base)

    @property
    def median(self) -> float:
        return statistics.median(self.gbs) if self.gbs else 0.0

    @property
    def step_median(self) -> float:
        return statistics.median(self.step_gbs) if self.step_gbs else 0.0

    def loads(self, nbytes: int) -> int:
        """Loads one pass over nbytes issues at this point's width (16-byte
        loads; ceil(nbytes/32) for 32-byte loads)."""
        return (nbytes + 31) // 32 if self.mech == SL_LDG32 else nbytes // 16

    @property
    def overlapped(self) -> bool:
        """Back-to-back passes run as programmatic dependent launches
        (sl_enqueue_steps): every mechanism and traversal."""
        return True

    @property
    def offered(self) -> int:
        """Offered in-flight bytes per CTA (for tie-breaking)."""
        if self.mech == SL_TMA:
            return self.stage_bytes * self.stages
        return self.k * self.copies * self.cta * (32 if self.mech == SL_LDG32 else 16)

    def label(self) -> str:
        if self.mech == SL_TMA:
            ring = " per-warp stages" if self.ring == SL_RING_WARP else ""
            return f"tma S={self.stage_bytes // 1024}K x{self.stages} cta={self.cta}{ring}"
        dyn = " dyn" if self.order == 2 else ""
        if self.mech == SL_CPASYNC:
            g = f" G={self.copies}" if self.copies != 1 else ""
            return f"cpasync D={self.k}{g} cta={self.cta}{dyn}"
        return f"{MECH_NAMES[self.mech]} K={self.k} cta={self.cta} cop={self.cop}{dyn}"

    def spec(self) -> str:
        """The point in parse_point's notation."""
        if self.mech == SL_TMA:
            return f"{'tmaw' if self.ring == SL_RING_WARP else 'tma'}:{self.stage_bytes}:{self.stages}:{self.cta}"
        name = MECH_NAMES[self.mech] + ("dyn" if self.order == 2 else "")
        if self.mech == SL_LDG and self.order != 2:
            return f"ldg:{self.k}:{self.cta}:{self.cop}"
        if self.mech == SL_CPASYNC:
            g = f":{self.copies}" if self.copies != 1 else ""
            return f"{name}:{self.k}:{self.cta}{g}"
        return f"{name}:{self.k}:{self.cta}"

    def as_dict(self) -> dict:
        d = {"mech": MECH_NAMES[self.mech], "cta": self.cta, "grid": self.grid_used, "status": self.status,
             "resident_per_sm": self.resident, "gbs_median": round(self.median, 1),
             "gbs": [round(v, 1) for v in self.gbs]}
        if self.step_gbs:
            d.update(steps_gbs_median=round(self.step_median, 1), steps_overlapped=self.overlapped)
        if self.mech == SL_TMA:
            d.update(stage_bytes=self.stage_bytes, stages=self.stages,
                     ring="warp" if self.ring == SL_RING_WARP else "cta")
        else:
            d.update(k=self.k, cop=self.cop, order=self.order)
            if self.mech == SL_CPASYNC:
                d.update(copies=self.copies)
        return d


def parse_point(text: str) -> Point:
    """'ldg:K:cta[:cop]', 'ldgdyn:K:cta', 'ldg32:K:cta', 'ldg32dyn:K:cta', 'cpasync:D:cta[:G]',
    'cpasyncdyn:D:cta[:G]',
    'tma:stage_bytes:stages:cta' (one ring per CTA, producer warp) or 'tmaw:stage_bytes:stages[:cta]'
    (the CTA's stages dealt to its warps; cta defaults to warp_ring_cta)."""
    f = text.split(":")
    if f[0] == "tmaw":
        sb, n = int(f[1]), int(f[2])
        return Point(SL_TMA, stage_bytes=sb, stages=n, ring=SL_RING_WARP,
                     cta=int(f[3]) if len(f) > 3 else warp_ring_cta(sb, n))
    if f[0] in ("ldgdyn", "ldg32dyn", "ldg32"):
        return Point(SL_LDG32 if f[0].startswith("ldg32") else SL_LDG, k=int(f[1]),
                     cta=int(f[2]) if len(f) > 2 else 256, order=2 if f[0].endswith("dyn") else 0)
    mech = f[0]
    if mech == "tma":
        return Point(SL_TMA, stage_bytes=int(f[1]), stages=int(f[2]), cta=int(f[3]) if len(f) > 3 else 256)
    if mech == "ldg":
        return Point(SL_LDG, k=int(f[1]), cta=int(f[2]) if len(f) > 2 else 256, cop=int(f[3]) if len(f) > 3 else 0)
    if mech in ("cpasync", "cpasyncdyn"):
        return Point(SL_CPASYNC, k=int(f[1]), cta=int(f[2]) if len(f) > 2 else 256,
                     copies=int(f[3]) if len(f) > 3 else 1, order=2 if mech.endswith("dyn") else 0)
    raise ValueError(f"bad point {text!r}")


def warp_ring_cta(stage_bytes: int, stages: int) -> int:
    """CTA size of a TMA point whose CTA ring is dealt to its warps: one warp
    per stage (each warp owns one stage of stage_bytes)."""
    return 32 * stages


# cp.async points with several copies per commit group (D, G): the same bytes
# in flight as D*G one-copy groups, with fewer commits and waits
CP_GROUP_POINTS = ((1, 2), (2, 2), (1, 4), (2, 4), (1, 8))
# cp.async under the dynamic-chunk traversal (D, G)
CP_DYN_POINTS = ((2, 1), (3, 1), (4, 1), (6, 1), (8, 1), (1, 8), (2, 8))
TMA_STAGE_BYTES = (4096, 16384, 65536)
TMA_STAGES = tuple(range(2, 9))


def default_points(cta: int = 256) -> list[Point]:
    """The K-response catalogue: LDG K 1-16 (16 bytes, .cg), four .L2::256B
    points, the dynamic-chunk traversal, 32-byte loads, cp.async D 1-8 (and
    five points with 2-8 copies per commit group, and seven under the
    dynamic-chunk traversal), and
    TMA stage sizes 4/16/64 KiB x 2-8 stages in both ring layouts (read by
    all `cta` consumer threads, and by 128 for 4 KiB stages; dealt to the
    warps, one stage per warp and, for even stage counts, two).
    Points whose shared memory does not fit are kept and recorded as
    infeasible by measure()."""
    pts = [Point(SL_LDG, k=k, cta=cta) for k in range(1, 17)]
    pts += [Point(SL_LDG, k=k, cta=cta, cop=1) for k in (1, 2, 4, 8)]
    pts += [Point(SL_LDG, k=k, cta=cta, order=2) for k in (1, 2, 3, 4, 6, 8, 12, 16)]
    pts += [Point(SL_LDG, k=k, cta=512, order=2) for k in (2, 4)]
    pts += [Point(SL_LDG32, k=k, cta=cta) for k in (1, 2, 3, 4, 6, 8)]
    pts += [Point(SL_LDG32, k=k, cta=cta, order=2) for k in (1, 2, 3, 4, 6, 8)]
    pts += [Point(SL_CPASYNC, k=d, cta=cta) for d in range(1, 9)]
    pts += [Point(SL_CPASYNC, k=d, cta=cta, copies=g) for d, g in CP_GROUP_POINTS]
    pts += [Point(SL_CPASYNC, k=d, cta=cta, copies=g, order=2) for d, g in CP_DYN_POINTS]
    pts += [Point(SL_TMA, cta=cta, stage_bytes=s, stages=n) for s in TMA_STAGE_BYTES for n in TMA_STAGES]
    # with 4 KiB stages a 256-thread CTA gives each consumer lane a single
    # 16-byte vector per stage; 128 consumer threads read two
    pts += [Point(SL_TMA, cta=128, stage_bytes=4096, stages=n) for n in TMA_STAGES]
    pts += [Point(SL_TMA, cta=c, stage_bytes=s, stages=n, ring=SL_RING_WARP)
            for s in TMA_STAGE_BYTES for n in TMA_STAGES
            for c in ([32 * n, 16 * n] if n % 2 == 0 else [32 * n])]
    return pts


def measure(buf, nbytes: int, points: list[Point], dtype: int = SL_U32, repeats: int = 3, warmup: int = 1,
            sweep_order=SL_ASC, flush_l2: bool = False) -> list[Point]:
    """Measure every point with sl_sweep (one sweep over all feasible cells)."""
    feasible = []
    for p in points:
        try:
            r = sl_plan(nbytes, dtype, p.cfg())
            p.resident = r.resident_per_sm
            p.grid_used = r.grid
            feasible.append(p)
        except SLError as e:
            p.status = e.status
    if not feasible:
        return points
    rows = sl_sweep(buf, [p.cfg(flush_l2=flush_l2) for p in feasible], nbytes=nbytes, dtype=dtype,
                    repeats=repeats, warmup=warmup, sweep_order=sweep_order)
    for p, row in zip(feasible, rows):
        p.results.update((r.sum_u32, r.xor_u64, r.issued_loads, r.status) for r in row)
        p.status = next((r.status for r in row if r.status != SL_OK), SL_OK)
        p.gbs = [nbytes / r.device_ns for r in row if r.status == SL_OK and r.device_ns]
        p.window_gbs = [nbytes / r.window_ns for r in row if r.status == SL_OK and r.window_ns]
    return points


def measure_steps(bufs, nbytes: int, points: list[Point], steps: int = 8, repeats: int = 3,
                  dtype: int = SL_U32) -> list[Point]:
    """Throughput of `steps` back-to-back passes for every measured point,
    pass i reading bufs[i % len(bufs)]: one sl_enqueue_steps call
    (overlapped passes, one full wave of CTAs) where the point allows it, else
    `steps` sl_enqueue calls; CUDA events on the current stream around the
    passes, after one untimed round; median of `repeats` into step_gbs.  The
    passes' results of the last repeat join the point's `results`."""
    import torch

    from . import RESULT_BYTES, sl_enqueue, sl_enqueue_steps, sl_result
    bufs = list(bufs) if isinstance(bufs, (list, tuple)) else [bufs]
    out = torch.zeros(steps * RESULT_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def run(p, cfg):
        if p.overlapped:
            sl_enqueue_steps(bufs, out, steps, nbytes=nbytes, dtype=dtype, cfg=p.cfg(grid=0))
        else:
            for i in range(steps):
                sl_enqueue(bufs[i % len(bufs)], out[i * RESULT_BYTES:], nbytes=nbytes, dtype=dtype, cfg=cfg)

    for p in points:
        if p.status != SL_OK or not p.gbs:
            continue
        cfg = p.cfg()
        run(p, cfg)
        p.step_gbs = []
        for _ in range(repeats):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run(p, cfg)
            e1.record(stream)
            torch.cuda.synchronize()
            p.step_gbs.append(nbytes * steps / (e0.elapsed_time(e1) * 1e6))
        raw = out.cpu().numpy().tobytes()
        for i in range(steps):
            r = sl_result.from_buffer_copy(raw[i * RESULT_BYTES:(i + 1) * RESULT_BYTES])
            p.results.add((r.sum_u32, r.xor_u64, r.issued_loads, r.status))
    return points


def choose(points: list[Point], tie_frac: float = 0.005, steps: bool = False) -> Point:
    """Highest median GB/s of single launches (steps=False) or of back-to-back
    passes (steps=True); ties within tie_frac go to fewer bytes in flight,
    then LDG before cp.async before TMA."""
    def val(p):
        return p.step_median if steps else p.median
    ok = [p for p in points if p.status == SL_OK and (p.step_gbs if steps else p.gbs)]
    if not ok:
        raise RuntimeError("no feasible measured point")
    best = max(val(p) for p in ok)
    ties = [p for p in ok if val(p) >= best * (1 - tie_frac)]
    return min(ties, key=lambda p: (p.offered, p.mech))
