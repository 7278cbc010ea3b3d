"""Autotuner of the batched form: per size class, the mechanism, K (or D, or
stage size x stages) and CTA shape with the highest measured aggregate GB/s.

For every (dtype, size class) present in a batch, each candidate
configuration is run as a one-class batch over exactly that class's buffers
(the same class kernel, graph and combine the full batch uses), timed with
CUDA events around the graph launch (best of `repeats` after a warm-up), and
the fastest candidate wins; candidates within `tie_frac` of the best count as
ties, broken towards fewer bytes in flight per CTA.  The result is a tuning
table for sl_batch_create plus the measured response curve of every class.
"""
from __future__ import annotations

import json

from . import (SL_CPASYNC, SL_LDG, SL_TMA, config, sl_batch_create, sl_batch_destroy, sl_batch_run,
               tune_entry, SLError)

KIB, MIB = 1 << 10, 1 << 20
# size classes (inclusive bounds), by orders of magnitude of the 64 KiB - 256 MiB range
CLASSES = [(0, MIB - 1), (MIB, 16 * MIB - 1), (16 * MIB, 1 << 62)]


def candidates():
    c = [dict(mech=SL_LDG, k=k, cta=256) for k in (2, 4, 8, 16)]
    c += [dict(mech=SL_LDG, k=k, cta=512) for k in (4, 8)]
    c += [dict(mech=SL_LDG, k=8, cta=128)]
    c += [dict(mech=SL_CPASYNC, k=d, cta=256) for d in (4, 6)]
    c += [dict(mech=SL_TMA, cta=256, stage_bytes=sb, stages=n) for sb, n in ((16384, 2), (16384, 4), (65536, 2),
                                                                             (4096, 8))]
    return c


def _cfg(c):
    if c["mech"] == SL_TMA:
        return config(SL_TMA, cta=c["cta"], stage_bytes=c["stage_bytes"], stages=c["stages"])
    return config(c["mech"], k=c["k"], cta=c["cta"])


def _offered(c):
    return c["stage_bytes"] * c["stages"] if c["mech"] == SL_TMA else c["k"] * c["cta"] * 16


def label(c) -> str:
    if c["mech"] == SL_TMA:
        return f"tma S={c['stage_bytes'] // KIB}K x{c['stages']} cta={c['cta']}"
    return f"{'ldg K' if c['mech'] == SL_LDG else 'cpasync D'}={c['k']} cta={c['cta']}"


def tune(buffers, repeats: int = 3, tie_frac: float = 0.01, verbose: bool = False):
    """buffers: sequence of (device buffer, nbytes, dtype).  Returns
    (table: list of sl_tune_entry, report: list of dicts)."""
    table, report = [], []
    dtypes = sorted({int(dt) for _, _, dt in buffers})
    for dt in dtypes:
        for lo, hi in CLASSES:
            sub = [(b, nb, d) for b, nb, d in buffers if int(d) == dt and lo <= nb <= hi]
            if not sub:
                continue
            nbytes = sum(nb for _, nb, _ in sub)
            curve = []
            for c in candidates():
                entry = tune_entry(lo, hi, _cfg(c), dtype=dt)
                try:
                    b = sl_batch_create(sub, [entry])
                except SLError as e:
                    curve.append({"cand": label(c), "status": e.status})
                    continue
                try:
                    sl_batch_run(b, results=False)  # warm-up
                    best_ns = min(sl_batch_run(b, results=False)[1] for _ in range(repeats))
                except SLError as e:
                    curve.append({"cand": label(c), "status": e.status})
                    continue
                finally:
                    sl_batch_destroy(b)
                curve.append({"cand": label(c), "status": 0, "gbs": nbytes / best_ns, "cfg": c})
            ok = [p for p in curve if p["status"] == 0]
            top = max(p["gbs"] for p in ok)
            pick = min((p for p in ok if p["gbs"] >= top * (1 - tie_frac)), key=lambda p: _offered(p["cfg"]))
            table.append(tune_entry(lo, hi, _cfg(pick["cfg"]), dtype=dt))
            rep = {"dtype": dt, "class": [lo, hi], "buffers": len(sub), "bytes": nbytes, "choice": pick["cand"],
                   "gbs": round(pick["gbs"], 1),
                   "curve": [{k: (round(v, 1) if isinstance(v, float) else v) for k, v in p.items() if k != "cfg"}
                             for p in curve]}
            report.append(rep)
            if verbose:
                print(json.dumps({k: rep[k] for k in ("dtype", "class", "buffers", "choice", "gbs")}), flush=True)
    return table, report


def plain_table(cfg=None):
    """A one-entry table applying one configuration to every buffer."""
    return [tune_entry(0, 1 << 62, cfg or config(SL_LDG, k=2, cta=256), dtype=-1)]
