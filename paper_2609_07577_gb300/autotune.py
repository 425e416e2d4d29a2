"""Autotuning of the histogram tier thresholds by input size.

The histogram engine (neighbour histograms of coarsening, connection
histograms of refinement) places each vertex on a warp, a block, a large
block or the split tier by the work its histogram visits; the thresholds
between the tiers (wwork, bwork, gwork) decide that placement, never a
result. `sweep` times whole passes of sample jobs of each input-size class
under candidate thresholds (coordinate descent: one threshold at a time,
starting from the built-in defaults), checks that every setting gives the
same Conn, and writes the best setting per class to tier_table.json beside
this file. `load_table` hands that table to the library
(snnmap_set_tier_table), after which every handle built from an input of P
pins takes the row of its size class; `_native.lib()` calls it when it
loads the library.

    python -m paper_2609_07577_gb300.autotune [--out PATH]
"""
from __future__ import annotations

import json
import os
import time

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "tier_table.json")

# size classes by level-0 pins (upper bounds), and the candidates tried for
# each threshold
CLASSES = [1 << 21, 1 << 23, 1 << 25, 1 << 62]
CANDIDATES = {
    "wwork": [2048, 4096, 8192, 16384],
    "bwork": [1 << 14, 1 << 15, 1 << 16, 1 << 17],
    "gwork": [1 << 20, 1 << 21, 1 << 22, 1 << 23],
}
DEFAULTS = {"wwork": 8192, "bwork": 1 << 16, "gwork": 1 << 22}


def load_table(path=TABLE):
    """Installs the table at `path` in the library (no-op without a file);
    returns its rows."""
    from . import _native as N
    try:
        with open(path) as f:
            rows = json.load(f)["rows"]
    except (OSError, ValueError, KeyError):
        return []
    N.snnmap_set_tier_table([tuple(int(x) for x in r) for r in rows])
    return rows


def sample_jobs(per_class=2, scan=64):
    """Jobs of the batched workload (seed = job index), the first `per_class`
    of each generator (layered, power-law) in every size class; classes the
    batched workload does not reach take scaled-up instances of the conv
    and power-law generators."""
    import snngen
    picked = {c: [] for c in CLASSES}
    kinds = {c: set() for c in CLASSES}
    for j in range(scan):
        hg = snngen.batch_jobs_one(j)
        c = next(c for c in CLASSES if hg.P <= c)
        kind = j % 2
        if sum(1 for k in picked[c] if k[0] == kind) < per_class:
            picked[c].append((kind, hg))
            kinds[c].add(kind)
    big = [snngen.by_name("cfg2q"),
           snngen.powerlaw(1 << 19, 65536, 8, 16384, 2.1, 0.7, seed=7, omega=4096, delta=16384,
                           phi=65536, name="pl19")]
    for hg in big:
        c = next(c for c in CLASSES if hg.P <= c)
        if len(picked[c]) < 2 * per_class:
            picked[c].append((-1, hg))
    return {c: [hg for _, hg in v] for c, v in picked.items()}


def time_passes(hgs, tiers, repeat=2):
    """Summed median pass time (s) of the jobs under `tiers`, and their Conn."""
    import torch

    from .api import HGraph
    total, costs = 0.0, []
    for hg in hgs:
        G = HGraph.from_hypergraph(hg)
        try:
            G.set_histogram_tiers(tiers["wwork"], tiers["bwork"], tiers["gwork"])
            ts = []
            for _ in range(repeat):
                torch.cuda.synchronize()
                t = time.perf_counter()
                _, cost, _ = G.partition()
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t)
            costs.append(cost)
        finally:
            G.close()
        total += sorted(ts)[len(ts) // 2]
    return total, costs


def sweep(out=TABLE, per_class=2, log=print):
    """Coordinate descent per size class; writes and returns the table."""
    import torch

    from . import _native as N
    N.snnmap_set_tier_table([])
    jobs = sample_jobs(per_class)
    rows, detail = [], []
    for c in CLASSES:
        hgs = jobs[c]
        if not hgs:
            continue
        best = dict(DEFAULTS)
        t0, ref = time_passes(hgs, best)
        tried = [(dict(best), t0)]
        for key in ("wwork", "bwork", "gwork"):
            for v in CANDIDATES[key]:
                if v == best[key]:
                    continue
                cand = dict(best, **{key: v})
                if cand["wwork"] > cand["bwork"] or cand["bwork"] > cand["gwork"]:
                    continue
                t, costs = time_passes(hgs, cand)
                if costs != ref:
                    raise RuntimeError(f"tier setting {cand} changed a result: {costs} != {ref}")
                tried.append((cand, t))
                if t < t0:
                    best, t0 = cand, t
        log(f"class <= {c} pins: {len(hgs)} jobs, best {best} {t0:.3f} s")
        rows.append([c, best["wwork"], best["bwork"], best["gwork"]])
        detail.append({"max_pins": c, "jobs": [(hg.name, hg.P) for hg in hgs],
                       "tried": [(t, round(s, 4)) for t, s in tried]})
    table = {"rows": rows, "gpu": torch.cuda.get_device_name(0),
             "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()), "detail": detail}
    with open(out, "w") as f:
        json.dump(table, f, indent=1)
    N.snnmap_set_tier_table([tuple(r) for r in rows])
    return table


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=TABLE)
    ap.add_argument("--per-class", type=int, default=2)
    a = ap.parse_args()
    sweep(a.out, a.per_class)
