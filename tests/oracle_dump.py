"""Triage of a parity mismatch. `dump` steps the oracle through the
coarsening of a named workload and writes every intermediate -- each level's
arrays, candidates, scores, shared inbound counts, matching and cid map --
and the final partition to one .npz, in the key layout of
paper_2609_07577_gb300.api.save_hierarchy (which HGraph.dump_hierarchy
writes on the GPU side). `compare` reads two such files and names the first
level and array that differ (hyperedges compared in canonical order, since
the two sides may list them differently).

    python tests/oracle_dump.py dump <workload> <out.npz> [--max-levels N]
    python tests/oracle_dump.py compare <a.npz> <b.npz>

Test infrastructure: it runs the oracle."""
import argparse
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

import oracle  # noqa: E402
import snngen  # noqa: E402
from helpers import canonical_hedges  # noqa: E402

VERTEX_KEYS = ("size", "inpins", "in_count", "in_internal")
STEP_KEYS = ("cand", "cscore", "cov", "match")


def dump(name, out, max_levels=None):
    """Writes the oracle's hierarchy of workload `name`; returns the number
    of levels written."""
    hg = snngen.by_name(name)
    prm = oracle.params_of(hg)
    L = oracle.Level.from_hypergraph(hg, prm)
    arrays = {}
    lev = 0
    while True:
        for k, v in L.arrays().items():
            arrays[f"L{lev}_{k}"] = np.asarray(v)
        if max_levels is not None and lev >= max_levels:
            break
        cand, cscore, cov = L.affinity(prm)
        if not (cand >= 0).any():
            break
        match, _ = oracle.match(cand, cscore)
        for k, v in zip(STEP_KEYS, (cand, cscore, cov, match)):
            arrays[f"L{lev}_{k}"] = v
        L, cid = L.contract(match, cand, cov)
        arrays[f"L{lev}_cid"] = cid
        lev += 1
    arrays["n_levels"] = np.int64(lev + 1)
    if max_levels is None:
        rho, cost, _, *_ = oracle.partition(hg, prm)
        arrays["rho"] = rho
        arrays["cost"] = np.int64(cost)
    np.savez_compressed(out, **arrays)
    return lev + 1


def compare(a, b):
    """Returns a list of differences (empty when the hierarchies agree)."""
    from paper_2609_07577_gb300.api import load_hierarchy
    la, ca = load_hierarchy(a)
    lb, cb = load_hierarchy(b)
    diffs = []
    if len(la) != len(lb):
        diffs.append(f"levels: {len(la)} vs {len(lb)}")
    for lev, (x, y) in enumerate(zip(la, lb)):
        tag = f"level {lev}"
        for k in ("V", "E", "P"):
            if x.get(k) != y.get(k):
                diffs.append(f"{tag} {k}: {x.get(k)} vs {y.get(k)}")
        for k in VERTEX_KEYS + STEP_KEYS:
            if k in x and k in y and not np.array_equal(x[k], y[k]):
                i = int(np.flatnonzero(np.asarray(x[k]) != np.asarray(y[k]))[0]) \
                    if np.shape(x[k]) == np.shape(y[k]) else -1
                diffs.append(f"{tag} {k}" + (f" first at vertex {i}" if i >= 0 else " sizes"))
        if all(k in x and k in y for k in ("off", "pins", "w", "k", "selfdst")):
            hx = canonical_hedges(x["off"], x["pins"], x["w"], x["k"], x["selfdst"])
            hy = canonical_hedges(y["off"], y["pins"], y["w"], y["k"], y["selfdst"])
            if hx != hy:
                first = next((i for i, (p, q) in enumerate(zip(hx, hy)) if p != q),
                             min(len(hx), len(hy)))
                diffs.append(f"{tag} hyperedges: first canonical difference at {first}")
        if diffs:
            break
    if not diffs:
        for lev, (x, y) in enumerate(zip(ca, cb)):
            if not np.array_equal(x, y):
                diffs.append(f"level {lev} cid")
                break
    return diffs


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    d = sub.add_parser("dump")
    d.add_argument("workload")
    d.add_argument("out")
    d.add_argument("--max-levels", type=int, default=None)
    c = sub.add_parser("compare")
    c.add_argument("a")
    c.add_argument("b")
    args = ap.parse_args(argv)
    if args.cmd == "dump":
        n = dump(args.workload, args.out, args.max_levels)
        print(f"{n} levels written to {args.out}")
        return 0
    diffs = compare(args.a, args.b)
    for line in diffs:
        print(line)
    print("equal" if not diffs else "different")
    return 1 if diffs else 0


if __name__ == "__main__":
    sys.exit(main())
