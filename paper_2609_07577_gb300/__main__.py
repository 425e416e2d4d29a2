"""Command line: map an SNN hypergraph file onto cores.

    python -m paper_2609_07577_gb300 map INPUT.npz OUT.npz [--omega N --delta N --phi N]
                                         [--place] [--starts 64] [--seed 0]

INPUT.npz is snnfile.save_snn's format (off, pins, w, V and the per-core limits;
limits given here override the file's). The partition runs on the GPU
(Sec. 4.1); with --place, the partition hypergraph G_P is placed on the
smallest near-square lattice of cores by the multi-start placement of Sec.
4.2. OUT.npz holds rho (neuron -> partition), cost (Conn), the pass's
statistics, and with --place the G_P arrays over the non-empty partitions
(parts: the partition id of each G_P node), gamma (G_P node -> core), the
lattice and the total residual distance."""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np


def parse(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2609_07577_gb300",
                                 description=__doc__.split("\n\n")[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    m = sub.add_parser("map", help="partition (and optionally place) an SNN hypergraph")
    m.add_argument("input")
    m.add_argument("output")
    m.add_argument("--omega", type=int, default=None)
    m.add_argument("--delta", type=int, default=None)
    m.add_argument("--phi", type=int, default=None)
    m.add_argument("--place", action="store_true")
    m.add_argument("--starts", type=int, default=64)
    m.add_argument("--seed", type=int, default=0)
    args = ap.parse_args(argv)
    if args.starts < 1:
        ap.error("--starts must be at least 1")
    return args


def map_file(args):
    """Runs one `map` command; returns the dict written to the output."""
    import torch

    from .api import HGraph, place
    from .snnfile import load_snn
    hg = load_snn(args.input, args.omega, args.delta, args.phi)
    G = HGraph.from_hypergraph(hg)
    try:
        rho, cost, stats = G.partition()
        out = {"rho": rho.cpu().numpy(), "cost": np.int64(cost),
               "stats": np.asarray(json.dumps(stats))}
        if args.place:
            # G_P over the non-empty partitions only, numbered densely in
            # the order of their ids (parts[i] is the id of G_P node i), so
            # that no core is spent on a partition refinement emptied
            rho_h = out["rho"]
            parts = np.unique(rho_h).astype(np.int32)
            dense = np.searchsorted(parts, rho_h).astype(np.int32)
            K = int(parts.shape[0])
            gp = G.partition_graph(torch.from_numpy(dense).to(rho.device), K)
            res = place(K, gp["off"], gp["pins"], gp["eta"], n_starts=args.starts,
                        seed=args.seed)
            out.update(gp_off=gp["off"], gp_pins=gp["pins"], gp_eta=gp["eta"], parts=parts,
                       gamma=res["gamma"], trd=np.int64(res["trd"]),
                       lattice=np.asarray([res["width"], res["height"]], np.int32))
    finally:
        G.close()
    np.savez_compressed(args.output, **out)
    return out


def main(argv=None):
    args = parse(argv)
    out = map_file(args)
    stats = json.loads(str(out["stats"]))
    line = f"{args.input}: {stats['nonempty_parts']} partitions, Conn {int(out['cost'])}"
    if "trd" in out:
        line += f", placed on {out['lattice'][0]}x{out['lattice'][1]} cores, " \
                f"total residual distance {int(out['trd'])}"
    print(line)
    return 0


if __name__ == "__main__":
    sys.exit(main())
