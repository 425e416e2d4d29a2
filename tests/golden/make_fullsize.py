"""Writes the full-size expected values of the oracle (tests/golden/full_<name>.json):
final Conn, the level log (V, E, P, candidates and pairs per level), the
per-round log, the stats and the sha256 of rho. Every value comes from
``oracle.partition`` on the seeded generator of ``snngen``; nothing here
runs the CUDA library.

    python tests/golden/make_fullsize.py cfg3m cfg2
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import snngen  # noqa: E402


def golden(name):
    hg = snngen.by_name(name)
    t = time.perf_counter()
    rho, cost, stats, levels, rounds = oracle.partition(hg, log_cap=1 << 16)
    dt = time.perf_counter() - t
    rho = np.ascontiguousarray(rho, np.int32)
    return {
        "workload": name,
        "source": "oracle.partition on snngen.by_name(%r) (tests/golden/make_fullsize.py)" % name,
        "V": int(hg.V), "E": int(hg.off.shape[0] - 1), "P": int(hg.P),
        "cost": int(cost), "stats": {k: int(v) for k, v in stats.items()},
        "rho_sha256": hashlib.sha256(rho.tobytes()).hexdigest(),
        "levels": levels, "rounds": rounds, "oracle_s": round(dt, 1),
    }


if __name__ == "__main__":
    for name in sys.argv[1:]:
        g = golden(name)
        with open(os.path.join(HERE, f"full_{name}.json"), "w") as f:
            json.dump(g, f, separators=(",", ":"))
        print(name, g["cost"], g["stats"]["levels"], g["oracle_s"], "s", flush=True)
