"""The triage CLI (tests/oracle_dump.py): the oracle's hierarchy of a
workload is written level by level with its intermediates, reads back
through the package's load_hierarchy, matches the oracle's own pass (level
count, final cost), compares equal to itself, and a planted difference in a
hyperedge or a matching is named at the right level."""
import numpy as np

import oracle
import oracle_dump
import snngen
from paper_2609_07577_gb300.api import load_hierarchy


def test_dump_and_compare(tmp_path):
    a = str(tmp_path / "a.npz")
    n = oracle_dump.dump("cfg1s", a)
    hg = snngen.by_name("cfg1s")
    _, cost, stats, *_ = oracle.partition(hg, oracle.params_of(hg))
    assert n == stats["levels"] + 1
    levels, cids = load_hierarchy(a)
    assert len(levels) == n and len(cids) == n - 1
    assert all("match" in levels[l] for l in range(n - 1))
    with np.load(a) as z:
        assert int(z["cost"]) == cost
        assert len(z["rho"]) == hg.V
    assert oracle_dump.compare(a, a) == []
    assert oracle_dump.main(["compare", a, a]) == 0

    # a hyperedge changed at level 1, and a matching changed at level 2
    with np.load(a) as z:
        d = {k: z[k] for k in z.files}
    d["L1_w"] = d["L1_w"].copy()
    d["L1_w"][3] += 1
    b = str(tmp_path / "b.npz")
    np.savez_compressed(b, **d)
    diffs = oracle_dump.compare(a, b)
    assert diffs and diffs[0].startswith("level 1 hyperedges")
    with np.load(a) as z:
        d = {k: z[k] for k in z.files}
    d["L2_match"] = d["L2_match"].copy()
    d["L2_match"][0] = -7
    np.savez_compressed(b, **d)
    diffs = oracle_dump.compare(a, b)
    assert diffs == ["level 2 match first at vertex 0"]
    assert oracle_dump.main(["compare", a, b]) == 1


def test_dump_stops_at_level_cap(tmp_path):
    out = str(tmp_path / "c.npz")
    assert oracle_dump.dump("cfg1s", out, max_levels=2) == 3
    levels, cids = load_hierarchy(out)
    assert len(levels) == 3 and len(cids) == 2
