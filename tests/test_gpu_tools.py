"""HGraph.dump_hierarchy on the GPU: after a pass, the .npz holds every
level's arrays and cid maps exactly as the inspection calls return them
(levels released under the memory budget are rebuilt for the dump), and its
level 0 has the oracle's sizes (the parity tests compare the arrays). The
JSONL trace of a profiled pass holds its stage times, levels and rounds, and
the command line maps a hypergraph file (partition and placement)."""
import numpy as np
import pytest

import oracle
import snngen

pytestmark = pytest.mark.gpu


def test_dump_equals_inspection(tmp_path):
    from paper_2609_07577_gb300 import HGraph
    from paper_2609_07577_gb300.api import load_hierarchy
    hg = snngen.by_name("cfg1s")
    G = HGraph.from_hypergraph(hg)
    try:
        G.partition()
        G.dump_hierarchy(tmp_path / "h.npz")
        levels, cids = load_hierarchy(tmp_path / "h.npz")
        n = G.num_levels()
        assert len(levels) == n and len(cids) == n - 1
        for l in sorted({0, n // 2, n - 1}):
            want = G.level_arrays(l)
            assert want.keys() == levels[l].keys()
            for k in want:
                np.testing.assert_array_equal(np.asarray(levels[l][k]), np.asarray(want[k]))
        for l in range(n - 1):
            np.testing.assert_array_equal(cids[l], G.level_cid(l))
    finally:
        G.close()
    L0 = oracle.Level.from_hypergraph(hg, oracle.params_of(hg))
    assert (levels[0]["V"], levels[0]["E"], levels[0]["P"]) == L0.dims()


def test_trace_jsonl(tmp_path):
    import json
    from paper_2609_07577_gb300 import HGraph
    hg = snngen.by_name("cfg1s")
    G = HGraph.from_hypergraph(hg)
    try:
        G.profile(True)
        G.partition()
        path = tmp_path / "t.jsonl"
        G.trace(path, {"workload": "cfg1s"})
        levels, rounds = G.level_logs(), G.round_logs()
    finally:
        G.close()
    lines = [json.loads(x) for x in open(path)]
    assert lines[0]["kind"] == "pass" and lines[0]["workload"] == "cfg1s"
    assert lines[0]["stages"]["affinity"]["calls"] > 0
    assert sum(x["kind"] == "level" for x in lines) == len(levels) > 0
    assert sum(x["kind"] == "round" for x in lines) == len(rounds) > 0


def test_cli_map_with_placement(tmp_path):
    """python -m paper_2609_07577_gb300 map: the partition equals the
    oracle's, and the placement gives every partition its own core of the
    lattice."""
    from paper_2609_07577_gb300.__main__ import main
    from paper_2609_07577_gb300.snnfile import save_snn
    hg = snngen.by_name("cfg1s")
    src, dst = str(tmp_path / "in.npz"), str(tmp_path / "out.npz")
    save_snn(src, hg)
    assert main(["map", src, dst, "--place", "--starts", "4"]) == 0
    rho_o, cost_o, st_o, *_ = oracle.partition(hg, oracle.params_of(hg))
    with np.load(dst) as z:
        np.testing.assert_array_equal(z["rho"], rho_o)
        assert int(z["cost"]) == cost_o
        gamma, (w, h) = z["gamma"], z["lattice"]
        # one G_P node (and core) per non-empty partition, in id order
        np.testing.assert_array_equal(z["parts"], np.unique(rho_o))
        assert len(gamma) == st_o["nonempty_parts"] and len(set(gamma.tolist())) == len(gamma)
        assert gamma.min() >= 0 and gamma.max() < w * h and int(z["trd"]) > 0
