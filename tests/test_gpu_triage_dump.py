"""HGraph.dump_hierarchy on the GPU: after a pass, the .npz holds every
level's arrays and cid maps exactly as the inspection calls return them
(levels released under the memory budget are rebuilt for the dump), and its
level 0 has the oracle's sizes (the parity tests compare the arrays). The
JSONL trace of a profiled pass holds its stage times, levels and rounds."""
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
