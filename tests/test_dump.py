"""The triage dump of a level hierarchy (save_hierarchy / load_hierarchy,
written on the GPU side by HGraph.dump_hierarchy) round-trips every array,
size and cid map, including levels 10 and above whose key prefixes share
their first characters with levels 1 to 9."""
import numpy as np

from paper_2609_07577_gb300.api import load_hierarchy, save_hierarchy


def test_round_trip(tmp_path):
    rng = np.random.Generator(np.random.PCG64(0))
    levels, cids = [], []
    for l in range(12):
        V, E, P = 20 - l, 10 - l // 2, 30 - l
        levels.append({"off": np.sort(rng.integers(0, P, E + 1)).astype(np.int64),
                       "pins": rng.integers(0, V, P).astype(np.int32),
                       "w": rng.integers(1, 9, E).astype(np.int64),
                       "selfdst": rng.integers(0, 2, E).astype(np.uint8),
                       "size": rng.integers(1, 4, V).astype(np.int32), "V": V, "E": E, "P": P})
        if l < 11:
            cids.append(rng.integers(0, V - 1, V).astype(np.int32))
    path = tmp_path / "h.npz"
    save_hierarchy(path, levels, cids)
    got_levels, got_cids = load_hierarchy(path)
    assert len(got_levels) == 12 and len(got_cids) == 11
    for a, b in zip(levels, got_levels):
        assert a.keys() == b.keys()
        for k in a:
            np.testing.assert_array_equal(np.asarray(a[k]), np.asarray(b[k]))
            if k in ("V", "E", "P"):
                assert isinstance(b[k], int)
            else:
                assert b[k].dtype == a[k].dtype
    for a, b in zip(cids, got_cids):
        np.testing.assert_array_equal(a, b)


def test_write_trace(tmp_path):
    import json
    from paper_2609_07577_gb300.api import write_trace
    path = tmp_path / "t.jsonl"
    stages = {"affinity": {"calls": 3, "ms": 1.5}}
    levels = [{"V": 10, "E": 5, "P": 20, "n_cand": 8, "n_pairs": 4, "pair_terms": 30,
               "n_block": 0, "n_global": 0}, {"V": 6, "E": 4, "P": 12, "n_cand": 0,
                                              "n_pairs": 0, "pair_terms": 9, "n_block": 0,
                                              "n_global": 0}]
    rounds = [{"level": 1, "round": 0, "n_props": 3, "istar": 2, "n_active": 6, "rows": 0,
               "gain": 7}]
    assert write_trace(path, stages, levels, rounds, {"workload": "t"}) == 4
    assert write_trace(path, stages, levels[:1], [], None) == 2
    lines = [json.loads(x) for x in open(path)]
    assert [x["kind"] for x in lines] == ["pass", "level", "level", "round", "pass", "level"]
    assert lines[0]["workload"] == "t" and lines[0]["stages"] == stages
    assert lines[2]["level"] == 1 and lines[2]["V"] == 6
    assert lines[3]["gain"] == 7 and lines[3]["istar"] == 2
