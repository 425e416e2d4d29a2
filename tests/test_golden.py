"""Oracle against hand-worked examples (tests/golden/*.json, each citing the
passage of the paper it works through)."""
import json
import os

import numpy as np

import oracle
from helpers import canonical_hedges, hypergraph

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def test_conn_examples():
    g = load("conn_examples.json")
    for c in g["cases"]:
        hg = hypergraph(c["V"], c["hedges"], c["w"], 100, 100, 100)
        L = oracle.Level.from_hypergraph(hg)
        assert L.conn(np.array(c["rho"], np.int32)) == c["conn"]


def test_affinity_example_step_by_step():
    g = load("affinity_example.json")
    hg = hypergraph(g["V"], g["hedges"], g["w"], g["omega"], g["delta"], g["phi"])
    prm = oracle.params_of(hg)
    L = oracle.Level.from_hypergraph(hg, prm)
    cand, cscore, cov = L.affinity(prm)
    assert cand.tolist() == g["cand"]
    assert cscore.tolist() == g["cscore"]
    assert cov.tolist() == g["cov"]
    for n in range(g["V"]):
        assert L.cand_one(n, prm) == (g["cand"][n], g["cscore"][n], g["cov"][n])
    m, pairs = oracle.match(cand, cscore)
    assert m.tolist() == g["match"]
    assert pairs == 2
    C, cid = L.contract(m, cand, cov)
    assert cid.tolist() == g["cid"]
    a = C.arrays()
    for key in ("size", "inpins", "in_count", "in_internal"):
        assert a[key].tolist() == g["coarse"][key], key
    got = canonical_hedges(a["off"], a["pins"], a["w"], a["k"], a["selfdst"])
    want = sorted((h[0], h[1], tuple(h[2]), h[3], h[4]) for h in g["coarse"]["hedges"])
    assert got == want
    c2, _, _ = C.affinity(prm)
    assert (c2 < 0).all()


def test_affinity_example_full_pass():
    g = load("affinity_example.json")
    hg = hypergraph(g["V"], g["hedges"], g["w"], g["omega"], g["delta"], g["phi"])
    rho, cost, st, levels, rounds = oracle.partition(hg)
    assert rho.tolist() == g["rho"]
    assert cost == g["conn"]
    assert st["levels"] == g["levels"]


def test_match_forest():
    g = load("match_forest.json")
    m, pairs = oracle.match(np.array(g["cand"], np.int32), np.array(g["cscore"], np.int64))
    assert m.tolist() == g["match"]
    assert pairs == sum(1 for i, x in enumerate(g["match"]) if x > i)


def test_refine_examples():
    g = load("refine_examples.json")
    for c in g["cases"]:
        hg = hypergraph(c["V"], c["hedges"], c["w"], c["omega"], c["delta"], c["phi"])
        prm = oracle.params_of(hg)
        L = oracle.Level.from_hypergraph(hg, prm)
        rho = np.array(c["rho_in"], np.int32)
        assert L.conn(rho) == c["conn_in"], c["name"]
        rounds, moves, logs = L.refine(c["K"], rho, prm)
        assert rho.tolist() == c["rho_out"], c["name"]
        assert L.conn(rho) == c["conn_out"], c["name"]
        assert [{k: r[k] for k in ("n_props", "istar", "gain")} for r in logs] == c["rounds"]
