"""Full-size checks on the 1,048,576-neuron conv workload, in the launch
configuration bench.py times (device-resident inputs, snnmap_partition).

The whole pass equals the oracle's stored result (tests/golden/full_cfg2.json:
Conn, statistics, every level's and every round's log, the hash of rho), and
so does the 2^17-neuron power-law workload in four path settings. Besides,
the oracle checks a random sample of level-0 candidates one vertex at a
time, and properties that hold at any size are checked: the matching pairs
vertices along candidate arcs and never twice, contraction conserves
neurons, inbound pins and axons, the final partition respects Omega, Phi and
Delta, its Conn recomputed independently equals the reported cost, and the
host-buffer entry point returns the same partition.
"""
import numpy as np
import pytest
import torch

import oracle
import snngen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    import __graft_entry__ as g
    g.build()
    hg = snngen.cfg2()
    return hg


def conn_np(hg, rho):
    E = hg.E
    hid = np.repeat(np.arange(E, dtype=np.int64), np.diff(hg.off))
    K = int(rho.max()) + 1
    key = np.unique(hid * K + rho[hg.pins].astype(np.int64))
    lam = np.bincount(key // K, minlength=E)
    return int((hg.w.astype(np.int64) * (lam - 1)).sum())


def test_level0_candidates_sampled(big):
    from paper_2609_07577_gb300 import HGraph
    hg = big
    prm = oracle.params_of(hg)
    G = HGraph.from_hypergraph(hg)
    try:
        nc, npairs = G.coarsen_level()
        cand, cs, cov, match = G.last_matching()
    finally:
        G.close()
    L = oracle.Level.from_hypergraph(hg, prm)
    rng = np.random.default_rng(7)
    sample = np.concatenate([rng.choice(hg.V, 1500, replace=False), [0, hg.V - 1]])
    for n in sample:
        assert (cand[n], cs[n], cov[n]) == L.cand_one(int(n), prm), n
    assert nc == int((cand >= 0).sum())
    # matching: symmetric, along candidate arcs, roots matched
    idx = np.nonzero(match >= 0)[0]
    assert (match[match[idx]] == idx).all()
    assert ((cand[idx] == match[idx]) | (cand[match[idx]] == idx)).all()
    has = cand >= 0
    roots = has & (cand[np.where(has, cand, 0)] == np.arange(hg.V))
    assert (match[roots] == cand[roots]).all()
    assert npairs == int((match > np.arange(hg.V)).sum())


def test_full_pass_properties(big):
    from paper_2609_07577_gb300 import HGraph, params_for, snnmap_partition_host
    hg = big
    G = HGraph.from_hypergraph(hg)
    try:
        rho_t, cost, st = G.partition()
        rho = rho_t.cpu().numpy()
        levels = G.level_logs()
        rounds = G.round_logs()
        a0 = G.level_arrays(0)
    finally:
        G.close()
    assert cost == conn_np(hg, rho)
    assert st["cost_initial"] - sum(r["gain"] for r in rounds) == cost
    assert all(r["gain"] > 0 for r in rounds if r["istar"] > 0)
    K = st["n_parts"]
    assert rho.min() >= 0 and rho.max() < K
    assert (np.bincount(rho, minlength=K) <= hg.omega).all()
    assert (np.bincount(rho, weights=a0["inpins"], minlength=K) <= hg.phi).all()
    isdst = np.ones(hg.P, bool)
    isdst[hg.off[:-1]] = False
    hid = np.repeat(np.arange(hg.E, dtype=np.int64), np.diff(hg.off))
    key = np.unique(rho[hg.pins[isdst]].astype(np.int64) * hg.E + hid[isdst])
    assert (np.bincount(key // hg.E, minlength=K) <= hg.delta).all()
    # coarsening shrinks the vertex count at every contraction
    Vs = [g["V"] for g in levels]
    assert all(b < a for a, b in zip(Vs, Vs[1:]))
    # the host-buffer entry point gives the same partition
    h_rho = np.empty(hg.V, np.int32)
    c2, _ = snnmap_partition_host(params_for(hg.omega, hg.delta, hg.phi), hg.V, hg.E,
                                  np.ascontiguousarray(hg.off), np.ascontiguousarray(hg.pins),
                                  np.ascontiguousarray(hg.w), h_rho)
    assert c2 == cost and np.array_equal(h_rho, rho)


def test_contraction_conserves(big):
    from paper_2609_07577_gb300 import HGraph
    hg = big
    G = HGraph.from_hypergraph(hg)
    try:
        a0 = G.level_arrays(0)
        for _ in range(3):
            nc, npairs = G.coarsen_level()
            if npairs == 0:
                break
            G.contract()
        a = G.level_arrays(G.num_levels() - 1)
    finally:
        G.close()
    assert int(a["size"].sum()) == hg.V
    assert int(a["inpins"].sum()) == int(a0["inpins"].sum())
    assert int(a["k"].sum()) + int(a["in_internal"].sum()) == a0["E"]
    # in_count equals its recomputation from the coarse hyperedges
    inc = a["in_internal"].astype(np.int64).copy()
    lens = np.diff(a["off"])
    hid = np.repeat(np.arange(a["E"]), lens)
    isdst = np.ones(a["P"], bool)
    isdst[a["off"][:-1]] = False
    np.add.at(inc, a["pins"][isdst], a["k"][hid[isdst]])
    sd = a["selfdst"].astype(bool)
    np.add.at(inc, a["pins"][a["off"][:-1]][sd], a["k"][sd])
    assert (inc == a["in_count"]).all()
    assert (a["size"] <= hg.omega).all() and (a["inpins"] <= hg.phi).all()
    assert (a["in_count"] <= hg.delta).all()


# ---------------------------------------------------------------------------
# Whole passes against the oracle's stored results (tests/golden/full_*.json,
# written by tests/golden/make_fullsize.py from oracle.partition alone): the
# 1,048,576-neuron conv workload, and the 2^17-neuron power-law workload that
# has the 2^23-neuron workload's fan-out law, locality and limits.

def _golden(name):
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", f"full_{name}.json")
    with open(path) as f:
        return json.load(f)


def _check_against_golden(hg, gold, setup=None):
    import hashlib
    from paper_2609_07577_gb300 import HGraph
    G = HGraph.from_hypergraph(hg)
    try:
        if setup is not None:
            setup(G)
        rho, cost, st = G.partition()
        rho = rho.cpu().numpy()
        lv, rl = G.level_logs(), G.round_logs()
    finally:
        G.close()
    assert (hg.V, hg.E, hg.P) == (gold["V"], gold["E"], gold["P"])
    assert cost == gold["cost"]
    for k, v in gold["stats"].items():
        assert st[k] == v, k
    assert [(g["V"], g["E"], g["P"], g["n_cand"], g["n_pairs"]) for g in lv] == \
           [(g["V"], g["E"], g["P"], g["n_cand"], g["n_pairs"]) for g in gold["levels"]]
    assert [(r["level"], r["round"], r["n_props"], r["istar"], r["gain"]) for r in rl] == \
           [(r["level"], r["round"], r["n_props"], r["istar"], r["gain"]) for r in gold["rounds"]]
    assert hashlib.sha256(np.ascontiguousarray(rho, np.int32).tobytes()).hexdigest() == \
        gold["rho_sha256"]
    return lv


def test_full_pass_equals_oracle_conv(big):
    _check_against_golden(big, _golden("cfg2"))


@pytest.mark.parametrize("mode,rows", [(0, None), (1, 0), (2, 0), (2, None)])
def test_full_pass_equals_oracle_power_law(mode, rows):
    hg = snngen.by_name("cfg3m")

    def setup(G):
        G.set_coarsen_mode(mode)
        if rows is not None:
            G.set_row_budget(rows)

    lv = _check_against_golden(hg, _golden("cfg3m"), setup)
    if mode == 2 and rows == 0:
        assert all(x["carried"] == 1 for x in lv[1:])


def _properties(hg, rho, cost, levels, inpins):
    assert cost == conn_np(hg, rho)
    K = int(rho.max()) + 1
    assert (np.bincount(rho, minlength=K) <= hg.omega).all()
    assert (np.bincount(rho, weights=inpins, minlength=K) <= hg.phi).all()
    isdst = np.ones(hg.P, bool)
    isdst[hg.off[:-1]] = False
    hid = np.repeat(np.arange(hg.E, dtype=np.int64), np.diff(hg.off))
    key = np.unique(rho[hg.pins[isdst]].astype(np.int64) * hg.E + hid[isdst])
    assert (np.bincount(key // hg.E, minlength=K) <= hg.delta).all()
    Vs = [g["V"] for g in levels]
    assert all(b < a for a, b in zip(Vs, Vs[1:]))


def test_power_law_2e23_sampled_and_properties():
    """The 2^23-neuron power-law workload: level-0 candidates of 1,500
    sampled vertices equal the oracle's one-vertex evaluation, and the whole
    pass satisfies Conn, Omega, Phi and Delta."""
    from paper_2609_07577_gb300 import HGraph
    hg = snngen.cfg3()
    prm = oracle.params_of(hg)
    G = HGraph.from_hypergraph(hg)
    try:
        G.coarsen_level()
        cand, cs, cov, _ = G.last_matching()
        a0 = G.level_arrays(0)
    finally:
        G.close()
    L = oracle.Level.from_hypergraph(hg, prm)
    rng = np.random.default_rng(9)
    for n in np.concatenate([rng.choice(hg.V, 1500, replace=False), [0, hg.V - 1]]):
        assert (cand[n], cs[n], cov[n]) == L.cand_one(int(n), prm), n
    del L
    G = HGraph.from_hypergraph(hg)
    try:
        rho_t, cost, st = G.partition()
        rho = rho_t.cpu().numpy()
        levels = G.level_logs()
    finally:
        G.close()
    _properties(hg, rho, cost, levels, a0["inpins"])
