"""Oracle pinned to brute force on random hypergraphs of at most 12 neurons.

Every level the oracle builds is checked against the definitions restated in
``bruteforce.py`` on the original neurons: super-node state, coarse
hyperedges, score/overlap/candidate (Eq. neigh_histogram), the matching
(Eq. matching, memoised recursion), one refinement round (gains as Conn
differences, validity by direct constraint checks), and the whole pass
(feasible, cost = Conn, cost >= the exhaustive optimum, zero cost when every
connected component fits one core).
"""
import numpy as np
import pytest

import bruteforce as bf
import oracle
import snngen
from helpers import canonical_hedges

SEEDS = range(2400)


def _levels(hg, prm):
    """Drive the oracle level by level; yields (level, cid chain, cand, cscore, cov)."""
    L = oracle.Level.from_hypergraph(hg, prm)
    cids = []
    while True:
        cand, cs, cov = L.affinity(prm)
        yield L, list(cids), cand, cs, cov
        if (cand < 0).all() or len(cids) >= prm.max_levels:
            return
        m, pairs = oracle.match(cand, cs)
        L, cid = L.contract(m, cand, cov)
        cids.append(cid)


def _single_infeasible(hg, prm):
    ins = bf.in_sets(hg)
    return any(not bf.group_ok(hg, {n}, prm, ins) for n in range(hg.V))


@pytest.mark.parametrize("chunk", range(6))
def test_levels_match_bruteforce(chunk):
    checked = 0
    for seed in SEEDS[chunk::6]:
        hg = snngen.tiny_random(seed)
        prm = oracle.params_of(hg)
        try:
            gen = list(_levels(hg, prm))
        except oracle.OracleError as e:
            assert e.code == oracle.ERR_INFEASIBLE
            assert _single_infeasible(hg, prm)
            continue
        assert not _single_infeasible(hg, prm)
        for L, cids, cand, cs, cov in gen:
            img, mem = bf.members(cids, hg.V)
            a = L.arrays()
            size, inpins, in_count, internal = bf.level_state(hg, img, mem)
            assert a["size"].tolist() == size
            assert a["inpins"].tolist() == inpins
            assert a["in_count"].tolist() == in_count
            assert a["in_internal"].tolist() == internal
            assert canonical_hedges(a["off"], a["pins"], a["w"], a["k"], a["selfdst"]) == \
                bf.coarse_hedges(hg, img)
            bc, bs, bo = bf.candidates(hg, img, mem, prm)
            assert cand.tolist() == bc
            assert cs.tolist() == bs
            assert cov.tolist() == bo
            if (cand >= 0).any():
                m, pairs = oracle.match(cand, cs)
                bm = bf.matching(cand.tolist(), cs.tolist())
                assert m.tolist() == bm
                assert pairs == sum(1 for i, x in enumerate(bm) if x > i) > 0
            checked += 1
    assert checked > 50


@pytest.mark.parametrize("chunk", range(4))
def test_refine_round_matches_bruteforce(chunk):
    rng = np.random.default_rng(1234 + chunk)
    rounds_checked = moved = 0
    for seed in range(chunk, 2400, 4):
        hg = snngen.tiny_random(10_000 + seed)
        prm = oracle.params_of(hg, max_refine_rounds=1)
        try:
            levels = list(_levels(hg, prm))
        except oracle.OracleError:
            continue
        for L, cids, _, _, _ in levels:
            img, mem = bf.members(cids, hg.V)
            VL = len(mem)
            for _ in range(3):
                K = int(rng.integers(1, VL + 1))
                rho = rng.integers(0, K, size=VL).astype(np.int32)
                if not bf.feasible(hg, rho[img], prm):
                    continue
                want, props, istar, gain = bf.refine_round(hg, img, VL, rho.tolist(), K, prm)
                got = rho.copy()
                r, mv, logs = L.refine(K, got, prm)
                assert got.tolist() == want
                assert logs[0]["n_props"] == props
                assert logs[0]["istar"] == istar
                assert logs[0]["gain"] == gain
                assert bf.conn(hg, rho[img]) - bf.conn(hg, got[img]) == gain
                rounds_checked += 1
                moved += istar > 0
    assert rounds_checked > 100 and moved > 20


@pytest.mark.parametrize("chunk", range(3))
def test_whole_pass_against_optimum(chunk):
    nopt = 0
    for seed in range(chunk, 240, 3):
        hg = snngen.tiny_random(50_000 + seed, V=int(3 + seed % 6))
        prm = oracle.params_of(hg)
        try:
            rho, cost, st, levels, rounds = oracle.partition(hg, prm)
        except oracle.OracleError as e:
            assert e.code == oracle.ERR_INFEASIBLE
            continue
        assert bf.feasible(hg, rho, prm)
        assert cost == bf.conn(hg, rho)
        assert st["cost_initial"] - cost == sum(r["gain"] for r in rounds)
        opt = bf.optimum(hg, prm)
        assert cost >= opt
        if bf.components_fit(hg, prm):
            assert cost == 0 == opt
        nopt += 1
    assert nopt > 30


def test_components_fitting_one_core_cost_zero():
    """Special case pinned exactly: loose limits collapse every component."""
    n = 0
    for seed in range(200):
        hg = snngen.tiny_random(70_000 + seed)
        hg.omega, hg.delta, hg.phi = 12, 10_000, 10_000
        rho, cost, st, levels, rounds = oracle.partition(hg)
        assert bf.components_fit(hg, oracle.params_of(hg))
        assert cost == 0
        n += 1
    assert n == 200


def test_invalid_inputs_rejected():
    from helpers import hypergraph
    bad = [
        hypergraph(3, [[0, 1, 1]], [1], 5, 5, 5),     # duplicate destination
        hypergraph(3, [[0, 1, 0]], [1], 5, 5, 5),     # source among destinations
        hypergraph(3, [[0, 3]], [1], 5, 5, 5),        # id out of range
        hypergraph(3, [[0, 1]], [-1], 5, 5, 5),       # negative weight
        hypergraph(3, [[0, 1]], [1], 0, 5, 5),        # Omega < 1
    ]
    for hg in bad:
        with pytest.raises(oracle.OracleError) as e:
            oracle.Level.from_hypergraph(hg)
        assert e.value.code == oracle.ERR_INVALID
    empty = hypergraph(3, [[0, 1], []], [1, 1], 5, 5, 5)   # hyperedge with no pin
    with pytest.raises(oracle.OracleError):
        oracle.Level.from_hypergraph(empty)
    inf = hypergraph(3, [[0, 2], [1, 2]], [1, 1], 5, 1, 5)  # neuron 2 alone has 2 inbound axons
    with pytest.raises(oracle.OracleError) as e:
        oracle.Level.from_hypergraph(inf)
    assert e.value.code == oracle.ERR_INFEASIBLE


@pytest.mark.parametrize("chunk", range(2))
def test_refine_round_variant_matches_bruteforce(chunk):
    """The variant of reading R19 (every vertex proposes its best feasible
    adjacent move whatever its gain) against the set-based restatement: the
    non-positive proposals join the sorted sequence and a prefix is still
    enacted only with positive cumulative gain and validity."""
    rng = np.random.default_rng(4321 + chunk)
    rounds_checked = moved = extra = 0
    for seed in range(chunk, 2400, 4):
        hg = snngen.tiny_random(10_000 + seed)
        prm = oracle.params_of(hg, max_refine_rounds=1, refine_nonpositive=1)
        base = oracle.params_of(hg, max_refine_rounds=1)
        try:
            levels = list(_levels(hg, base))
        except oracle.OracleError:
            continue
        for L, cids, _, _, _ in levels:
            img, mem = bf.members(cids, hg.V)
            VL = len(mem)
            for _ in range(2):
                K = int(rng.integers(1, VL + 1))
                rho = rng.integers(0, K, size=VL).astype(np.int32)
                if not bf.feasible(hg, rho[img], prm):
                    continue
                want, props, istar, gain = bf.refine_round(hg, img, VL, rho.tolist(), K, prm)
                _, props0, _, _ = bf.refine_round(hg, img, VL, rho.tolist(), K, base)
                got = rho.copy()
                r, mv, logs = L.refine(K, got, prm)
                assert got.tolist() == want
                assert logs[0]["n_props"] == props >= props0
                assert logs[0]["istar"] == istar
                assert logs[0]["gain"] == gain
                rounds_checked += 1
                moved += istar > 0
                extra += props > props0
    assert rounds_checked > 50 and moved > 10 and extra > 10
