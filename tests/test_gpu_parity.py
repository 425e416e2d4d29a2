"""CUDA path against the oracle, bit-exact: every level's arrays, candidates,
scores, shared inbound counts, matching and cid maps, then the final
partition, its Conn and the refinement logs, on seeded inputs of several
shapes (scaled-down generators spanning many warps, blocks and all
hyperedge size buckets, plus tiny random hypergraphs)."""
import numpy as np
import pytest
import torch

import oracle
import snngen
from gpu_helpers import lockstep
from helpers import hypergraph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__ as g
    g.build()
    import paper_2609_07577_gb300 as P
    P.lib()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("name", ["cfg1s", "cfg1", "cfg2s", "cfg3s"])
def test_coarsening_lockstep(name):
    hg = snngen.by_name(name)
    n = lockstep(hg, max_levels=40)
    assert n >= 1


def _partition_both(hg, budget=None, rows=None, **kw):
    from paper_2609_07577_gb300 import partition
    prm = oracle.params_of(hg, **kw)
    rho_o, cost_o, st_o, lv_o, rl_o = oracle.partition(hg, prm)
    from paper_2609_07577_gb300 import HGraph, params_for
    G = HGraph.from_hypergraph(hg, params=params_for(hg.omega, hg.delta, hg.phi, **kw))
    try:
        if budget is not None:
            G.set_level_budget(budget)
        if rows is not None:
            G.set_row_budget(rows)
        rho, cost, st = G.partition()
        rl = G.round_logs()
        lv = G.level_logs()
    finally:
        G.close()
    return (rho.cpu().numpy(), cost, st, lv, rl), (rho_o, cost_o, st_o, lv_o, rl_o)


@pytest.mark.parametrize("name,budget,rows", [
    ("cfg1s", None, None), ("cfg1", None, None), ("cfg2s", None, None), ("cfg3s", None, None),
    ("cfg1", 1, None), ("cfg3s", 1, None), ("cfg2s", 4 << 20, None),
    ("cfg1s", None, 0), ("cfg1", None, 0), ("cfg2s", None, 0), ("cfg3s", None, 0),
    ("cfg1", None, 1 << 20), ("cfg2s", None, 1 << 20), ("cfg3s", None, 4 << 20)])
def test_partition_parity(name, budget, rows):
    """budget=1 releases every intermediate level during coarsening, so
    uncoarsening rebuilds each one from level 0 through composed cid maps;
    4 MiB keeps a stride of them. rows=None refines every level of these
    sizes from connection rows, rows=0 from per-round histograms, and a few
    MiB switches from rows to histograms partway down the hierarchy."""
    hg = snngen.by_name(name)
    (rho, cost, st, lv, rl), (rho_o, cost_o, st_o, lv_o, rl_o) = _partition_both(hg, budget, rows)
    assert cost == cost_o
    assert np.array_equal(rho, rho_o)
    for k in ("levels", "n_parts", "nonempty_parts", "rounds", "moves", "cost_initial", "cost"):
        assert st[k] == st_o[k], k
    assert [(r["level"], r["round"], r["n_props"], r["istar"], r["gain"]) for r in rl] == \
           [(r["level"], r["round"], r["n_props"], r["istar"], r["gain"]) for r in rl_o]
    assert [(g["V"], g["E"], g["P"], g["n_cand"], g["n_pairs"]) for g in lv] == \
           [(g["V"], g["E"], g["P"], g["n_cand"], g["n_pairs"]) for g in lv_o]


def test_tiny_random_partitions():
    n = 0
    for seed in range(300):
        hg = snngen.tiny_random(90_000 + seed)
        try:
            rho_o, cost_o, st_o, lv_o, rl_o = oracle.partition(hg)
        except oracle.OracleError:
            continue
        (rho, cost, st, lv, rl), _ = _partition_both(hg)
        assert cost == cost_o, seed
        assert np.array_equal(rho, rho_o), seed
        n += 1
    assert n > 100


def test_level_cap_and_no_refinement():
    hg = snngen.by_name("cfg1s")
    (rho, cost, st, lv, rl), (rho_o, cost_o, st_o, lv_o, rl_o) = _partition_both(
        hg, max_levels=3, max_refine_rounds=0)
    assert st["levels"] == 3 == st_o["levels"]
    assert cost == cost_o and np.array_equal(rho, rho_o)
    (rho, cost, st, lv, rl), (rho_o, cost_o, st_o, lv_o, rl_o) = _partition_both(
        hg, max_levels=0, max_refine_rounds=3)
    assert cost == cost_o and np.array_equal(rho, rho_o)


def test_error_codes():
    from paper_2609_07577_gb300 import HGraph, SnnmapError, params_for
    import paper_2609_07577_gb300._native as N
    cases = [
        (hypergraph(3, [[0, 1, 1]], [1], 5, 5, 5), N.ERR_INVALID),
        (hypergraph(3, [[0, 1, 0]], [1], 5, 5, 5), N.ERR_INVALID),
        (hypergraph(3, [[0, 3]], [1], 5, 5, 5), N.ERR_INVALID),
        (hypergraph(3, [[0, 1]], [-1], 5, 5, 5), N.ERR_INVALID),
        (hypergraph(3, [[0, 2], [1, 2]], [1, 1], 5, 1, 5), N.ERR_INFEASIBLE),
    ]
    for hg, code in cases:
        with pytest.raises(SnnmapError) as e:
            HGraph.from_hypergraph(hg)
        assert e.value.code == code
    hg = hypergraph(3, [[0, 1]], [1], 5, 5, 5)
    off = torch.tensor(hg.off)  # host memory: rejected, not dereferenced
    with pytest.raises(SnnmapError) as e:
        HGraph(params_for(5, 5, 5), 3, off, torch.tensor(hg.pins), torch.tensor(hg.w))
    assert e.value.code == N.ERR_INVALID


def test_empty_and_degenerate():
    from paper_2609_07577_gb300 import partition
    # no hyperedges: every neuron its own partition
    hg = hypergraph(5, [], [], 3, 3, 3)
    rho, cost, st = partition(hg)
    assert cost == 0 and st["n_parts"] == 5 and list(rho) == [0, 1, 2, 3, 4]
    # hyperedges without destinations are dropped
    hg = hypergraph(4, [[0], [1, 2], [3]], [5, 1, 7], 4, 4, 4)
    rho_o, cost_o, *_ = oracle.partition(hg)
    rho, cost, st = partition(hg)
    assert cost == cost_o and np.array_equal(rho, rho_o)
    # a star: one pair per level until the level cap
    hg = hypergraph(40, [list(range(40))], [3], 40, 100, 100)
    rho_o, cost_o, st_o, *_ = oracle.partition(hg)
    rho, cost, st = partition(hg)
    assert cost == cost_o == 0 and np.array_equal(rho, rho_o)
    assert st["levels"] == st_o["levels"]


def test_connectivity_entry_point():
    """S12 as its own call: Conn of arbitrary partitions equals the oracle's."""
    from paper_2609_07577_gb300 import HGraph, SnnmapError, snnmap_connectivity
    import paper_2609_07577_gb300._native as N
    rng = np.random.default_rng(5)
    for name in ("cfg1s", "cfg3s"):
        hg = snngen.by_name(name)
        L = oracle.Level.from_hypergraph(hg)
        G = HGraph.from_hypergraph(hg)
        try:
            for K in (1, 7, 300, hg.V):
                rho = rng.integers(0, K, size=hg.V).astype(np.int32)
                got = snnmap_connectivity(G.handle, K, torch.from_numpy(rho).cuda())
                assert got == L.conn(rho), (name, K)
            bad = torch.full((hg.V,), 5, dtype=torch.int32, device="cuda")
            with pytest.raises(SnnmapError) as e:
                snnmap_connectivity(G.handle, 5, bad)
            assert e.value.code == N.ERR_INVALID
        finally:
            G.close()


def test_rebuilt_levels_equal_oracle_levels():
    """Levels released under a tiny memory budget and rebuilt on demand equal
    the oracle's levels (arrays compared canonically)."""
    from gpu_helpers import assert_level_equal
    from paper_2609_07577_gb300 import HGraph
    hg = snngen.by_name("cfg3s")
    prm = oracle.params_of(hg)
    G = HGraph.from_hypergraph(hg)
    try:
        G.set_level_budget(1)
        L = oracle.Level.from_hypergraph(hg, prm)
        olevels = [L]
        for _ in range(12):
            nc, npairs = G.coarsen_level()
            if npairs == 0:
                break
            G.contract()
            cand, cs, cov = olevels[-1].affinity(prm)
            m, _ = oracle.match(cand, cs)
            C, _ = olevels[-1].contract(m, cand, cov)
            olevels.append(C)
        assert len(olevels) > 5
        for lev in (3, 1, len(olevels) - 2, 2):
            assert_level_equal(G.level_arrays(lev), olevels[lev].arrays(), f"rebuilt level {lev}")
    finally:
        G.close()


@pytest.mark.parametrize("name,rows", [("cfg1s", None), ("cfg2s", None), ("cfg3s", None),
                                       ("cfg1s", 0), ("cfg2s", 0), ("cfg3s", 0)])
def test_partition_parity_nonpositive_variant(name, rows):
    """Reading R19: every vertex proposes its best feasible adjacent move
    whatever its gain; same partition, cost, stats and round logs as the
    oracle, on connection rows (rows=None) and on histograms (rows=0)."""
    hg = snngen.by_name(name)
    (rho, cost, st, lv, rl), (rho_o, cost_o, st_o, lv_o, rl_o) = _partition_both(
        hg, None, rows, refine_nonpositive=1)
    assert cost == cost_o
    assert np.array_equal(rho, rho_o)
    for k in ("levels", "n_parts", "nonempty_parts", "rounds", "moves", "cost_initial", "cost"):
        assert st[k] == st_o[k], k
    assert [(r["level"], r["round"], r["n_props"], r["istar"], r["gain"]) for r in rl] == \
        [(r["level"], r["round"], r["n_props"], r["istar"], r["gain"]) for r in rl_o]


def test_tiny_random_nonpositive_variant():
    from paper_2609_07577_gb300 import partition
    n = 0
    for seed in range(120):
        hg = snngen.tiny_random(50_000 + seed)
        prm = oracle.params_of(hg, refine_nonpositive=1)
        try:
            rho_o, cost_o, *_ = oracle.partition(hg, prm)
        except oracle.OracleError:
            continue
        rho, cost, st = partition(hg, refine_nonpositive=1)
        assert cost == cost_o, seed
        assert np.array_equal(rho, rho_o), seed
        n += 1
    assert n > 40
