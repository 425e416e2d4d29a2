"""Helpers for GPU parity tests: drive the oracle and the CUDA library level
by level on the same seeded input and compare what must be equal."""
import numpy as np

import oracle
from helpers import canonical_hedges


def assert_level_equal(ga, oa, tag=""):
    for key in ("size", "inpins", "in_count", "in_internal"):
        assert np.array_equal(ga[key], oa[key]), f"{tag} {key}"
    assert ga["V"] == oa["V"] and ga["E"] == oa["E"] and ga["P"] == oa["P"], tag
    cg = canonical_hedges(ga["off"], ga["pins"], ga["w"], ga["k"], ga["selfdst"])
    co = canonical_hedges(oa["off"], oa["pins"], oa["w"], oa["k"], oa["selfdst"])
    assert cg == co, f"{tag} hyperedges"


def lockstep(hg, max_levels=None, check_levels=True, setup=None, logs=None):
    """Runs coarsening on both sides; returns the number of levels compared.
    setup(G) runs on the CUDA handle first; logs (a list) receives its level
    logs."""
    from paper_2609_07577_gb300 import HGraph
    prm = oracle.params_of(hg)
    L = oracle.Level.from_hypergraph(hg, prm)
    G = HGraph.from_hypergraph(hg)
    if setup is not None:
        setup(G)
    try:
        lev = 0
        while True:
            if check_levels:
                assert_level_equal(G.level_arrays(lev), L.arrays(), f"level {lev}")
            cand, cs, cov = L.affinity(prm)
            nc, npairs = G.coarsen_level()
            assert nc == int((cand >= 0).sum()), f"level {lev} n_cand"
            if nc == 0:
                break
            gcand, gcs, gcov, gmatch = G.last_matching()
            assert np.array_equal(gcand, cand), f"level {lev} cand"
            assert np.array_equal(gcs, cs), f"level {lev} cscore"
            assert np.array_equal(gcov, cov), f"level {lev} cov"
            m, pairs = oracle.match(cand, cs)
            assert np.array_equal(gmatch, m), f"level {lev} match"
            assert npairs == pairs
            L, cid = L.contract(m, cand, cov)
            G.contract()
            assert np.array_equal(G.level_cid(lev), cid), f"level {lev} cid"
            lev += 1
            if max_levels is not None and lev >= max_levels:
                if check_levels:
                    assert_level_equal(G.level_arrays(lev), L.arrays(), f"level {lev}")
                break
        if logs is not None:
            logs.extend(G.level_logs())
        return lev
    finally:
        G.close()
