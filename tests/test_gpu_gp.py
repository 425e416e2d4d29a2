"""G_P (Sec. 3, Partitioning Definition) on the GPU against the oracle:
hyperedges compared in canonical order, eta, merged axon counts and the
internal weight, for partitions found by the pass and for random ones;
error codes."""
import numpy as np
import pytest
import torch

import oracle
import snngen

pytestmark = pytest.mark.gpu


def canonical(g):
    rows = []
    for i in range(len(g["eta"])):
        p = g["pins"][g["off"][i]:g["off"][i + 1]].tolist()
        rows.append((p[0], len(p), tuple(p[1:]), int(g["eta"][i]), int(g["axons"][i])))
    return sorted(rows)


def check(hg, rho, K):
    from paper_2609_07577_gb300 import HGraph, params_for
    G = HGraph.from_hypergraph(hg, params=params_for(10**6, 10**9, 10**9))
    try:
        g = G.partition_graph(torch.from_numpy(np.asarray(rho, np.int32)).cuda(), K)
    finally:
        G.close()
    L = oracle.Level.from_hypergraph(hg, oracle.params(10**6, 10**9, 10**9))
    o = L.partition_graph(rho)
    assert canonical(g) == canonical(o)
    assert g["internal"] == o["internal"]
    # destinations ascending after the source, no destination equal to it
    for i in range(len(g["eta"])):
        p = g["pins"][g["off"][i]:g["off"][i + 1]]
        assert len(p) >= 2 and (np.diff(p[1:]) > 0).all() and p[0] not in p[1:]


@pytest.mark.parametrize("name", ["cfg1s", "cfg2s", "cfg3s"])
def test_gp_of_the_pass(name):
    from paper_2609_07577_gb300 import HGraph
    hg = snngen.by_name(name)
    G = HGraph.from_hypergraph(hg)
    try:
        rho, cost, st = G.partition()
        g = G.partition_graph(rho, st["n_parts"])
    finally:
        G.close()
    rho = rho.cpu().numpy()
    L = oracle.Level.from_hypergraph(hg, oracle.params_of(hg))
    o = L.partition_graph(rho)
    assert canonical(g) == canonical(o)
    assert g["internal"] == o["internal"]
    ndst = np.diff(g["off"]) - 1
    assert int((g["eta"] * ndst).sum()) == cost


@pytest.mark.parametrize("K", [1, 2, 7, 64, 4096, 1 << 14])
def test_gp_random_partitions(K):
    hg = snngen.by_name("cfg3s")
    rng = np.random.Generator(np.random.PCG64(K))
    check(hg, rng.integers(0, K, size=hg.V).astype(np.int32), K)


def test_gp_tiny_and_errors():
    from paper_2609_07577_gb300 import HGraph, params_for, SnnmapError
    for seed in range(40):
        hg = snngen.tiny_random(seed)
        rng = np.random.Generator(np.random.PCG64(100 + seed))
        K = int(rng.integers(1, hg.V + 1))
        check(hg, rng.integers(0, K, size=hg.V).astype(np.int32), K)
    hg = snngen.tiny_random(3)
    G = HGraph.from_hypergraph(hg, params=params_for(10**6, 10**9, 10**9))
    try:
        bad = torch.full((hg.V,), 5, dtype=torch.int32, device="cuda")
        with pytest.raises(SnnmapError) as ei:
            G.partition_graph(bad, 5)
        assert ei.value.code == 1
        import paper_2609_07577_gb300 as P
        with pytest.raises(SnnmapError) as ei:
            P.snnmap_partition_graph_copy(G.handle)     # nothing computed yet
        assert ei.value.code == 6
    finally:
        G.close()
