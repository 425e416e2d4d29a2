"""The partition hypergraph G_P (Sec. 3, Partitioning Definition; reading
R18) computed by the oracle, pinned by a hand-worked example, by a
set-based restatement on the original axons, and by two identities:
sum(eta) + internal = sum(omega), and Conn(rho) = sum over A of
eta(a) * |dst(a)| (an axon's lambda - 1 is the number of destination
partitions left once its source's partition is discarded)."""
import json
import os

import numpy as np
import pytest

import oracle
import snngen
from bruteforce import conn as bf_conn, hedges
from helpers import hypergraph

HERE = os.path.dirname(os.path.abspath(__file__))


def gp_bruteforce(hg, rho):
    """A = {(rho(src), {rho(d)} - {rho(src)})}, eta summed, axons counted;
    canonical order (source, size, destinations)."""
    groups, internal = {}, 0
    for s, d, w in hedges(hg):
        if not d:
            continue                      # not an axon of the hypergraph
        src = int(rho[s])
        dst = tuple(sorted({int(rho[x]) for x in d} - {src}))
        if not dst:
            internal += w
            continue
        g = groups.setdefault((src, dst), [0, 0])
        g[0] += w
        g[1] += 1
    keys = sorted(groups, key=lambda k: (k[0], len(k[1]), k[1]))
    return [((k[0],) + k[1], groups[k][0], groups[k][1]) for k in keys], internal


def gp_list(g):
    out = []
    for i in range(len(g["eta"])):
        p = g["pins"][g["off"][i]:g["off"][i + 1]].tolist()
        out.append((tuple(p), int(g["eta"][i]), int(g["axons"][i])))
    return out


def test_golden_example():
    with open(os.path.join(HERE, "golden", "gp_example.json")) as f:
        ex = json.load(f)
    hg = hypergraph(ex["V"], ex["hedges"], ex["w"], omega=5, delta=10, phi=10)
    L = oracle.Level.from_hypergraph(hg, oracle.params_of(hg))
    g = L.partition_graph(ex["rho"])
    assert gp_list(g) == [(tuple(p), eta, ax) for p, eta, ax in ex["gp"]]
    assert g["internal"] == ex["internal"]
    assert L.conn(ex["rho"]) == ex["conn"]


@pytest.mark.parametrize("chunk", range(4))
def test_matches_bruteforce_and_identities(chunk):
    for seed in range(chunk * 150, (chunk + 1) * 150):
        hg = snngen.tiny_random(seed)
        rng = np.random.Generator(np.random.PCG64(7000 + seed))
        K = int(rng.integers(1, hg.V + 1))
        rho = rng.integers(0, K, size=hg.V).astype(np.int32)
        # G_P does not depend on the limits: none binding
        L = oracle.Level.from_hypergraph(hg, oracle.params(10**6, 10**9, 10**9))
        g = L.partition_graph(rho)
        want, internal = gp_bruteforce(hg, rho)
        assert gp_list(g) == want, seed
        assert g["internal"] == internal, seed
        wsum = sum(w for s, d, w in hedges(hg) if d)
        assert int(g["eta"].sum()) + g["internal"] == wsum
        ndst = np.diff(g["off"]) - 1
        assert int((g["eta"] * ndst).sum()) == bf_conn(hg, rho) == L.conn(rho)


def test_identity_and_single_partition():
    hg = snngen.by_name("cfg1s")
    L = oracle.Level.from_hypergraph(hg, oracle.params_of(hg))
    ident = np.arange(hg.V, dtype=np.int32)
    g = L.partition_graph(ident)
    assert g["internal"] == 0
    assert len(g["eta"]) == L.dims()[1]          # every axon distinct already
    one = np.zeros(hg.V, np.int32)
    g1 = L.partition_graph(one)
    assert len(g1["eta"]) == 0 and g1["internal"] == int(hg.w.sum())
