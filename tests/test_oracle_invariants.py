"""Oracle invariants on generated workloads (scaled-down generators).

Checks what Sec. 4.1 states or implies at any size: every super-node within
Omega/Phi/Delta at every level ("all constraints are enforced on every
super-node"), conservation of neurons, inbound pins and axons through
contraction, in_count equal to its recomputed value, the pseudo-forest
property of the candidate graph, Conn unchanged by projection, and
refinement never increasing Conn.
"""
import numpy as np
import pytest

import oracle
import snngen

NAMES = ["cfg1s", "cfg1", "cfg2s"]


def conn_np(off, pins, w, rho):
    """Eq. connectivity with numpy: distinct partitions per hyperedge."""
    E = len(off) - 1
    hid = np.repeat(np.arange(E, dtype=np.int64), np.diff(off))
    K = int(rho.max()) + 1
    key = np.unique(hid * K + rho[pins].astype(np.int64))
    lam = np.bincount(key // K, minlength=E)
    return int((w.astype(np.int64) * (lam - 1)).sum())


def recompute_in_count(a):
    V = a["V"]
    out = a["in_internal"].astype(np.int64).copy()
    off, pins = a["off"], a["pins"]
    for e in range(a["E"]):
        p = pins[off[e]:off[e + 1]]
        out[p[1:]] += a["k"][e]
        if a["selfdst"][e]:
            out[p[0]] += a["k"][e]
    return out[:V]


@pytest.mark.parametrize("name", NAMES)
def test_level_invariants(name):
    hg = snngen.by_name(name)
    prm = oracle.params_of(hg)
    L = oracle.Level.from_hypergraph(hg, prm)
    a0 = L.arrays()
    V0, E0 = a0["V"], a0["E"]
    total_inpins = int(a0["inpins"].sum())
    total_w = int(a0["w"].sum())
    img = np.arange(V0)
    hid0 = np.repeat(np.arange(E0), np.diff(a0["off"]))
    levels = 0
    while True:
        a = L.arrays()
        assert (a["size"] <= prm.omega).all()
        assert (a["inpins"] <= prm.phi).all()
        assert (a["in_count"] <= prm.delta).all()
        assert int(a["size"].sum()) == V0
        assert int(a["inpins"].sum()) == total_inpins
        assert int(a["k"].sum()) + int(a["in_internal"].sum()) == E0
        assert (recompute_in_count(a) == a["in_count"]).all()
        # axons whose image collapsed into one super-node carry the missing weight
        pimg = img[a0["pins"]]
        lo = np.minimum.reduceat(pimg, a0["off"][:-1])
        hi = np.maximum.reduceat(pimg, a0["off"][:-1])
        dropped_w = int(a0["w"][lo == hi].sum())
        assert int(a["w"].sum()) + dropped_w == total_w
        cand, cs, cov = L.affinity(prm)
        has = cand >= 0
        if not has.any():
            break
        # pseudo-forest: scores non-decreasing along arcs, only 2-cycles
        assert (cs[has] <= cs[cand[has]]).all()
        two = has & (cand[np.where(has, cand, 0)] == np.arange(a["V"]))
        m, pairs = oracle.match(cand, cs)
        assert pairs >= 1
        mm = m >= 0
        idx = np.nonzero(mm)[0]
        assert (m[m[idx]] == idx).all()
        assert ((cand[idx] == m[idx]) | (cand[m[idx]] == idx)).all()
        assert (m[two] == cand[two]).all()
        L, cid = L.contract(m, cand, cov)
        img = cid[img]
        levels += 1
    assert levels >= 1


@pytest.mark.parametrize("name", NAMES)
def test_pass_conn_and_monotone(name):
    hg = snngen.by_name(name)
    rho, cost, st, levels, rounds = oracle.partition(hg)
    assert cost == conn_np(hg.off, hg.pins, hg.w, rho)
    assert all(r["gain"] > 0 for r in rounds if r["istar"] > 0)
    assert all(r["gain"] == 0 for r in rounds if r["istar"] == 0)
    assert st["cost_initial"] - sum(r["gain"] for r in rounds) == cost
    assert st["moves"] == sum(r["istar"] for r in rounds)
    # feasible partition
    prm = oracle.params_of(hg)
    L = oracle.Level.from_hypergraph(hg, prm)
    a = L.arrays()
    K = int(rho.max()) + 1
    assert (np.bincount(rho, weights=a["size"], minlength=K) <= prm.omega).all()
    assert (np.bincount(rho, weights=a["inpins"], minlength=K) <= prm.phi).all()
    # distinct inbound axons per partition
    off, pins = a["off"], a["pins"]
    hid = np.repeat(np.arange(a["E"], dtype=np.int64), np.diff(off))
    isdst = np.ones(len(pins), bool)
    isdst[off[:-1]] = False
    key = np.unique(rho[pins[isdst]].astype(np.int64) * a["E"] + hid[isdst])
    assert (np.bincount(key // a["E"], minlength=K) <= prm.delta).all()


def test_projection_keeps_conn():
    hg = snngen.by_name("cfg1s")
    prm = oracle.params_of(hg, max_refine_rounds=0)
    rho, cost, st, levels, rounds = oracle.partition(hg, prm)
    assert cost == st["cost_initial"]
