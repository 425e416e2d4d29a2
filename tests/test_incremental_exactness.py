"""The facts the CUDA path's incremental shortcuts rest on, checked by brute
force on every level of the oracle's own hierarchies (CPU only).

After a contraction the CUDA path does not recompute everything: it carries
each vertex's candidate over (only new super-nodes are histogrammed in
full), derives a super-node's distinct inbound-axon count from its members,
and keeps the connection rows of unmatched vertices. Each shortcut is exact
by a property of Eq. neigh_histogram, Eq. matching and the contraction of
Sec. 4.1:

1. For two vertices neither of which merged, score and shared inbound count
   of the pair are unchanged by the contraction.
2. Hence an unmatched vertex's next candidate is its old candidate's image if
   that did not merge (KEEP) or, failing that, the best valid new super-node;
   with no old candidate (NONE) only a new super-node can be one; if the old
   candidate merged into w (MERGED) and w is a valid partner, the best valid
   new super-node is the candidate. (Under Eq. matching a vertex that is
   some vertex's candidate is always matched, so KEEP does not arise after a
   matching; the test asserts that too.)
3. A pair's super-node has in_count(n) + in_count(m) - shared(n, m), the
   shared count being the candidate overlap of the member whose candidate is
   the other (pairs are matched along candidate arcs).
4. A hyperedge holding no merged vertex keeps its size, weight, multiplicity
   and roles, and no other hyperedge becomes equal to it.
5. The connection row of an unmatched vertex (conn and inbound overlap per
   partition) is the same on both levels under the projected partition.

The scores, overlaps, limits and rows below are recomputed from the original
neurons and axons (tests/bruteforce.py) or from a level's arrays, never taken
from the oracle's candidate arithmetic; the oracle supplies the hierarchy
(its matchings and contractions) and the candidates that are compared.
"""
import numpy as np
import pytest

import bruteforce as bf
import oracle
import snngen


def _inputs():
    out = [snngen.tiny_random(900 + s, V=int(18 + (s * 7) % 23), E=int(30 + (s * 11) % 50))
           for s in range(40)]
    out += [snngen.conv(3, 4, 2, 1, seed=s, omega=8, delta=64, phi=400, name=f"conv{s}")
            for s in range(6)]
    out += [snngen.powerlaw(96, block=32, fmin=2, fmax=24, seed=s, omega=8, delta=40, phi=120,
                            name=f"pl{s}") for s in range(6)]
    return out


def _hierarchy(hg, prm, max_levels=64):
    """The oracle's levels, each with its candidates, matching, cid map and
    the image of every original neuron."""
    try:
        L = oracle.Level.from_hypergraph(hg, prm)
    except oracle.OracleError:
        return []
    img = np.arange(hg.V)
    out = []
    for _ in range(max_levels):
        cand, cscore, cov = L.affinity(prm)
        match, pairs = oracle.match(cand, cscore)
        if pairs == 0:
            break
        L2, cid = L.contract(match, cand, cov)
        out.append({"L": L, "img": img, "cand": cand, "cscore": cscore, "cov": cov,
                    "match": match, "cid": cid, "L2": L2, "img2": cid[img]})
        img = cid[img]
        L = L2
    return out


def _members(img, V):
    mem = [set() for _ in range(V)]
    for q, x in enumerate(img.tolist()):
        mem[x].add(q)
    return mem


CASES = [(hg, oracle.params_of(hg)) for hg in _inputs()]


@pytest.mark.parametrize("k", range(len(CASES)))
def test_pair_scores_survive_contraction(k):
    hg, prm = CASES[k]
    for lv in _hierarchy(hg, prm):
        sc0, ov0 = bf.score_ov(hg, lv["img"])
        sc1, ov1 = bf.score_ov(hg, lv["img2"])
        cid, match = lv["cid"], lv["match"]
        un = set(np.flatnonzero(match < 0).tolist())
        back = {int(cid[u]): u for u in un}
        for src, dst in ((sc0, sc1), (ov0, ov1)):
            for (u, v), s in src.items():
                if u in un and v in un:
                    assert dst.get((int(cid[u]), int(cid[v]))) == s
            for (x, y), s in dst.items():
                if x in back and y in back:
                    assert src.get((back[x], back[y])) == s


@pytest.mark.parametrize("k", range(len(CASES)))
def test_carried_candidates(k):
    hg, prm = CASES[k]
    ins = bf.in_sets(hg)
    lvs = _hierarchy(hg, prm)
    checked = 0
    for i, lv in enumerate(lvs):
        L2 = lv["L2"]
        cand1 = lvs[i + 1]["cand"] if i + 1 < len(lvs) else L2.affinity(prm)[0]
        cscore1 = lvs[i + 1]["cscore"] if i + 1 < len(lvs) else L2.affinity(prm)[1]
        V2 = L2.dims()[0]
        mem1 = _members(lv["img2"], V2)
        sc1, _ = bf.score_ov(hg, lv["img2"])
        cid, match, cand = lv["cid"], lv["match"], lv["cand"]
        new = {int(cid[n]) for n in np.flatnonzero(match >= 0)}

        def valid(x, y):
            return bf.group_ok(hg, mem1[x] | mem1[y], prm, ins)

        def best(x, ys):
            top = None
            for y in ys:
                if (x, y) in sc1 and valid(x, y):
                    key = (sc1[(x, y)], -y)
                    if top is None or key > top:
                        top = key
            return (-top[1], top[0]) if top else (-1, 0)

        for n in np.flatnonzero(match < 0).tolist():
            x = int(cid[n])
            c = int(cand[n])
            bn, bs = best(x, new)
            if c < 0:                                  # NONE
                want = (bn, bs)
            elif match[c] < 0:                         # KEEP
                raise AssertionError(f"candidate {c} of {n} left unmatched")
            else:                                      # MERGED
                w = int(cid[c])
                if not valid(x, w):
                    continue                           # a full histogram decides
                want = (bn, bs)
            assert (int(cand1[x]), int(cscore1[x]) if cand1[x] >= 0 else 0) == want, (i, n)
            checked += 1
    if lvs:
        assert checked > 0


@pytest.mark.parametrize("k", range(len(CASES)))
def test_in_count_of_pairs(k):
    hg, prm = CASES[k]
    for lv in _hierarchy(hg, prm):
        a0, a1 = lv["L"].arrays(), lv["L2"].arrays()
        cid, match, cand, cov = lv["cid"], lv["match"], lv["cand"], lv["cov"]
        for n in range(a0["V"]):
            m = int(match[n])
            if m < 0:
                assert a1["in_count"][cid[n]] == a0["in_count"][n]
            elif n < m:
                assert cand[n] == m or cand[m] == n      # matched along a candidate arc
                ov = cov[n] if cand[n] == m else cov[m]
                assert a1["in_count"][cid[n]] == a0["in_count"][n] + a0["in_count"][m] - ov


def _hedge_list(a):
    out = []
    for e in range(a["E"]):
        p = a["pins"][a["off"][e]:a["off"][e + 1]]
        out.append((int(p[0]), int(a["selfdst"][e]), tuple(sorted(p[1:].tolist())),
                    int(a["w"][e]), int(a["k"][e])))
    return out


@pytest.mark.parametrize("k", range(len(CASES)))
def test_untouched_hyperedges_pass_through(k):
    hg, prm = CASES[k]
    for lv in _hierarchy(hg, prm):
        a0, a1 = lv["L"].arrays(), lv["L2"].arrays()
        cid, merged = lv["cid"], lv["match"] >= 0
        coarse = {}
        for s, sd, D, w, kk in _hedge_list(a1):
            assert (s, sd, D) not in coarse                # the coarse level has no duplicates
            coarse[(s, sd, D)] = (w, kk)
        untouched = 0
        for s, sd, D, w, kk in _hedge_list(a0):
            if merged[s] or any(merged[q] for q in D):
                continue
            untouched += 1
            key = (int(cid[s]), sd, tuple(sorted(int(cid[q]) for q in D)))
            assert len(key[2]) == len(D)                 # same size
            assert coarse.get(key) == (w, kk)            # same weight and multiplicity, alone
        # every other coarse hyperedge holds a new super-node
        new = {int(cid[n]) for n in np.flatnonzero(merged)}
        touched_images = sum(1 for (s, sd, D) in coarse if s in new or new & set(D))
        assert untouched + touched_images == len(coarse)


def _rows(a, rho):
    """conn(n, p) = sum of w(e) over incident e with a pin in p, and the
    inbound overlap O(n, p) = sum of k(e) over e in which n is a destination
    and some destination lies in p (a level's destinations: its pins after
    the first, and the source when selfdst is set)."""
    conn, ovl = {}, {}
    for s, sd, D, w, kk in _hedge_list(a):
        pins = (s,) + D
        parts = {int(rho[q]) for q in pins}
        dsts = D + ((s,) if sd else ())
        dparts = {int(rho[q]) for q in dsts}
        for n in pins:
            for p in parts:
                conn[(n, p)] = conn.get((n, p), 0) + w
        for n in dsts:
            for p in dparts:
                ovl[(n, p)] = ovl.get((n, p), 0) + kk
    return conn, ovl


@pytest.mark.parametrize("k", range(len(CASES)))
def test_rows_of_unmatched_vertices_survive_projection(k):
    hg, prm = CASES[k]
    rng = np.random.Generator(np.random.PCG64(k))
    for lv in _hierarchy(hg, prm):
        a0, a1 = lv["L"].arrays(), lv["L2"].arrays()
        cid, match = lv["cid"], lv["match"]
        rho1 = rng.integers(0, max(1, min(a1["V"], 5)), size=a1["V"])
        rho0 = rho1[cid]
        c0, o0 = _rows(a0, rho0)
        c1, o1 = _rows(a1, rho1)
        for n in np.flatnonzero(match < 0).tolist():
            x = int(cid[n])
            for p in range(int(rho1.max()) + 1 if a1["V"] else 0):
                assert c0.get((n, p), 0) == c1.get((x, p), 0)
                assert o0.get((n, p), 0) == o1.get((x, p), 0)


# ---------------------------------------------------------------------------
# 6. Proposal update after an enacted prefix (refinement rounds after a
#    level's first). Moves between the partitions of P* (the sources and
#    targets of the enacted moves) change no other partition's contents, so
#    for a vertex n that did not move, a partition q outside P* keeps its
#    feasibility for n and conn(n, q), and the gain of every move of n to a
#    partition outside P* shifts by the same amount, the change of save(n)
#    (gain = conn(n, q) - W(n) + save(n)). So n's best move after the round
#    lies in {its previous proposal} + P*, unless n moved, its previous
#    proposal pointed into P*, or it had none and its save grew.


def _proposals(hg, rho, K, prm):
    """Best feasible move of every vertex on the original neurons: gain as
    the Conn it removes, ties to the lower partition; (-1, 0) if no move has
    a positive gain."""
    ins = bf.in_sets(hg)
    axons = [({s} | d) for s, d, w in bf.hedges(hg) if d]
    base = bf.conn(hg, rho)
    members = {}
    for n in range(hg.V):
        members.setdefault(int(rho[n]), set()).add(n)
    out = []
    for n in range(hg.V):
        adj = {int(rho[q]) for e in axons if n in e for q in e}
        best = None
        for p in sorted(adj):
            if p == rho[n] or not bf.group_ok(hg, members.get(p, set()) | {n}, prm, ins):
                continue
            r2 = list(rho)
            r2[n] = p
            g = base - bf.conn(hg, r2)
            if best is None or (g, -p) > best:
                best = (g, -p)
        out.append((-best[1], best[0]) if best is not None and best[0] > 0 else (-1, 0))
    return out


def _gain(hg, rho, n, p):
    r2 = list(rho)
    r2[n] = p
    return bf.conn(hg, rho) - bf.conn(hg, r2)


def _save(hg, rho, n):
    """Summed weight of n's axons in which n is the only neuron of its partition."""
    t = 0
    for s, d, w in bf.hedges(hg):
        if not d:
            continue
        e = {s} | d
        if n in e and sum(1 for q in e if rho[q] == rho[n]) == 1:
            t += w
    return t


@pytest.mark.parametrize("seed", range(60))
def test_proposal_update_after_prefix(seed):
    hg = snngen.tiny_random(5000 + seed, V=int(8 + seed % 9), E=int(10 + seed % 17))
    ins = bf.in_sets(hg)
    # limits every neuron meets alone, tight enough that some moves are refused
    top = max(len(x) for x in ins)
    prm = oracle.params(2 + seed % 3, top + seed % 4, 2 * top + seed % 7)
    assert all(bf.group_ok(hg, {n}, prm, ins) for n in range(hg.V))
    rho = list(range(hg.V))
    K = hg.V
    img = np.arange(hg.V)
    props = _proposals(hg, rho, K, prm)
    checked = 0
    for _ in range(6):
        rho1, n_props, istar, gain = bf.refine_round(hg, img, hg.V, rho, K, prm)
        if istar == 0:
            break
        moved = {n for n in range(hg.V) if rho1[n] != rho[n]}
        pstar = {rho[n] for n in moved} | {rho1[n] for n in moved}
        props1 = _proposals(hg, rho1, K, prm)
        for n in range(hg.V):
            pto, g0 = props[n]
            dsave = _save(hg, rho1, n) - _save(hg, rho, n)
            if n in moved or pto in pstar or (pto < 0 and dsave > 0):
                continue                                # rescanned in full
            if pto >= 0:
                assert _gain(hg, rho1, n, pto) == g0 + dsave
            # the best of {previous proposal} + P*, positive gains only
            best = None
            for p in sorted(pstar | ({pto} if pto >= 0 else set())):
                if p == rho1[n]:
                    continue
                if not any(rho1[q] == p for s, d, w in bf.hedges(hg) if d
                           for e in [{s} | d] if n in e for q in e):
                    continue                            # not adjacent
                grp = {q for q in range(hg.V) if rho1[q] == p} | {n}
                if not bf.group_ok(hg, grp, prm, ins):
                    continue
                g = _gain(hg, rho1, n, p)
                if best is None or (g, -p) > best:
                    best = (g, -p)
            want = (-best[1], best[0]) if best is not None and best[0] > 0 else (-1, 0)
            assert props1[n] == want, (n, props[n], props1[n], want, sorted(pstar))
            checked += 1
        rho, props = rho1, props1
