"""Brute-force restatements of the paper's definitions, for tiny hypergraphs.

These pin the oracle to the mathematics: every function here works on the
ORIGINAL neurons and axons (Sec. 2) with Python sets, and shares no code and
no formulation shortcut with the oracle. A super-node is just its set of
member neurons; a partition of level-l vertices is judged by the neurons it
holds.

* Conn            - Eq. connectivity, from the distinct partitions of each axon.
* constraints     - Sec. 3: |p| <= Omega, |union in(n)| <= Delta,
                    sum |in(n)| <= Phi, evaluated on member neurons.
* score / overlap - Eq. neigh_histogram: summed weight of axons that touch both
                    super-nodes; |in(n) & in(m)| on original axons.
* matching        - the recursive characterisation of Eq. matching, memoised.
* refinement      - a move's gain is the Conn it removes; a prefix's updated
                    gains are Conn differences after each move; validity is a
                    direct constraint check of every partition.
"""
from __future__ import annotations

import functools
import itertools

import numpy as np


def hedges(hg):
    """Original axons as (src, frozenset(dsts), weight); axons with no
    destination never reach the partitioner's objective or limits."""
    out = []
    for a in range(hg.E):
        p = hg.pins[hg.off[a]:hg.off[a + 1]].tolist()
        out.append((p[0], frozenset(p[1:]), int(hg.w[a])))
    return out


def in_sets(hg):
    """in(n): axons having n as a destination (Sec. 2)."""
    ins = [set() for _ in range(hg.V)]
    for a, (s, d, w) in enumerate(hedges(hg)):
        for q in d:
            ins[q].add(a)
    return ins


def conn(hg, rho0):
    """Eq. connectivity on the original hypergraph."""
    tot = 0
    for s, d, w in hedges(hg):
        parts = {int(rho0[s])} | {int(rho0[q]) for q in d}
        tot += w * (len(parts) - 1)
    return tot


def group_ok(hg, neurons, prm, ins=None):
    """Sec. 3 limits for one core holding ``neurons``."""
    ins = ins if ins is not None else in_sets(hg)
    if len(neurons) > prm.omega:
        return False
    if sum(len(ins[q]) for q in neurons) > prm.phi:
        return False
    u = set()
    for q in neurons:
        u |= ins[q]
    return len(u) <= prm.delta


def feasible(hg, rho0, prm):
    ins = in_sets(hg)
    groups = {}
    for n in range(hg.V):
        groups.setdefault(int(rho0[n]), []).append(n)
    return all(group_ok(hg, g, prm, ins) for g in groups.values())


def members(cid_chain, V0):
    """Level-l vertex -> set of original neurons, from cid maps 0..l-1."""
    img = np.arange(V0)
    for cid in cid_chain:
        img = np.asarray(cid)[img]
    VL = int(img.max()) + 1 if V0 else 0
    mem = [set() for _ in range(VL)]
    for q in range(V0):
        mem[int(img[q])].add(q)
    return img, mem


def level_state(hg, img, mem):
    """size, inpins, in_count, in_internal of each super-node, from members."""
    ins = in_sets(hg)
    size = [len(m) for m in mem]
    inpins = [sum(len(ins[q]) for q in m) for m in mem]
    in_count = []
    for m in mem:
        u = set()
        for q in m:
            u |= ins[q]
        in_count.append(len(u))
    internal = [0] * len(mem)
    for s, d, w in hedges(hg):
        if not d:
            continue
        pins = {int(img[s])} | {int(img[q]) for q in d}
        if len(pins) == 1:
            internal[int(img[s])] += 1
    return size, inpins, in_count, internal


def coarse_hedges(hg, img):
    """Coarse hyperedges as sorted (s, selfdst, D, w, k) from the images of
    the original axons that still span two super-nodes."""
    groups = {}
    for s, d, w in hedges(hg):
        if not d:
            continue
        s2 = int(img[s])
        dimg = {int(img[q]) for q in d}
        D = tuple(sorted(dimg - {s2}))
        if not D:
            continue
        key = (s2, int(s2 in dimg), D)
        g = groups.setdefault(key, [0, 0])
        g[0] += w
        g[1] += 1
    return sorted((k[0], k[1], k[2], v[0], v[1]) for k, v in groups.items())


def score_ov(hg, img):
    """score(n, m) and |in(n) & in(m)| for every ordered pair of distinct
    super-nodes that share an axon."""
    sc, ov = {}, {}
    for s, d, w in hedges(hg):
        if not d:
            continue
        pins = {int(img[s])} | {int(img[q]) for q in d}
        dimg = {int(img[q]) for q in d}
        for n in pins:
            for m in pins:
                if n != m:
                    sc[(n, m)] = sc.get((n, m), 0) + w
        for n in dimg:
            for m in dimg:
                if n != m:
                    ov[(n, m)] = ov.get((n, m), 0) + 1
    return sc, ov


def candidates(hg, img, mem, prm):
    """cand(n) by argmax over valid neighbours, ties to the lower id; the
    merged super-node's limits are checked on the union of members."""
    sc, ov = score_ov(hg, img)
    ins = in_sets(hg)
    VL = len(mem)
    cand = [-1] * VL
    cscore = [0] * VL
    cov = [0] * VL
    for n in range(VL):
        best = None
        for m in range(VL):
            if m == n or (n, m) not in sc:
                continue
            if not group_ok(hg, mem[n] | mem[m], prm, ins):
                continue
            key = (sc[(n, m)], -m)
            if best is None or key > best:
                best = key
        if best is not None:
            m = -best[1]
            cand[n], cscore[n], cov[n] = m, sc[(n, m)], ov.get((n, m), 0)
    return cand, cscore, cov


def matching(cand, cscore):
    """Eq. matching, evaluated literally by memoised recursion."""
    V = len(cand)
    children = [[] for _ in range(V)]
    for m in range(V):
        if cand[m] >= 0:
            children[cand[m]].append(m)

    @functools.lru_cache(maxsize=None)
    def M(n):
        c = cand[n]
        if c >= 0 and (cand[c] == n or M(c) == n):
            return c
        if children[n]:
            return max(children[n], key=lambda m: (cscore[m], -m))
        return -1

    return [M(n) for n in range(V)]


def refine_round(hg, img, VL, rho, K, prm):
    """One refinement round on level-l vertices (``img`` maps neurons to
    them). Returns (new rho, n_props, istar, gain)."""
    ins = in_sets(hg)
    mem = [set() for _ in range(VL)]
    for q in range(hg.V):
        mem[int(img[q])].add(q)
    rho = list(rho)

    def proj(r):
        return [r[int(img[q])] for q in range(hg.V)]

    def part_neurons(r, p):
        s = set()
        for n in range(VL):
            if r[n] == p:
                s |= mem[n]
        return s

    base = conn(hg, proj(rho))
    props = []
    pr0 = proj(rho)
    axons = [({s} | d) for s, d, w in hedges(hg) if d]
    nonpos = getattr(prm, "refine_nonpositive", 0)
    for n in range(VL):
        # partitions adjacent to n: holding a neuron of an axon that touches n
        adj = {pr0[q] for e in axons if e & mem[n] for q in e}
        best = None
        for p in range(K):
            if p == rho[n] or p not in adj:
                continue
            if not group_ok(hg, part_neurons(rho, p) | mem[n], prm, ins):
                continue
            r2 = list(rho)
            r2[n] = p
            g = base - conn(hg, proj(r2))
            if best is None or (g, -p) > best:
                best = (g, -p)
        if best is not None and (best[0] > 0 or nonpos):
            props.append((n, rho[n], -best[1], best[0]))
    props.sort(key=lambda t: (-t[3], t[0]))
    cur = list(rho)
    c0 = base
    G, bestG, istar = 0, 0, 0
    for i, (n, f, t, _) in enumerate(props):
        cur[n] = t
        c1 = conn(hg, proj(cur))
        G += c0 - c1
        c0 = c1
        valid = all(group_ok(hg, part_neurons(cur, p), prm, ins) for p in set(cur))
        if valid and G > 0 and G > bestG:
            bestG, istar = G, i + 1
    out = list(rho)
    for n, f, t, _ in props[:istar]:
        out[n] = t
    return out, len(props), istar, bestG


def set_partitions(V):
    """All partitions of range(V) as restricted growth strings."""
    def rec(i, a, mx):
        if i == V:
            yield list(a)
            return
        for b in range(mx + 2):
            a.append(b)
            yield from rec(i + 1, a, max(mx, b))
            a.pop()
    yield from rec(0, [], -1)


def optimum(hg, prm):
    """Exhaustive minimum of Eq. connectivity over feasible partitions."""
    best = None
    for rho in set_partitions(hg.V):
        if not feasible(hg, rho, prm):
            continue
        c = conn(hg, rho)
        if best is None or c < best:
            best = c
    return best


def components_fit(hg, prm):
    """True if every connected component of the hypergraph fits one core."""
    parent = list(range(hg.V))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for s, d, w in hedges(hg):
        for q in d:
            parent[find(q)] = find(s)
    comps = {}
    for n in range(hg.V):
        comps.setdefault(find(n), set()).add(n)
    ins = in_sets(hg)
    return all(group_ok(hg, c, prm, ins) for c in comps.values())


__all__ = [n for n in dir() if not n.startswith("_") and n not in ("functools", "itertools", "np")]


# --- placement (Sec. 4.2) -------------------------------------------------

def place_trd(hedges_, eta, width, gamma):
    """Total residual distance: eta-weighted Manhattan distances of all
    unordered pin pairs of every hyperedge."""
    d = 0
    for pins, w in zip(hedges_, eta):
        for i in range(len(pins)):
            for j in range(i + 1, len(pins)):
                a, b = gamma[pins[i]], gamma[pins[j]]
                d += w * (abs(a % width - b % width) + abs(a // width - b // width))
    return d


def place_round(hedges_, eta, width, height, gamma):
    """One swap-refinement round restated with tension := the residual
    distance a swap removes (recomputed from scratch), Eq. matching by the
    memoised restatement, and the prefix by sequential recomputation.
    Returns (new gamma, props, swaps, applied, gain)."""
    nh = width * height
    gamma = list(gamma)
    pi = [-1] * nh
    for p, h in enumerate(gamma):
        pi[h] = p

    def swapped(g, pi_, h, k):
        g2, pi2 = list(g), list(pi_)
        a, b = pi2[h], pi2[k]
        pi2[h], pi2[k] = b, a
        if a >= 0:
            g2[a] = k
        if b >= 0:
            g2[b] = h
        return g2, pi2

    def tension(g, pi_, h, k):
        g2, _ = swapped(g, pi_, h, k)
        return place_trd(hedges_, eta, width, g) - place_trd(hedges_, eta, width, g2)

    cand, cs = [-1] * nh, [0] * nh
    props = 0
    for h in range(nh):
        if pi[h] < 0:
            continue
        x, y = h % width, h // width
        nb = [k for k, ok in ((h - width, y > 0), (h - 1, x > 0), (h + 1, x + 1 < width),
                              (h + width, y + 1 < height)) if ok]
        best = None
        for k in sorted(nb):
            t = tension(gamma, pi, h, k)
            if best is None or t > best[0]:
                best = (t, k)
        if best is not None and best[0] > 0:
            cand[h], cs[h] = best[1], best[0]
            props += 1
    m = matching(cand, cs)
    sw = sorted(((tension(gamma, pi, h, m[h]), h, m[h]) for h in range(nh) if m[h] > h),
                key=lambda t: (-t[0], t[1]))
    g, p_ = list(gamma), list(pi)
    G = bestG = istar = 0
    for i, (_, h, k) in enumerate(sw):
        G += tension(g, p_, h, k)
        g, p_ = swapped(g, p_, h, k)
        if G > 0 and G > bestG:
            bestG, istar = G, i + 1
    g, p_ = list(gamma), list(pi)
    for _, h, k in sw[:istar]:
        g, p_ = swapped(g, p_, h, k)
    return g, props, len(sw), istar, bestG


def initial_sequence(hedges_, eta, seq0):
    """Readings RI2-RI4 restated recursively on node sets: halving, steepest
    swaps between the halves, then bottom-up orientation against each
    section's sibling."""
    def cut(A, B):
        return sum(w for e, w in zip(hedges_, eta) if set(e) & A and set(e) & B)

    def build(seq):
        if len(seq) <= 1:
            return {"seq": list(seq), "kids": None}
        mid = (len(seq) + 1) // 2
        L, R = list(seq[:mid]), list(seq[mid:])
        cur = cut(set(L), set(R))
        for _ in range(4 * min(len(L), len(R))):
            best = None
            for x in L:
                for y in R:
                    L2 = [y if v == x else v for v in L]
                    R2 = [x if v == y else v for v in R]
                    d = cur - cut(set(L2), set(R2))
                    if d > 0 and (best is None or (-d, x, y) < (-best[0], best[1], best[2])):
                        best = (d, x, y, L2, R2)
            if best is None:
                break
            cur -= best[0]
            L, R = best[3], best[4]
        return {"seq": None, "kids": [build(L), build(R)]}

    def flat(t):
        return t["seq"] if t["kids"] is None else flat(t["kids"][0]) + flat(t["kids"][1])

    def orient(t, sib=None, sib_right=None):
        if t["kids"] is None:
            return t["seq"]
        a, b = t["kids"]
        sa = orient(a, set(flat(b)), True)
        sb = orient(b, set(flat(a)), False)
        seq = sa + sb
        if sib is not None:
            ca, cb = cut(set(sa), sib), cut(set(sb), sib)
            if (ca > cb) if sib_right else (cb > ca):
                seq = seq[::-1]
        return seq

    return orient(build(list(seq0)))
