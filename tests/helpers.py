"""Small test helpers shared by the oracle and GPU test files (no method
arithmetic: array plumbing only)."""
import numpy as np

import snngen


def hypergraph(V, hedges, w, omega, delta, phi, name="hand"):
    """Hypergraph from explicit pin lists (source first)."""
    off = np.zeros(len(hedges) + 1, np.int64)
    off[1:] = np.cumsum([len(h) for h in hedges])
    pins = np.array([q for h in hedges for q in h], np.int32)
    return snngen.Hypergraph(name, V, off, pins, np.array(w, np.int32), omega, delta, phi)


def canonical_hedges(off, pins, w, k, selfdst):
    """Hyperedges as a sorted list of (s, selfdst, D tuple, w, k), with equal
    (s, selfdst, D) keys merged (level 0 may list one axon shape twice)."""
    acc = {}
    for a in range(len(off) - 1):
        p = pins[off[a]:off[a + 1]].tolist()
        key = (p[0], int(selfdst[a]), tuple(sorted(p[1:])))
        g = acc.setdefault(key, [0, 0])
        g[0] += int(w[a])
        g[1] += int(k[a])
    return sorted(key + (v[0], v[1]) for key, v in acc.items())
