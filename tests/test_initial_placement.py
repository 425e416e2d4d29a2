"""Initial placement of G_P (Sec. 4.2, "Initial Placement"; readings
RI1-RI4) in the oracle: the Hilbert order of the lattice (on power-of-two
squares consecutive cores are lattice neighbours), the node sequence from
recursive bisection with label propagation and folding against a recursive
set-based restatement and a hand-worked example, and its use as the start
of the swap refinement."""
import json
import os

import numpy as np
import pytest

import oracle
import bruteforce as bf

HERE = os.path.dirname(os.path.abspath(__file__))


def csr(hedges_):
    off = np.cumsum([0] + [len(h) for h in hedges_]).astype(np.int64)
    pins = np.concatenate([np.asarray(h, np.int32) for h in hedges_]) if hedges_ else \
        np.zeros(0, np.int32)
    return off, pins


@pytest.mark.parametrize("side", [1, 2, 4, 8, 16, 32])
def test_hilbert_square_is_a_lattice_walk(side):
    order = oracle.hilbert_order(side, side)
    assert sorted(order.tolist()) == list(range(side * side))
    for u, v in zip(order[:-1], order[1:]):
        assert abs(u % side - v % side) + abs(u // side - v // side) == 1
    assert order[0] == 0


@pytest.mark.parametrize("w,h", [(3, 5), (7, 2), (1, 9), (6, 6)])
def test_hilbert_any_lattice_is_a_permutation(w, h):
    assert sorted(oracle.hilbert_order(w, h).tolist()) == list(range(w * h))


def test_golden_example():
    with open(os.path.join(HERE, "golden", "initial_placement_example.json")) as f:
        ex = json.load(f)
    off, pins = csr(ex["hedges"])
    seq = oracle.initial_sequence(ex["n_nodes"], off, pins, ex["eta"], ex["seq0"])
    assert seq.tolist() == ex["seq"]
    assert oracle.hilbert_order(ex["width"], ex["height"]).tolist() == ex["hilbert"]
    g = oracle.initial_placement(ex["n_nodes"], off, pins, ex["eta"], ex["width"], ex["height"],
                                 ex["seq0"])
    assert g.tolist() == ex["gamma"]
    assert oracle.place_trd(ex["n_nodes"], off, pins, ex["eta"], ex["width"], g) == ex["trd"]


def test_sequence_matches_restatement():
    checked = 0
    for seed in range(400):
        rng = np.random.Generator(np.random.PCG64(seed))
        n = int(rng.integers(1, 11))
        hedges_ = [rng.choice(n, size=int(rng.integers(2, min(n, 4) + 1)), replace=False).tolist()
                   for _ in range(int(rng.integers(0, 2 * n))) if n >= 2]
        eta = rng.integers(1, 6, size=len(hedges_)).tolist()
        seq0 = rng.permutation(n).tolist()
        off, pins = csr(hedges_)
        seq = oracle.initial_sequence(n, off, pins, eta, seq0)
        assert sorted(seq.tolist()) == list(range(n))
        assert seq.tolist() == bf.initial_sequence(hedges_, eta, seq0), seed
        checked += 1
    assert checked == 400


def test_multi_start_then_refine():
    """Several starts (different initial orders), each refined; the refined
    residual distance never exceeds its start's, and the best start is kept."""
    rng = np.random.Generator(np.random.PCG64(77))
    n, w, h = 12, 4, 4
    hedges_ = [rng.choice(n, size=3, replace=False).tolist() for _ in range(20)]
    eta = rng.integers(1, 6, size=len(hedges_)).tolist()
    off, pins = csr(hedges_)
    best = None
    for start in range(8):
        seq0 = np.random.Generator(np.random.PCG64(1000 + start)).permutation(n)
        g0 = oracle.initial_placement(n, off, pins, eta, w, h, seq0)
        assert len(set(g0.tolist())) == n
        d0 = oracle.place_trd(n, off, pins, eta, w, g0)
        g1, logs = oracle.place_refine(n, off, pins, eta, w, h, g0)
        d1 = oracle.place_trd(n, off, pins, eta, w, g1)
        assert d1 == d0 - sum(r["gain"] for r in logs) <= d0
        best = d1 if best is None else min(best, d1)
    assert best is not None
