"""Placement swap refinement of G_P (Sec. 4.2, "Swap Proposals" and
"Placement Refinement"; readings RP1-RP6) in the oracle, pinned by a
hand-worked example, by a restatement of whole rounds in which a swap's
tension is the residual distance it removes (recomputed from scratch), and
by invariants: the placement stays injective, every round lowers the total
residual distance by exactly its logged gain, and refinement stops when a
round applies nothing."""
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


def random_case(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    width, height = int(rng.integers(1, 5)), int(rng.integers(1, 4))
    nh = width * height
    n = int(rng.integers(1, nh + 1))
    hedges_ = []
    for _ in range(int(rng.integers(0, 2 * n + 1))):
        k = int(rng.integers(2, min(n, 4) + 1)) if n >= 2 else 0
        if k < 2:
            break
        hedges_.append(rng.choice(n, size=k, replace=False).tolist())
    eta = rng.integers(1, 6, size=len(hedges_)).tolist()
    gamma = rng.choice(nh, size=n, replace=False).tolist()
    return width, height, n, hedges_, eta, gamma


def test_golden_example():
    with open(os.path.join(HERE, "golden", "place_example.json")) as f:
        ex = json.load(f)
    off, pins = csr(ex["hedges"])
    g, logs = oracle.place_refine(ex["n_nodes"], off, pins, ex["eta"], ex["width"],
                                  ex["height"], ex["gamma"])
    assert g.tolist() == ex["gamma_final"]
    assert logs == ex["logs"]
    assert oracle.place_trd(ex["n_nodes"], off, pins, ex["eta"], ex["width"], ex["gamma"]) == \
        ex["trd"][0]
    assert oracle.place_trd(ex["n_nodes"], off, pins, ex["eta"], ex["width"], g) == ex["trd"][1]


@pytest.mark.parametrize("chunk", range(3))
def test_round_matches_restatement(chunk):
    rounds = applied = 0
    for seed in range(chunk, 900, 3):
        width, height, n, hedges_, eta, gamma = random_case(seed)
        if not hedges_:
            continue
        off, pins = csr(hedges_)
        g, logs = oracle.place_refine(n, off, pins, eta, width, height, gamma, max_rounds=1)
        want, props, swaps, istar, gain = bf.place_round(hedges_, eta, width, height, gamma)
        assert g.tolist() == want, seed
        assert logs[0] == {"props": props, "swaps": swaps, "applied": istar, "gain": gain}, seed
        assert oracle.place_trd(n, off, pins, eta, width, gamma) == \
            bf.place_trd(hedges_, eta, width, gamma)
        rounds += 1
        applied += istar > 0
    assert rounds > 150 and applied > 50


def test_refinement_invariants():
    for seed in range(300):
        width, height, n, hedges_, eta, gamma = random_case(10_000 + seed)
        if not hedges_:
            continue
        off, pins = csr(hedges_)
        d0 = bf.place_trd(hedges_, eta, width, gamma)
        g, logs = oracle.place_refine(n, off, pins, eta, width, height, gamma)
        assert len(set(g.tolist())) == n and g.min() >= 0 and g.max() < width * height
        assert d0 - sum(r["gain"] for r in logs) == bf.place_trd(hedges_, eta, width, g.tolist())
        assert all(r["gain"] > 0 for r in logs if r["applied"])
        assert logs[-1]["applied"] == 0


def test_invalid_placement_rejected():
    off, pins = csr([[0, 1]])
    with pytest.raises(oracle.OracleError):
        oracle.place_refine(2, off, pins, [1], 2, 1, [0, 0])
