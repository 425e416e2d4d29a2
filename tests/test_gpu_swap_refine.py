"""Placement swap refinement on the GPU (snnmap_place_refine, Sec. 4.2,
"Swap Proposals" and "Placement Refinement"; readings RP1-RP6) against the
oracle: per start the same placement, the same rounds and the same
per-round logs, on random lattices (empty cores, one-row and one-column
lattices, several starts at once, round caps) and on G_P of a partitioned
SNN refined from 64 random starts together (the paper's Pi), where sampled
starts are checked one by one and every start by invariants (an injective
placement, a total residual distance lowered by exactly the summed gains).
The total residual distance (snnmap_place_trd) equals the oracle's; invalid
input is rejected and leaves gamma unchanged.

The initial placement the refinement starts from (snnmap_place_initial,
snnmap_hilbert_order; readings RI1-RI4) is checked the same way: final
sequences and placements equal the oracle's start by start (random
hypergraphs, the G_P of cfg2s, larger random cases, several starts at once),
the Hilbert order equals the oracle's, and 64 starts on the G_P of cfg1s
(too large for the oracle's label propagation) are checked by invariants
and then refined."""
import numpy as np
import pytest
import torch

import oracle
from test_place_emul import gp_case, gp_of, larger_initial_case, random_initial_case
from test_placement import csr, random_case

pytestmark = pytest.mark.gpu


def dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt).cuda()


def upload(off, pins, eta):
    return dev(off, torch.int64), dev(pins, torch.int32), dev(eta, torch.int64)


def gpu_refine(n, off, pins, eta, width, height, gammas, max_rounds=1000, cap=4096):
    import paper_2609_07577_gb300 as P
    d_off, d_pins, d_eta = upload(off, pins, eta)
    flat = np.concatenate([np.asarray(x, np.int32) for x in gammas]) if n else \
        np.zeros(0, np.int32)
    g = dev(flat, torch.int32)
    rounds, logs = P.snnmap_place_refine(n, len(off) - 1, d_off, d_pins, d_eta, width, height,
                                         len(gammas), g, max_rounds, log_cap=cap)
    out = g.cpu().numpy().reshape(len(gammas), n)
    return [out[s].tolist() for s in range(len(gammas))], rounds, logs


def gpu_trd(n, off, pins, eta, width, height, gammas):
    import paper_2609_07577_gb300 as P
    d_off, d_pins, d_eta = upload(off, pins, eta)
    g = dev(np.concatenate([np.asarray(x, np.int32) for x in gammas]), torch.int32)
    return P.snnmap_place_trd(n, len(off) - 1, d_off, d_pins, d_eta, width, height, len(gammas),
                              g)


def test_single_starts_match_oracle():
    moved = 0
    for seed in range(300):
        width, height, n, hedges_, eta, gamma = random_case(seed)
        off, pins = csr(hedges_)
        want_g, want_logs = oracle.place_refine(n, off, pins, eta, width, height, gamma)
        got, rounds, logs = gpu_refine(n, off, pins, eta, width, height, [gamma])
        assert got[0] == want_g.tolist(), seed
        assert rounds[0] == len(want_logs) and logs[0] == want_logs, seed
        moved += any(r["applied"] for r in want_logs)
    assert moved > 75


def test_several_starts_and_round_caps():
    rng = np.random.Generator(np.random.PCG64(77))
    for seed in range(100):
        width, height, n, hedges_, eta, gamma = random_case(5000 + seed)
        off, pins = csr(hedges_)
        gammas = [gamma] + [rng.choice(width * height, size=n, replace=False).tolist()
                            for _ in range(int(rng.integers(1, 4)))]
        mr = int(rng.integers(1, 6))
        got, rounds, logs = gpu_refine(n, off, pins, eta, width, height, gammas, max_rounds=mr)
        for s, gm in enumerate(gammas):
            want_g, want_logs = oracle.place_refine(n, off, pins, eta, width, height, gm,
                                                    max_rounds=mr)
            assert got[s] == want_g.tolist(), (seed, s)
            assert rounds[s] == len(want_logs) and logs[s] == want_logs, (seed, s)


@pytest.mark.parametrize("shape", [(1, 9), (9, 1), (1, 1), (3, 3)])
def test_row_column_and_single_core_lattices(shape):
    width, height = shape
    rng = np.random.Generator(np.random.PCG64(width * 10 + height))
    nh = width * height
    for _ in range(20):
        n = int(rng.integers(1, nh + 1))
        hedges_ = [rng.choice(n, size=min(n, int(rng.integers(2, 4))), replace=False).tolist()
                   for _ in range(int(rng.integers(0, 2 * n + 1)))] if n >= 2 else []
        eta = rng.integers(1, 6, size=len(hedges_)).tolist()
        gamma = rng.choice(nh, size=n, replace=False).tolist()
        off, pins = csr(hedges_)
        want_g, want_logs = oracle.place_refine(n, off, pins, eta, width, height, gamma)
        got, rounds, logs = gpu_refine(n, off, pins, eta, width, height, [gamma])
        assert got[0] == want_g.tolist()
        assert logs[0] == want_logs


def test_gp_sixty_four_starts():
    K, off, pins, eta, width, height, gammas = gp_case(2, 64)
    got, rounds, logs = gpu_refine(K, off, pins, eta, width, height, gammas)
    for s in (0, 9, 27, 63):
        want_g, want_logs = oracle.place_refine(K, off, pins, eta, width, height, gammas[s])
        assert got[s] == want_g.tolist(), s
        assert logs[s] == want_logs, s
    trd0 = gpu_trd(K, off, pins, eta, width, height, gammas)
    trd1 = gpu_trd(K, off, pins, eta, width, height, got)
    for s in range(64):
        g = np.asarray(got[s])
        assert len(set(g.tolist())) == K and g.min() >= 0 and g.max() < width * height
        assert logs[s][-1]["applied"] == 0 and all(r["applied"] > 0 for r in logs[s][:-1])
        assert trd0[s] == oracle.place_trd(K, off, pins, eta, width, gammas[s])
        assert trd1[s] == oracle.place_trd(K, off, pins, eta, width, g)
        assert trd0[s] - trd1[s] == sum(r["gain"] for r in logs[s]), s
    assert min(trd1) < min(trd0)


def test_trd_matches_oracle():
    for seed in range(100):
        width, height, n, hedges_, eta, gamma = random_case(9000 + seed)
        if n == 0:
            continue
        off, pins = csr(hedges_)
        assert gpu_trd(n, off, pins, eta, width, height, [gamma]) == \
            [oracle.place_trd(n, off, pins, eta, width, gamma)]


def test_edge_cases():
    # no hyperedges: one round, nothing proposed
    got, rounds, logs = gpu_refine(3, [0], [], [], 2, 2, [[3, 0, 1]])
    assert got == [[3, 0, 1]] and rounds == [1]
    assert logs[0] == [{"props": 0, "swaps": 0, "applied": 0, "gain": 0}]
    # no nodes
    got, rounds, logs = gpu_refine(0, [0], [], [], 2, 2, [[]])
    assert rounds == [1] and logs[0][0]["props"] == 0
    # a round cap of zero runs nothing
    off, pins = csr([[0, 1]])
    got, rounds, logs = gpu_refine(2, off, pins, [5], 3, 1, [[0, 2]], max_rounds=0)
    assert got == [[0, 2]] and rounds == [0] and logs == [[]]
    # two pins at distance two on a row: one swap brings them together
    got, rounds, logs = gpu_refine(2, off, pins, [5], 3, 1, [[0, 2]])
    want_g, want_logs = oracle.place_refine(2, off, pins, [5], 3, 1, [0, 2])
    assert got[0] == want_g.tolist() and logs[0] == want_logs
    assert abs(got[0][0] - got[0][1]) == 1


def test_invalid_input_rejected():
    import paper_2609_07577_gb300 as P
    off, pins = csr([[0, 1], [1, 2]])
    eta = [1, 2]
    d_off, d_pins, d_eta = upload(off, pins, eta)
    for gammas in ([[0, 0, 1]], [[0, 1, 4]], [[0, 1, -1]], [[0, 1, 2], [3, 2, 3]]):
        flat = np.concatenate([np.asarray(x, np.int32) for x in gammas])
        g = dev(flat, torch.int32)
        with pytest.raises(P.SnnmapError) as e:
            P.snnmap_place_refine(3, 2, d_off, d_pins, d_eta, 2, 2, len(gammas), g, 10)
        assert e.value.code == P._native.ERR_INVALID
        assert g.cpu().numpy().tolist() == flat.tolist()
    g = dev([0, 1, 2], torch.int32)
    bad_pins = dev([0, 1, 1, 3], torch.int32)
    with pytest.raises(P.SnnmapError):
        P.snnmap_place_refine(3, 2, d_off, bad_pins, d_eta, 2, 2, 1, g, 10)
    bad_off = dev([0, 3, 2], torch.int64)
    with pytest.raises(P.SnnmapError):
        P.snnmap_place_refine(3, 2, bad_off, d_pins, d_eta, 2, 2, 1, g, 10)
    with pytest.raises(P.SnnmapError):
        P.snnmap_place_refine(5, 2, d_off, d_pins, d_eta, 2, 2, 1, g, 10)   # 5 nodes, 4 cores
    with pytest.raises(P.SnnmapError):
        P.snnmap_place_trd(3, 2, d_off, d_pins, d_eta, 0, 2, 1, g)
    assert g.cpu().numpy().tolist() == [0, 1, 2]


def test_runs_native_kernels():
    import paper_2609_07577_gb300 as P
    before = P.snnmap_launch_count()
    off, pins = csr([[0, 1, 2]])
    gpu_refine(3, off, pins, [4], 3, 3, [[0, 4, 8]])
    assert P.snnmap_launch_count() > before


# --- initial placement ---

def gpu_initial(n, off, pins, eta, width, height, seq0s):
    import paper_2609_07577_gb300 as P
    d_off, d_pins, d_eta = upload(off, pins, eta)
    S = len(seq0s)
    s0 = dev(np.concatenate([np.asarray(x, np.int32) for x in seq0s]), torch.int32)
    seq = torch.zeros(S * n, dtype=torch.int32, device="cuda")
    gamma = torch.zeros(S * n, dtype=torch.int32, device="cuda")
    P.snnmap_place_initial(n, len(off) - 1, d_off, d_pins, d_eta, width, height, S, s0, gamma,
                           d_seq_out=seq)
    seq = seq.cpu().numpy().reshape(S, n)
    gamma = gamma.cpu().numpy().reshape(S, n)
    return [seq[s].tolist() for s in range(S)], [gamma[s].tolist() for s in range(S)]


def test_initial_random_cases_match_oracle():
    for seed in range(150):
        n, hedges_, eta, width, height, seq0s = random_initial_case(seed)
        off, pins = csr(hedges_)
        seqs, gammas = gpu_initial(n, off, pins, eta, width, height, seq0s)
        for s, s0 in enumerate(seq0s):
            assert seqs[s] == oracle.initial_sequence(n, off, pins, eta, s0).tolist(), (seed, s)
            assert gammas[s] == oracle.initial_placement(n, off, pins, eta, width, height,
                                                         s0).tolist(), (seed, s)


def test_initial_gp_and_larger_cases_match_oracle():
    K, off, pins, eta, width, height = gp_of("cfg2s")
    rng = np.random.Generator(np.random.PCG64(3))
    seq0s = [rng.permutation(K).tolist() for _ in range(8)]
    seqs, gammas = gpu_initial(K, off, pins, eta, width, height, seq0s)
    for s, s0 in enumerate(seq0s):
        assert seqs[s] == oracle.initial_sequence(K, off, pins, eta, s0).tolist(), s
        assert gammas[s] == oracle.initial_placement(K, off, pins, eta, width, height,
                                                     s0).tolist(), s
    for seed in range(3):
        n, hedges_, eta, width, height, seq0s = larger_initial_case(seed)
        off, pins = csr(hedges_)
        _, gammas = gpu_initial(n, off, pins, eta, width, height, seq0s)
        for s, s0 in enumerate(seq0s):
            assert gammas[s] == oracle.initial_placement(n, off, pins, eta, width, height,
                                                         s0).tolist(), (seed, s)


@pytest.mark.parametrize("shape", [(1, 1), (1, 9), (9, 1), (3, 5), (22, 22), (37, 5), (64, 64)])
def test_hilbert_order_matches_oracle(shape):
    import paper_2609_07577_gb300 as P
    w, h = shape
    out = torch.zeros(w * h, dtype=torch.int32, device="cuda")
    P.snnmap_hilbert_order(w, h, out)
    assert out.cpu().numpy().tolist() == oracle.hilbert_order(w, h).tolist()


def test_initial_then_refine_sixty_four_starts():
    import paper_2609_07577_gb300 as P
    K, off, pins, eta, width, height, _ = gp_case(2, 1)
    rng = np.random.Generator(np.random.PCG64(64))
    seq0s = [rng.permutation(K).tolist() for _ in range(64)]
    seqs, gammas = gpu_initial(K, off, pins, eta, width, height, seq0s)
    first = set(oracle.hilbert_order(width, height)[:K].tolist())
    for s in range(64):
        assert sorted(seqs[s]) == list(range(K))
        assert set(gammas[s]) == first and len(set(gammas[s])) == K
    trd0 = gpu_trd(K, off, pins, eta, width, height, gammas)
    assert trd0 == [oracle.place_trd(K, off, pins, eta, width, g) for g in gammas]
    got, rounds, logs = gpu_refine(K, off, pins, eta, width, height, gammas)
    trd1 = gpu_trd(K, off, pins, eta, width, height, got)
    for s in range(64):
        assert trd0[s] - trd1[s] == sum(r["gain"] for r in logs[s])
        assert len(set(got[s])) == K
    # the initial placement already beats random ones on this G_P
    rand = [rng.choice(width * height, size=K, replace=False) for _ in range(8)]
    assert min(trd0) < min(gpu_trd(K, off, pins, eta, width, height, rand))


def test_initial_invalid_input_rejected():
    import paper_2609_07577_gb300 as P
    off, pins = csr([[0, 1, 0]])
    d_off, d_pins, d_eta = upload(off, pins, [1])
    g = torch.full((2,), 7, dtype=torch.int32, device="cuda")
    with pytest.raises(P.SnnmapError):
        P.snnmap_place_initial(2, 1, d_off, d_pins, d_eta, 2, 1, 1, dev([0, 1], torch.int32), g)
    off, pins = csr([[0, 1]])
    d_off, d_pins, d_eta = upload(off, pins, [1])
    for s0 in ([0, 0], [0, 2], [1, -1]):
        with pytest.raises(P.SnnmapError):
            P.snnmap_place_initial(2, 1, d_off, d_pins, d_eta, 2, 1, 1, dev(s0, torch.int32), g)
    with pytest.raises(P.SnnmapError):
        P.snnmap_place_initial(3, 1, d_off, d_pins, d_eta, 2, 1, 1,
                               dev([0, 1, 2], torch.int32), g)   # 3 nodes, 2 cores
    with pytest.raises(P.SnnmapError):
        P.snnmap_hilbert_order(0, 3, g)
    assert g.cpu().numpy().tolist() == [7, 7]


def test_place_flow_matches_oracle_composition():
    """paper_2609_07577_gb300.place: initial placements from seeded random
    orders, refinement, the start of smallest total residual distance --
    equal to the oracle's steps composed the same way."""
    import paper_2609_07577_gb300 as P
    K, off, pins, eta, width, height = gp_of("cfg2s")
    res = P.place(K, off, pins, eta, n_starts=8, seed=5)
    assert (res["width"], res["height"]) == (width, height)
    rng = np.random.Generator(np.random.PCG64(5))
    finals, trds, trds0 = [], [], []
    for _ in range(8):
        s0 = rng.permutation(K)
        g0 = oracle.initial_placement(K, off, pins, eta, width, height, s0)
        trds0.append(oracle.place_trd(K, off, pins, eta, width, g0))
        g1, _ = oracle.place_refine(K, off, pins, eta, width, height, g0)
        finals.append(g1)
        trds.append(oracle.place_trd(K, off, pins, eta, width, g1))
    best = min(range(8), key=lambda s: (trds[s], s))
    assert res["trds_initial"] == trds0 and res["trds"] == trds
    assert res["start"] == best and res["trd"] == trds[best]
    assert res["gamma"].tolist() == finals[best].tolist()


def test_place_best_choice():
    """snnmap_place_best: every start's total residual distance equals the
    oracle's, and the chosen start has the smallest one, the lowest start on
    ties (start 3 repeats start 0's placement)."""
    import paper_2609_07577_gb300 as P
    K, off, pins, eta, width, height = gp_of("cfg2s")
    rng = np.random.default_rng(3)
    g = [rng.permutation(width * height)[:K].astype(np.int32) for _ in range(3)]
    g.append(g[0].copy())
    d_gamma = torch.from_numpy(np.concatenate(g)).cuda()
    d_off, d_pins, d_eta = (torch.from_numpy(np.ascontiguousarray(a)).cuda()
                            for a in (off, pins.astype(np.int32), eta.astype(np.int64)))
    best, trd, trds = P.snnmap_place_best(K, len(off) - 1, d_off, d_pins, d_eta, width, height,
                                          4, d_gamma)
    ref = [oracle.place_trd(K, off, pins, eta, width, x) for x in g]
    assert trds == ref
    assert best == min(range(4), key=lambda s: (ref[s], s)) and trd == ref[best]
    assert best != 3
