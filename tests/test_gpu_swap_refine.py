"""Placement swap refinement on the GPU (snnmap_place_refine, Sec. 4.2,
"Swap Proposals" and "Placement Refinement"; readings RP1-RP6) against the
oracle: per start the same placement, the same rounds and the same
per-round logs, on random lattices (empty cores, one-row and one-column
lattices, several starts at once, round caps) and on G_P of a partitioned
SNN refined from 64 random starts together (the paper's Pi), where sampled
starts are checked one by one and every start by invariants (an injective
placement, a total residual distance lowered by exactly the summed gains).
The total residual distance (snnmap_place_trd) equals the oracle's; invalid
input is rejected and leaves gamma unchanged."""
import numpy as np
import pytest
import torch

import oracle
from test_place_emul import gp_case
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
