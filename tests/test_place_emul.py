"""The placement refinement kernels' steps (csrc/place_items.cuh) run on the
host in the kernels' phase order (tests/place_emul.cpp) and compared with
the oracle (Sec. 4.2; readings RP1-RP6): per start, the same placement, the
same rounds and the same per-round logs, for single starts and for several
starts refined together; the total residual distance agrees too. This pins
the GPU path's decomposition (forces per pin entry, tensions from
directional forces, re-evaluation through ranks, per-start prefixes) on the
CPU; the GPU parity tests run the kernels themselves."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import snngen
from test_placement import csr, random_case

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2609_07577_gb300", "csrc")


@pytest.fixture(scope="module")
def emul(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("emul") / "libplace_emul.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC,
                    os.path.join(HERE, "place_emul.cpp"), "-o", out], check=True)
    L = C.CDLL(out)
    vp, i32 = C.c_void_p, C.c_int32
    L.emul_place_refine.restype = C.c_int
    L.emul_place_refine.argtypes = [i32, i32, vp, vp, vp, i32, i32, i32, vp, i32, vp, vp, vp,
                                    vp, vp, i32]
    L.emul_place_trd.restype = None
    L.emul_place_trd.argtypes = [i32, i32, vp, vp, vp, i32, i32, vp, vp]
    return L


def ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def run_emul(L, n, off, pins, eta, width, height, gammas, max_rounds=1000, cap=4096):
    S = len(gammas)
    off = np.ascontiguousarray(off, np.int64)
    pins = np.ascontiguousarray(pins, np.int32)
    eta = np.ascontiguousarray(eta, np.int64)
    g = np.ascontiguousarray(np.concatenate([np.asarray(x, np.int32) for x in gammas])
                             if n else np.zeros(0, np.int32))
    rounds = np.zeros(S, np.int32)
    lp = np.zeros(S * cap, np.int32)
    ls = np.zeros(S * cap, np.int32)
    la = np.zeros(S * cap, np.int32)
    lg = np.zeros(S * cap, np.int64)
    rc = L.emul_place_refine(n, len(off) - 1, ptr(off), ptr(pins), ptr(eta), width, height, S,
                             ptr(g), max_rounds, ptr(rounds), ptr(lp), ptr(ls), ptr(la), ptr(lg),
                             cap)
    if rc:
        return rc, None, None
    outs, logs = [], []
    for s in range(S):
        outs.append(g[s * n:(s + 1) * n].tolist())
        logs.append([{"props": int(lp[s * cap + r]), "swaps": int(ls[s * cap + r]),
                      "applied": int(la[s * cap + r]), "gain": int(lg[s * cap + r])}
                     for r in range(min(int(rounds[s]), cap))])
    return 0, outs, logs


def trd_emul(L, n, off, pins, eta, width, gammas):
    S = len(gammas)
    off = np.ascontiguousarray(off, np.int64)
    pins = np.ascontiguousarray(pins, np.int32)
    eta = np.ascontiguousarray(eta, np.int64)
    g = np.ascontiguousarray(np.concatenate([np.asarray(x, np.int32) for x in gammas]))
    out = np.zeros(S, np.int64)
    L.emul_place_trd(n, len(off) - 1, ptr(off), ptr(pins), ptr(eta), width, S, ptr(g), ptr(out))
    return out.tolist()


def test_single_start_matches_oracle(emul):
    compared = moved = 0
    for seed in range(600):
        width, height, n, hedges_, eta, gamma = random_case(seed)
        off, pins = csr(hedges_)
        want_g, want_logs = oracle.place_refine(n, off, pins, eta, width, height, gamma)
        rc, got, logs = run_emul(emul, n, off, pins, eta, width, height, [gamma])
        assert rc == 0, seed
        assert got[0] == want_g.tolist(), seed
        assert logs[0] == want_logs, seed
        compared += 1
        moved += any(r["applied"] for r in want_logs)
    assert compared == 600 and moved > 150


def gp_case(seed, n_starts):
    """G_P of a small SNN under the oracle's partition, on the smallest
    near-square lattice that holds it, with n_starts random placements."""
    hg = snngen.tiny_random(seed) if seed % 2 else snngen.by_name("cfg1s")
    rho, _, st, *_ = oracle.partition(hg, oracle.params_of(hg))
    K = int(st["n_parts"])
    L = oracle.Level.from_hypergraph(hg, oracle.params_of(hg))
    gp = L.partition_graph(rho)
    off, pins, eta = gp["off"], gp["pins"], gp["eta"]
    width = int(np.ceil(np.sqrt(K)))
    height = int(np.ceil(K / width)) + (seed % 3 == 0)   # some lattices with empty rows
    rng = np.random.Generator(np.random.PCG64(seed))
    gammas = [rng.choice(width * height, size=K, replace=False) for _ in range(n_starts)]
    return K, off, pins, eta, width, height, gammas


@pytest.mark.parametrize("seed", [1, 2, 3, 5])
def test_multi_start_equals_each_start_alone(emul, seed):
    K, off, pins, eta, width, height, gammas = gp_case(seed, 5)
    rc, got, logs = run_emul(emul, K, off, pins, eta, width, height, gammas)
    assert rc == 0
    for s, gamma in enumerate(gammas):
        want_g, want_logs = oracle.place_refine(K, off, pins, eta, width, height, gamma)
        assert got[s] == want_g.tolist(), s
        assert logs[s] == want_logs, s
    trds = trd_emul(emul, K, off, pins, eta, width, got)
    assert trds == [oracle.place_trd(K, off, pins, eta, width, g) for g in got]


def test_multi_start_random_cases(emul):
    rng = np.random.Generator(np.random.PCG64(77))
    for seed in range(200):
        width, height, n, hedges_, eta, gamma = random_case(5000 + seed)
        off, pins = csr(hedges_)
        gammas = [gamma] + [rng.choice(width * height, size=n, replace=False).tolist()
                            for _ in range(int(rng.integers(1, 4)))]
        mr = int(rng.integers(1, 6))
        rc, got, logs = run_emul(emul, n, off, pins, eta, width, height, gammas, max_rounds=mr)
        assert rc == 0
        for s, gm in enumerate(gammas):
            want_g, want_logs = oracle.place_refine(n, off, pins, eta, width, height, gm,
                                                    max_rounds=mr)
            assert got[s] == want_g.tolist(), (seed, s)
            assert logs[s] == want_logs, (seed, s)


def test_invalid_placement_rejected(emul):
    off, pins = csr([[0, 1]])
    assert run_emul(emul, 2, off, pins, [1], 2, 1, [[0, 0]])[0] == 1
    assert run_emul(emul, 2, off, pins, [1], 2, 1, [[0, 2]])[0] == 1


# --- initial placement (Sec. 4.2, "Initial Placement"; readings RI1-RI4) ---

def initial_emul(L, n, off, pins, eta, width, height, seq0s):
    S = len(seq0s)
    off = np.ascontiguousarray(off, np.int64)
    pins = np.ascontiguousarray(pins, np.int32)
    eta = np.ascontiguousarray(eta, np.int64)
    s0 = np.ascontiguousarray(np.concatenate([np.asarray(x, np.int32) for x in seq0s]))
    seq = np.zeros(S * n, np.int32)
    gamma = np.zeros(S * n, np.int32)
    rc = L.emul_place_initial(n, len(off) - 1, ptr(off), ptr(pins), ptr(eta), width, height, S,
                              ptr(s0), ptr(seq), ptr(gamma))
    if rc:
        return rc, None, None
    return 0, [seq[s * n:(s + 1) * n].tolist() for s in range(S)], \
        [gamma[s * n:(s + 1) * n].tolist() for s in range(S)]


def random_initial_case(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    n = int(rng.integers(1, 40))
    hedges_ = [rng.choice(n, size=int(rng.integers(2, min(n, 6) + 1)), replace=False).tolist()
               for _ in range(int(rng.integers(0, 3 * n)))] if n >= 2 else []
    eta = rng.integers(1, 9, size=len(hedges_)).tolist()
    width = int(rng.integers(1, 8))
    height = -(-n // width) + int(rng.integers(0, 2))
    seq0s = [rng.permutation(n).tolist() for _ in range(int(rng.integers(1, 4)))]
    return n, hedges_, eta, width, height, seq0s


@pytest.fixture(scope="module")
def emul_initial(emul):
    emul.emul_place_initial.restype = C.c_int
    emul.emul_place_initial.argtypes = [C.c_int32, C.c_int32] + [C.c_void_p] * 3 + \
        [C.c_int32] * 3 + [C.c_void_p] * 3
    return emul


def test_initial_matches_oracle(emul_initial):
    for seed in range(300):
        n, hedges_, eta, width, height, seq0s = random_initial_case(seed)
        off, pins = csr(hedges_)
        rc, seqs, gammas = initial_emul(emul_initial, n, off, pins, eta, width, height, seq0s)
        assert rc == 0
        for s, s0 in enumerate(seq0s):
            assert seqs[s] == oracle.initial_sequence(n, off, pins, eta, s0).tolist(), (seed, s)
            assert gammas[s] == oracle.initial_placement(n, off, pins, eta, width, height,
                                                         s0).tolist(), (seed, s)


def gp_of(name):
    """G_P of a named SNN under the oracle's partition, on the smallest
    near-square lattice that holds it."""
    hg = snngen.by_name(name)
    rho, _, st, *_ = oracle.partition(hg, oracle.params_of(hg))
    K = int(st["n_parts"])
    gp = oracle.Level.from_hypergraph(hg, oracle.params_of(hg)).partition_graph(rho)
    width = int(np.ceil(np.sqrt(K)))
    return K, gp["off"], gp["pins"], gp["eta"], width, int(np.ceil(K / width))


def test_initial_on_gp_matches_oracle(emul_initial):
    K, off, pins, eta, width, height = gp_of("cfg2s")
    rng = np.random.Generator(np.random.PCG64(3))
    seq0s = [rng.permutation(K).tolist() for _ in range(4)]
    rc, seqs, gammas = initial_emul(emul_initial, K, off, pins, eta, width, height, seq0s)
    assert rc == 0
    for s, s0 in enumerate(seq0s):
        assert seqs[s] == oracle.initial_sequence(K, off, pins, eta, s0).tolist(), s
        assert gammas[s] == oracle.initial_placement(K, off, pins, eta, width, height,
                                                     s0).tolist(), s


def larger_initial_case(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    n = int(rng.integers(48, 97))
    hedges_ = [rng.choice(n, size=int(rng.integers(2, 9)), replace=False).tolist()
               for _ in range(3 * n)]
    eta = rng.integers(1, 20, size=len(hedges_)).tolist()
    width = int(np.ceil(np.sqrt(n)))
    height = -(-n // width)
    return n, hedges_, eta, width, height, [rng.permutation(n).tolist() for _ in range(2)]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_initial_larger_cases_match_oracle(emul_initial, seed):
    n, hedges_, eta, width, height, seq0s = larger_initial_case(seed)
    off, pins = csr(hedges_)
    rc, seqs, gammas = initial_emul(emul_initial, n, off, pins, eta, width, height, seq0s)
    assert rc == 0
    for s, s0 in enumerate(seq0s):
        assert gammas[s] == oracle.initial_placement(n, off, pins, eta, width, height,
                                                     s0).tolist(), s


def test_initial_rejects_repeated_pins_and_bad_orders(emul_initial):
    off, pins = csr([[0, 1, 0]])
    assert initial_emul(emul_initial, 2, off, pins, [1], 2, 1, [[0, 1]])[0] == 1
    off, pins = csr([[0, 1]])
    assert initial_emul(emul_initial, 2, off, pins, [1], 2, 1, [[0, 0]])[0] == 1


def test_lattice_for():
    from paper_2609_07577_gb300.api import lattice_for
    for n in range(1, 300):
        w, h = lattice_for(n)
        assert w * h >= n and w * (h - 1) < n and abs(w - h) <= 1


def test_initial_large_hyperedges_match_oracle(emul_initial):
    """Hyperedges of up to 12 pins over 20-64 nodes, several starts: many
    swaps whose hyperedges cross the count thresholds the incremental
    updates of the gains and the correction matrix follow."""
    swaps_seen = 0
    for seed in range(40):
        rng = np.random.Generator(np.random.PCG64(70_000 + seed))
        n = int(rng.integers(20, 65))
        hedges_ = [rng.choice(n, size=int(rng.integers(2, 13)), replace=False).tolist()
                   for _ in range(int(rng.integers(n, 3 * n)))]
        eta = rng.integers(1, 30, size=len(hedges_)).tolist()
        width = int(np.ceil(np.sqrt(n)))
        height = -(-n // width)
        seq0s = [rng.permutation(n).tolist() for _ in range(3)]
        off, pins = csr(hedges_)
        rc, seqs, gammas = initial_emul(emul_initial, n, off, pins, eta, width, height, seq0s)
        assert rc == 0
        for s, s0 in enumerate(seq0s):
            want = oracle.initial_sequence(n, off, pins, eta, s0).tolist()
            assert seqs[s] == want, (seed, s)
            swaps_seen += sum(a != b for a, b in zip(s0, want))
    assert swaps_seen > 1000


def test_repeated_pins_count_with_multiplicity(emul):
    """snnmap_place_refine's contract: a pin repeated within a hyperedge
    counts as often as it appears, as in the oracle (forces, re-evaluation
    and the total residual distance)."""
    compared = 0
    for seed in range(200):
        rng = np.random.Generator(np.random.PCG64(90_000 + seed))
        width, height = int(rng.integers(2, 6)), int(rng.integers(1, 5))
        n = int(rng.integers(2, width * height + 1))
        hedges_ = [rng.integers(0, n, size=int(rng.integers(2, 6))).tolist()
                   for _ in range(int(rng.integers(1, 2 * n)))]
        eta = rng.integers(1, 6, size=len(hedges_)).tolist()
        gamma = rng.choice(width * height, size=n, replace=False).tolist()
        off, pins = csr(hedges_)
        want_g, want_logs = oracle.place_refine(n, off, pins, eta, width, height, gamma)
        rc, got, logs = run_emul(emul, n, off, pins, eta, width, height, [gamma])
        assert rc == 0
        assert got[0] == want_g.tolist() and logs[0] == want_logs, seed
        assert trd_emul(emul, n, off, pins, eta, width, got) == \
            [oracle.place_trd(n, off, pins, eta, width, want_g)]
        compared += any(len(set(h)) < len(h) for h in hedges_)
    assert compared > 100
