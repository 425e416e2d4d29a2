"""CUDA paths that the default settings reach only on some inputs, each
checked bit for bit against the oracle on the same seeded input:

- coarsening with carried candidates (every level after the first takes the
  carried form) and with full histograms only;
- every histogram tier (warp, block, large block, split) forced by the tier
  thresholds, with the level logs showing that the forced tier ran;
- 64-bit score accumulators (summed omega above 2^32, which also keeps the
  refinement off the int32 connection rows);
- zero-weight axons (a partition is adjacent through a hyperedge of weight 0);
- the refinement's proposal update after short enacted prefixes, which runs
  on every histogram level (rows budget 0).
"""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import snngen
from gpu_helpers import lockstep

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__ as g
    g.build()
    import paper_2609_07577_gb300 as P
    P.lib()
    assert torch.cuda.is_available()


_REF = {}


def _oracle(hg, **kw):
    """The oracle's pass, once per input and parameters (results do not
    depend on the CUDA-side settings the tests vary)."""
    key = (hg.name, tuple(sorted(kw.items())))
    if key not in _REF:
        _REF[key] = oracle.partition(hg, oracle.params_of(hg, **kw))
    return _REF[key]


def _both(hg, setup=None, **kw):
    from paper_2609_07577_gb300 import HGraph, params_for
    ref = _oracle(hg, **kw)
    G = HGraph.from_hypergraph(hg, params=params_for(hg.omega, hg.delta, hg.phi, **kw))
    try:
        if setup is not None:
            setup(G)
        rho, cost, st = G.partition()
        got = (rho.cpu().numpy(), cost, st, G.level_logs(), G.round_logs())
    finally:
        G.close()
    return got, ref


def _assert_same(got, ref):
    rho, cost, st, lv, rl = got
    rho_o, cost_o, st_o, lv_o, rl_o = ref
    assert cost == cost_o
    assert np.array_equal(rho, rho_o)
    for k in ("levels", "n_parts", "nonempty_parts", "rounds", "moves", "cost_initial", "cost"):
        assert st[k] == st_o[k], k
    assert [(r["level"], r["round"], r["n_props"], r["istar"], r["gain"]) for r in rl] == \
           [(r["level"], r["round"], r["n_props"], r["istar"], r["gain"]) for r in rl_o]
    assert [(g["V"], g["E"], g["P"], g["n_cand"], g["n_pairs"]) for g in lv] == \
           [(g["V"], g["E"], g["P"], g["n_cand"], g["n_pairs"]) for g in lv_o]


def _mode(mode, rows=0):
    """Coarsening mode; rows=0 also turns off the score matrix and the
    connection rows, so every level takes the histogram paths."""
    def setup(G):
        G.set_coarsen_mode(mode)
        if rows is not None:
            G.set_row_budget(rows)
    return setup


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("name", ["cfg1s", "cfg1", "cfg2s", "cfg3s"])
def test_coarsening_modes_lockstep(name, mode):
    hg = snngen.by_name(name)
    logs = []
    n = lockstep(hg, max_levels=60, setup=_mode(mode), logs=logs)
    assert n >= 1
    # mode 2 carries every level after the first; mode 1 none
    assert [x["carried"] for x in logs] == ([0] + [1] * (len(logs) - 1) if mode == 2
                                            else [0] * len(logs))


@pytest.mark.parametrize("rows", [0, None])
@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("name", ["cfg1", "cfg2s", "cfg3s", "cfg2m"])
def test_coarsening_modes_partition(name, mode, rows):
    hg = snngen.by_name(name)
    got, ref = _both(hg, setup=_mode(mode, rows))
    _assert_same(got, ref)
    carried = [x["carried"] for x in got[3]]
    if mode == 1:
        assert 1 not in carried
    if rows == 0:
        assert 2 not in carried   # no score matrix
        assert (1 in carried) == (mode == 2)


def test_carried_coarsening_tiny_random():
    n = 0
    for seed in range(200):
        hg = snngen.tiny_random(70_000 + seed)
        try:
            ref = oracle.partition(hg)
        except oracle.OracleError:
            continue
        got, _ = _both(hg, setup=_mode(2))
        assert got[1] == ref[1], seed
        assert np.array_equal(got[0], ref[0]), seed
        n += 1
    assert n > 80


# (wwork, bwork, gwork) forcing each tier, and the level-log field that must
# then be nonzero on some level
TIERS = {
    "split": ((0, 0, 0), "n_global"),
    "big": ((0, 0, 1 << 40), "n_block"),
    "block": ((0, 1 << 40, 1 << 40), "n_block"),
}


@pytest.mark.parametrize("tier", sorted(TIERS))
@pytest.mark.parametrize("name", ["cfg2s", "cfg3s"])
def test_forced_tiers_lockstep(name, tier):
    (w, b, g), field = TIERS[tier]
    logs = []
    lockstep(snngen.by_name(name), max_levels=12,
             setup=lambda G: (_mode(1)(G), G.set_histogram_tiers(w, b, g)), logs=logs)
    assert any(x[field] > 0 for x in logs), logs


@pytest.mark.parametrize("tier", sorted(TIERS))
@pytest.mark.parametrize("name", ["cfg2s", "cfg3s"])
def test_forced_tiers_partition(name, tier):
    (w, b, g), field = TIERS[tier]
    hg = snngen.by_name(name)

    def setup(G):
        G.set_row_budget(0)   # gains from histograms on every level, in the forced tier
        G.set_histogram_tiers(w, b, g)

    got, ref = _both(hg, setup=setup)
    _assert_same(got, ref)
    assert any(x[field] > 0 for x in got[3])


def _scaled(hg, factor, name):
    w = hg.w.astype(np.int64) * factor
    assert w.max() < 2 ** 31
    return dataclasses.replace(hg, w=w.astype(np.int32), name=name)


def test_wide_accumulators():
    """Summed omega above 2^32: the neighbour scores take 64-bit table
    entries, and connection rows (int32 entries) are refused, so every
    round reads histograms."""
    hg = _scaled(snngen.by_name("cfg2s"), 1 << 22, "cfg2s_wide")
    assert int(hg.w.astype(np.int64).sum()) >= 1 << 32
    assert lockstep(hg, max_levels=60, setup=_mode(2, None)) >= 1
    for mode in (1, 2):
        got, ref = _both(hg, setup=_mode(mode, None))
        _assert_same(got, ref)
        assert all(r["rows"] == 0 for r in got[4])


def test_wide_accumulators_power_law():
    hg = _scaled(snngen.by_name("cfg3s"), 1 << 20, "cfg3s_wide")
    assert int(hg.w.astype(np.int64).sum()) >= 1 << 32
    got, ref = _both(hg, setup=_mode(2, None))
    _assert_same(got, ref)


@pytest.mark.parametrize("name", ["cfg2s", "cfg3s"])
def test_zero_weight_axons(name):
    hg = snngen.by_name(name)
    w = hg.w.copy()
    w[::5] = 0
    hg = dataclasses.replace(hg, w=w, name=name + "_w0")
    for rows in (0, None):
        for mode in (1, 2):
            got, ref = _both(hg, setup=_mode(mode, rows))
            _assert_same(got, ref)


@pytest.mark.parametrize("name", ["cfg1", "cfg2s", "cfg3s", "cfg2m"])
def test_histogram_rounds_everywhere(name):
    """Row budget 0: every level refines from per-round histograms, so every
    round after a level's first takes the proposal update of the enacted
    prefix (column update for short prefixes, re-evaluation flags
    otherwise)."""
    hg = snngen.by_name(name)
    got, ref = _both(hg, setup=lambda G: G.set_row_budget(0))
    _assert_same(got, ref)


@pytest.mark.parametrize("name", ["cfg2s", "cfg3s"])
def test_nonpositive_variant_histograms(name):
    hg = snngen.by_name(name)
    got, ref = _both(hg, setup=lambda G: G.set_row_budget(0), refine_nonpositive=1)
    _assert_same(got, ref)
