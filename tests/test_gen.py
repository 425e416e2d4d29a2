"""Generator layout and shape checks (inputs only)."""
import numpy as np

import snngen


def _layout_ok(hg):
    s = hg.sizes()
    assert (s >= 1).all()
    assert hg.pins.dtype == np.int32 and hg.off.dtype == np.int64 and hg.w.dtype == np.int32
    assert hg.pins.min() >= 0 and hg.pins.max() < hg.V
    for a in range(0, hg.E, max(1, hg.E // 300)):
        p = hg.pins[hg.off[a]:hg.off[a + 1]]
        assert (np.diff(p[1:]) > 0).all() and (p[1:] != p[0]).all()


def test_cfg1_shape():
    hg = snngen.cfg1()
    _layout_ok(hg)
    assert hg.V == 4096 and hg.E == 3072
    s = hg.sizes()
    assert s.min() >= 33 and s.max() <= 41
    assert (hg.w >= 1).all()
    assert (hg.omega, hg.delta, hg.phi) == (256, 64, 4096)
    # window pins present: neuron i of layer 0 reaches i..i+31 of layer 1
    p = hg.pins[hg.off[5]:hg.off[6]]
    assert set(range(1024 + 5, 1024 + 37)) <= set(p.tolist())


def test_conv_window():
    hg = snngen.conv(3, 8, 8, 4, seed=3)
    _layout_ok(hg)
    S = 8 * 8 * 8
    assert hg.V == 3 * S and hg.E == 2 * S
    s = hg.sizes()
    assert s.min() >= 73 and s.max() <= 77
    # neuron (l=0, y=0, x=0, c=0): torus window covers y, x in {7, 0, 1}
    p = set(hg.pins[hg.off[0]:hg.off[1]].tolist())
    for y in (7, 0, 1):
        for x in (7, 0, 1):
            for c in range(8):
                assert S + (y * 8 + x) * 8 + c in p


def test_powerlaw_fanout_and_locality():
    hg = snngen.powerlaw(1 << 14, 4096, 8, 2048, 2.1, 0.7, seed=5)
    _layout_ok(hg)
    s = hg.sizes() - 1
    assert s.max() <= 2048
    assert np.median(s) >= 7
    hid = np.repeat(np.arange(hg.E), hg.sizes())
    dst = np.ones(hg.P, bool)
    dst[hg.off[:-1]] = False
    local = (hg.pins[dst] // 4096) == (hid[dst] // 4096)
    assert 0.65 < local.mean() < 0.85


def test_deterministic():
    a, b = snngen.by_name("cfg3s"), snngen.by_name("cfg3s")
    assert (a.pins == b.pins).all() and (a.off == b.off).all() and (a.w == b.w).all()


def test_batch_and_serve_descriptors():
    jobs = snngen.batch_jobs(n_jobs=4, nmin=2000, nmax=4000)
    assert len(jobs) == 4
    for j in jobs:
        _layout_ok(j)
        assert j.delta == 4 * j.omega and j.phi == 16 * j.omega
    st = snngen.serve_stream(n_jobs=50)
    t = [d["t"] for d in st]
    assert all(x < y for x, y in zip(t, t[1:]))
    _layout_ok(snngen.serve_job({"n": 5000, "kind": 0, "seed": 1}))
    _layout_ok(snngen.serve_job({"n": 5000, "kind": 1, "seed": 2}))


def test_powerlaw_pins_in_range_when_v_is_not_a_block_multiple():
    hg = snngen.powerlaw(10_000, 4096, 8, 512, 2.1, 0.7, seed=9, omega=256, delta=1024,
                         phi=4096)
    assert hg.pins.min() >= 0 and hg.pins.max() < hg.V
    # the cut last block still receives its local pins
    src = np.repeat(hg.pins[hg.off[:-1]], np.diff(hg.off))
    last = src >= 8192
    assert (hg.pins[last] >= 8192).mean() > 0.5
