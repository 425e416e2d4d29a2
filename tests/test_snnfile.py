"""SNN hypergraph files (paper_2609_07577_gb300.snnfile) and the command line's
arguments, without a GPU: from_axons builds the layout the C ABI takes
(source first, destinations deduplicated, sorted and without the source),
save/load round-trips arrays and limits (overridable), and malformed input
is refused on the host."""
import numpy as np
import pytest

import snngen
from paper_2609_07577_gb300.snnfile import check_snn, from_axons, load_snn, save_snn


def test_from_axons_layout():
    hg = from_axons(5, [(0, [3, 1, 1, 0]), (2, []), (4, [2])], [3, 1, 2], 2, 4, 8)
    assert hg.off.tolist() == [0, 3, 4, 6]
    assert hg.pins.tolist() == [0, 1, 3, 2, 4, 2]
    assert hg.w.tolist() == [3, 1, 2] and (hg.V, hg.E, hg.P) == (5, 3, 6)
    assert (hg.omega, hg.delta, hg.phi) == (2, 4, 8)


def test_round_trip_and_overrides(tmp_path):
    hg = snngen.by_name("cfg1s")
    path = tmp_path / "g.npz"
    save_snn(path, hg)
    got = load_snn(path)
    assert (got.V, got.E, got.P) == (hg.V, hg.E, hg.P)
    np.testing.assert_array_equal(got.off, hg.off)
    np.testing.assert_array_equal(got.pins, hg.pins)
    np.testing.assert_array_equal(got.w, hg.w)
    assert (got.omega, got.delta, got.phi) == (hg.omega, hg.delta, hg.phi)
    got = load_snn(path, omega=7)
    assert (got.omega, got.delta, got.phi) == (7, hg.delta, hg.phi)


@pytest.mark.parametrize("bad", ["pin", "off", "w", "limits"])
def test_malformed_input_refused(bad):
    hg = from_axons(4, [(0, [1, 2]), (3, [0])], [1, 1], 2, 2, 4)
    if bad == "pin":
        hg.pins[1] = 9
    elif bad == "off":
        hg.off[1] = 7
    elif bad == "w":
        hg.w[0] = -1
    else:
        hg.omega = 0
    with pytest.raises(ValueError):
        check_snn(hg)


def test_silent_axon_accepted():
    # a spike frequency of 0 is valid input for the library, so for the file too
    hg = from_axons(4, [(0, [1, 2]), (3, [0])], [0, 2], 2, 2, 4)
    check_snn(hg)
    assert hg.w.tolist() == [0, 2]


def test_cli_rejects_no_starts():
    from paper_2609_07577_gb300.__main__ import parse
    with pytest.raises(SystemExit):
        parse(["map", "in.npz", "out.npz", "--place", "--starts", "0"])


def test_cli_arguments():
    from paper_2609_07577_gb300.__main__ import parse
    a = parse(["map", "in.npz", "out.npz", "--omega", "64", "--place", "--starts", "8"])
    assert (a.cmd, a.input, a.output, a.omega, a.delta, a.place, a.starts, a.seed) == \
        ("map", "in.npz", "out.npz", 64, None, True, 8, 0)
