"""SNN hypergraphs in files: the CSR arrays the C ABI takes, plus the
per-core limits, in one .npz; and a builder from per-axon lists.

One neuron is one vertex; one axon is one hyperedge whose first pin is its
source neuron and whose other pins are the neurons it has synapses on
(Sec. 2). omega / delta / phi are the per-core limits on neurons, distinct
inbound axons and inbound synapses."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class SNNHypergraph:
    """off: int64[E+1] from 0; pins: int32[P], pin off[a] the source of axon
    a; w: int32[E] axon weights (spike frequencies, >= 1)."""
    name: str
    V: int
    off: np.ndarray
    pins: np.ndarray
    w: np.ndarray
    omega: int
    delta: int
    phi: int

    @property
    def E(self) -> int:
        return int(self.off.shape[0] - 1)

    @property
    def P(self) -> int:
        return int(self.pins.shape[0])


def check_snn(hg) -> None:
    """Raises ValueError unless the arrays have the layout the library takes
    (the library checks the same on the device and refuses bad input)."""
    off, pins, w = np.asarray(hg.off), np.asarray(hg.pins), np.asarray(hg.w)
    if off.ndim != 1 or off.shape[0] < 1 or off[0] != 0 or (np.diff(off) < 0).any():
        raise ValueError("off must start at 0 and not decrease")
    if off[-1] != pins.shape[0] or w.shape[0] != off.shape[0] - 1:
        raise ValueError("off[-1] must equal len(pins) and len(w) the number of axons")
    if pins.size and (pins.min() < 0 or pins.max() >= hg.V):
        raise ValueError("a pin outside [0, V)")
    if w.size and w.min() < 0:
        raise ValueError("axon weights (spike frequencies) must be >= 0")
    if hg.omega < 1 or hg.delta < 0 or hg.phi < 0:
        raise ValueError("omega must be >= 1, delta and phi >= 0")


def from_axons(V, axons, weights, omega, delta, phi, name="snn") -> SNNHypergraph:
    """Builds the CSR layout from per-axon (source, destinations) pairs:
    destinations are deduplicated and sorted, the source itself dropped from
    them, and axons left without a destination kept (the library drops them
    as carrying no connectivity)."""
    off = [0]
    pins = []
    for src, dsts in axons:
        d = sorted(set(int(x) for x in dsts) - {int(src)})
        pins.append(int(src))
        pins.extend(d)
        off.append(len(pins))
    hg = SNNHypergraph(name, int(V), np.asarray(off, np.int64), np.asarray(pins, np.int32),
                       np.asarray(weights, np.int32), int(omega), int(delta), int(phi))
    check_snn(hg)
    return hg


def save_snn(path, hg) -> None:
    """Writes an SNN hypergraph (any object with the SNNHypergraph fields)."""
    np.savez_compressed(path, V=np.int64(hg.V), off=np.asarray(hg.off, np.int64),
                        pins=np.asarray(hg.pins, np.int32), w=np.asarray(hg.w, np.int32),
                        omega=np.int64(hg.omega), delta=np.int64(hg.delta),
                        phi=np.int64(hg.phi), name=np.asarray(getattr(hg, "name", "snn")))


def load_snn(path, omega=None, delta=None, phi=None) -> SNNHypergraph:
    """Reads save_snn's format; limits given here override the file's."""
    with np.load(path) as z:
        lim = {k: (v if v is not None else int(z[k]) if k in z.files else None)
               for k, v in (("omega", omega), ("delta", delta), ("phi", phi))}
        if None in lim.values():
            raise ValueError("the per-core limits omega, delta and phi are needed")
        hg = SNNHypergraph(str(z["name"]) if "name" in z.files else "snn", int(z["V"]),
                           z["off"].astype(np.int64), z["pins"].astype(np.int32),
                           z["w"].astype(np.int32), lim["omega"], lim["delta"], lim["phi"])
    check_snn(hg)
    return hg
