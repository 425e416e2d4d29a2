"""Seeded synthetic SNN hypergraph generators (inputs only).

Each generator returns a :class:`Hypergraph`: one vertex per neuron and one
hyperedge per axon, stored as CSR over hyperedge pins with pin 0 of every
hyperedge equal to its source neuron and the remaining pins its distinct
destinations in ascending order (the SNN model of Sec. 2, "SNN and Hardware
Models"). The three per-core limits of Sec. 2 (neurons Omega, distinct inbound
axons Delta, inbound synapses Phi) travel with the hypergraph.

This module draws random numbers and lays out arrays; it holds none of the
partitioning method's arithmetic. It is the one module shared by the CPU
oracle tests and the CUDA path's tests and benchmark.

Shapes follow the synthetic stand-ins for the paper's benchmark networks
(Table "tab:snns": layered ANN-derived feedforward networks and cyclic
small-world networks):

* ``layered``      - feedforward layers, each neuron's axon reaching a
                      contiguous window of the next layer plus random picks.
* ``conv``         - layers of side x side x channels neurons, each axon
                      reaching a 3x3 x channels receptive window (torus
                      wrapped) of the next layer plus random picks.
* ``powerlaw``     - recurrent network, fan-out from a truncated Pareto
                      distribution, 70% of pins in the source's aligned
                      locality block and 30% uniform.
* ``tiny_random``  - small random hypergraphs for brute-force checks.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Hypergraph", "layered", "conv", "powerlaw", "tiny_random",
    "cfg1", "cfg2", "cfg3", "batch_jobs", "serve_stream", "by_name",
]


@dataclasses.dataclass
class Hypergraph:
    """CSR hypergraph: ``off[E+1]`` int64, ``pins[P]`` int32, ``w[E]`` int32.

    ``pins[off[a]]`` is the source of hyperedge ``a``; ``pins[off[a]+1:off[a+1]]``
    are its destinations (distinct, ascending, never the source).
    """
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

    def sizes(self) -> np.ndarray:
        return np.diff(self.off)

    def summary(self) -> dict:
        s = self.sizes()
        return {"name": self.name, "V": self.V, "E": self.E, "P": self.P,
                "max_hedge": int(s.max()) if s.size else 0,
                "sum_sq": int((s.astype(np.int64) ** 2).sum()),
                "omega": self.omega, "delta": self.delta, "phi": self.phi}


def _assemble(name, V, src, groups, w, omega, delta, phi) -> Hypergraph:
    """Build CSR from per-hyperedge sources and candidate destination pins.

    ``groups`` is a list of ``(hedge_ids, cand)`` with ``cand`` an
    ``len(hedge_ids) x width`` matrix of candidate destinations, ``-1`` for
    padding. Candidates equal to the source are removed and duplicates
    collapse to one pin (pins are drawn with replacement, then deduplicated).
    """
    E = int(src.shape[0])
    src = src.astype(np.int64)
    ndst = np.zeros(E, dtype=np.int64)
    cleaned = []
    for hids, cand in groups:
        if hids.shape[0] == 0:
            continue
        c = np.sort(cand.astype(np.int64), axis=1)
        keep = (c >= 0) & (c != src[hids][:, None])
        keep[:, 1:] &= c[:, 1:] != c[:, :-1]
        ndst[hids] = keep.sum(axis=1)
        cleaned.append((hids, c, keep))
    off = np.zeros(E + 1, dtype=np.int64)
    np.cumsum(ndst + 1, out=off[1:])
    pins = np.empty(int(off[-1]), dtype=np.int32)
    pins[off[:-1]] = src
    for hids, c, keep in cleaned:
        rank = np.cumsum(keep, axis=1) - 1
        pos = off[hids][:, None] + 1 + rank
        pins[pos[keep]] = c[keep]
    return Hypergraph(name, int(V), off, pins, np.ascontiguousarray(w, dtype=np.int32),
                      int(omega), int(delta), int(phi))


def _ragged_groups(count, flat):
    """Split a flat candidate list (``count[a]`` entries for hyperedge ``a``,
    in hyperedge order) into padded power-of-two-width matrices."""
    count = np.asarray(count, dtype=np.int64)
    start = np.zeros(count.shape[0] + 1, dtype=np.int64)
    np.cumsum(count, out=start[1:])
    width = np.maximum(1, count)
    bucket = np.ceil(np.log2(width)).astype(np.int64)
    groups = []
    for b in np.unique(bucket):
        hids = np.nonzero(bucket == b)[0]
        wd = 1 << int(b)
        col = np.arange(wd)[None, :]
        idx = start[hids][:, None] + col
        valid = col < count[hids][:, None]
        m = np.full((hids.shape[0], wd), -1, dtype=np.int64)
        m[valid] = flat[idx[valid]]
        groups.append((hids, m))
    return groups


def layered(layers=4, width=1024, window=32, nrand=8, seed=0,
            omega=256, delta=64, phi=None, name=None) -> Hypergraph:
    """Feedforward layered network: ``layers`` x ``width`` neurons.

    Neuron i of layer l < layers-1 has one axon to neurons (i+t) mod width,
    t = 0..window-1, of layer l+1, plus ``nrand`` uniform picks in layer l+1.
    Weight = Poisson(5) + 1 spikes.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    V = layers * width
    E = (layers - 1) * width
    src = np.arange(E, dtype=np.int64)
    lay = src // width
    i = src - lay * width
    nxt = (lay + 1) * width
    win = nxt[:, None] + (i[:, None] + np.arange(window)[None, :]) % width
    rnd = nxt[:, None] + rng.integers(0, width, size=(E, nrand))
    w = rng.poisson(5.0, size=E) + 1
    cand = np.concatenate([win, rnd], axis=1)
    if phi is None:
        phi = 16 * omega
    return _assemble(name or f"layered{layers}x{width}", V, src, [(src, cand)],
                     w, omega, delta, phi)


def conv(layers=8, side=128, channels=8, nrand=4, seed=1,
         omega=1024, delta=4096, phi=16384, name=None) -> Hypergraph:
    """Conv-like layered network of ``layers`` x side x side x channels neurons.

    Neuron ID = l*S + (y*side + x)*channels + c with S = side*side*channels.
    Each neuron of layers 0..layers-2 has one axon over the next layer's
    (x+dx, y+dy, c') for dx, dy in {-1,0,1}, all c' (wrapped as a torus), plus
    ``nrand`` uniform picks in the next layer. Weight ~ Geometric(p=0.2).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    S = side * side * channels
    V = layers * S
    E = (layers - 1) * S
    src = np.arange(E, dtype=np.int64)
    lay = src // S
    r = src - lay * S
    cell = r // channels
    y = cell // side
    x = cell - y * side
    nxt = (lay + 1) * S
    d = np.array([-1, 0, 1])
    yy = (y[:, None, None] + d[None, :, None]) % side
    xx = (x[:, None, None] + d[None, None, :]) % side
    base = nxt[:, None, None] + (yy * side + xx) * channels            # E x 3 x 3
    win = (base[..., None] + np.arange(channels)).reshape(E, -1)        # E x 9C
    rnd = nxt[:, None] + rng.integers(0, S, size=(E, nrand))
    w = rng.geometric(0.2, size=E)
    cand = np.concatenate([win, rnd], axis=1)
    return _assemble(name or f"conv{layers}x{side}x{side}x{channels}", V, src,
                     [(src, cand)], w, omega, delta, phi)


def powerlaw(V=1 << 23, block=65536, fmin=8, fmax=16384, alpha=2.1, local=0.7,
             seed=2, omega=4096, delta=16384, phi=65536, name=None) -> Hypergraph:
    """Recurrent power-law network: every neuron sources one axon.

    Fan-out is the integer part of an inverse-CDF draw of a Pareto law with
    survival proportional to x^-alpha, truncated to [fmin, fmax]. Each pin is
    drawn from the source's aligned ``block``-ID block (cut at V) with probability
    ``local``, else uniformly over all V neurons. Weight = max(1,
    round(lognormal(mu=1, sigma=1))).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    block = min(block, V)
    u = rng.random(V)
    lo = float(fmin) ** (-alpha)
    hi = float(fmax) ** (-alpha)
    fan = np.floor((lo - u * (lo - hi)) ** (-1.0 / alpha)).astype(np.int64)
    fan = np.clip(fan, fmin, fmax)
    total = int(fan.sum())
    hid = np.repeat(np.arange(V, dtype=np.int64), fan)
    is_local = rng.random(total) < local
    # the last block is cut at V when V is not a multiple of block; a draw r
    # in [0, block) is scaled onto it (unchanged for full blocks)
    base = (hid // block) * block
    width = np.minimum(block, V - base)
    loc = base + (rng.integers(0, block, size=total) * width) // block
    del base, width
    uni = rng.integers(0, V, size=total)
    cand = np.where(is_local, loc, uni)
    del loc, uni, is_local
    w = np.maximum(1, np.rint(rng.lognormal(1.0, 1.0, size=V))).astype(np.int64)
    w = np.minimum(w, np.iinfo(np.int32).max)
    src = np.arange(V, dtype=np.int64)
    return _assemble(name or f"powerlaw{V}", V, src, _ragged_groups(fan, cand),
                     w, omega, delta, phi)


def tiny_random(seed, V=None, E=None, wmax=5) -> Hypergraph:
    """Random hypergraph with at most 12 vertices and random core limits."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if V is None:
        V = int(rng.integers(2, 13))
    if E is None:
        E = int(rng.integers(1, 2 * V + 1))
    src = rng.integers(0, V, size=E)
    ndst = rng.integers(1, min(V, 6), size=E)
    cand = rng.integers(0, V, size=int(ndst.sum()))
    w = rng.integers(1, wmax + 1, size=E)
    groups = _ragged_groups(ndst, cand)
    omega = int(rng.integers(1, V + 1))
    delta = int(rng.integers(1, E + 2))
    phi = int(rng.integers(1, 3 * E + 2))
    return _assemble(f"tiny{seed}", V, src, groups, w, omega, delta, phi)


# --- the five workloads -----------------------------------------------------

def cfg1() -> Hypergraph:
    """Tiny feedforward SNN: 4 x 1024 neurons, 32-window + 8 random pins,
    Omega=256, Delta=64, Phi=16*Omega=4096, seed 0."""
    return layered(4, 1024, 32, 8, seed=0, omega=256, delta=64, phi=4096, name="cfg1")


def cfg2() -> Hypergraph:
    """Conv-like layered SNN: 8 layers of 128x128x8 (1,048,576 neurons), 72-pin
    receptive window + 4 random pins, Omega=1024, Delta=4096, Phi=16384, seed 1."""
    return conv(8, 128, 8, 4, seed=1, omega=1024, delta=4096, phi=16384, name="cfg2")


def cfg3() -> Hypergraph:
    """Recurrent power-law SNN: 2^23 neurons, Pareto(2.1) fan-out on [8, 16384],
    65536-ID locality blocks, Omega=4096, Delta=16384, Phi=65536, seed 2."""
    return powerlaw(1 << 23, 65536, 8, 16384, 2.1, 0.7, seed=2,
                    omega=4096, delta=16384, phi=65536, name="cfg3")


def batch_jobs_one(j, nmin=10_000, nmax=500_000):
    """Job j of a batched run: seed j; size log-uniform on [nmin, nmax]; even
    jobs are layered (4 layers), odd jobs power-law with locality block
    min(65536, N); Omega from {256, 1024, 4096}, Delta = 4*Omega,
    Phi = 16*Omega."""
    rng = np.random.Generator(np.random.PCG64(j))
    n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
    om = int(rng.choice([256, 1024, 4096]))
    if j % 2 == 0:
        width = max(64, n // 4)
        return layered(4, width, 32, 8, seed=j, omega=om, delta=4 * om, phi=16 * om,
                       name=f"job{j}")
    return powerlaw(n, min(65536, n), 8, 16384, 2.1, 0.7, seed=j, omega=om, delta=4 * om,
                    phi=16 * om, name=f"job{j}")


def batch_jobs(n_jobs=256, nmin=10_000, nmax=500_000):
    """The jobs 0..n_jobs-1 of a batched run (see batch_jobs_one)."""
    return [batch_jobs_one(j, nmin, nmax) for j in range(n_jobs)]


def serve_stream(n_jobs=2000, rate=200.0, nmin=10_000, nmax=2_000_000, seed=5):
    """Arrival times (seconds) and job descriptors of a served run: Poisson
    arrivals at ``rate`` jobs/s; sizes log-uniform on [nmin, nmax]; each job
    is conv-like or power-law with that workload's core limits."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, size=n_jobs)
    t = np.cumsum(gaps)
    sizes = np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=n_jobs))
    kinds = rng.integers(0, 2, size=n_jobs)
    out = []
    for j in range(n_jobs):
        out.append({"t": float(t[j]), "n": int(round(sizes[j])), "kind": int(kinds[j]),
                    "seed": 1000 + j})
    return out


def serve_job(desc) -> Hypergraph:
    """Materialise one served job from :func:`serve_stream`'s descriptor."""
    n, seed = desc["n"], desc["seed"]
    if desc["kind"] == 0:
        side = max(4, int(round(math.sqrt(n / 64.0))))
        return conv(8, side, 8, 4, seed=seed, omega=1024, delta=4096, phi=16384,
                    name=f"serve{seed}")
    return powerlaw(n, min(65536, n), 8, 16384, 2.1, 0.7, seed=seed,
                    omega=4096, delta=16384, phi=65536, name=f"serve{seed}")


def by_name(name: str) -> Hypergraph:
    """Named workloads, including the scaled-down variants used by tests."""
    table = {
        "cfg1": cfg1,
        "cfg2": cfg2,
        "cfg3": cfg3,
        # scaled-down instances of the same generators (oracle-sized)
        "cfg2s": lambda: conv(4, 16, 8, 4, seed=11, omega=1024, delta=4096, phi=16384,
                              name="cfg2s"),
        "cfg2m": lambda: conv(8, 32, 8, 4, seed=12, omega=1024, delta=4096, phi=16384,
                              name="cfg2m"),
        "cfg2q": lambda: conv(8, 64, 8, 4, seed=13, omega=1024, delta=4096, phi=16384,
                              name="cfg2q"),
        "cfg3s": lambda: powerlaw(1 << 14, 4096, 8, 2048, 2.1, 0.7, seed=21,
                                  omega=512, delta=2048, phi=8192, name="cfg3s"),
        "cfg3m": lambda: powerlaw(1 << 17, 65536, 8, 16384, 2.1, 0.7, seed=22,
                                  omega=4096, delta=16384, phi=65536, name="cfg3m"),
        "cfg1s": lambda: layered(4, 256, 32, 8, seed=3, omega=64, delta=48, phi=1024,
                                 name="cfg1s"),
    }
    return table[name]()
