"""CPU oracle of the multilevel hypergraph partitioning pass (Sec. 4.1).

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the
benchmark's CPU-baseline leg are the only callers. The oracle is plain C
(``snnmap_oracle.c``), single-threaded and integer-exact, compiled here with
gcc and loaded through ctypes. It shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "snnmap_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_INVALID, ERR_INFEASIBLE, ERR_OOM = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("omega", C.c_int32), ("delta", C.c_int32), ("phi", C.c_int32),
                ("max_levels", C.c_int32), ("max_refine_rounds", C.c_int32),
                ("refine_nonpositive", C.c_int32)]


class RoundLog(C.Structure):
    _fields_ = [("level", C.c_int32), ("round", C.c_int32), ("n_props", C.c_int32),
                ("istar", C.c_int32), ("gain", C.c_int64)]


class LevelLog(C.Structure):
    _fields_ = [("V", C.c_int32), ("E", C.c_int32), ("P", C.c_int64),
                ("n_cand", C.c_int32), ("n_pairs", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("levels", C.c_int32), ("n_parts", C.c_int32), ("nonempty_parts", C.c_int32),
                ("rounds", C.c_int32), ("moves", C.c_int64), ("cost_initial", C.c_int64),
                ("cost", C.c_int64)]


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # SNNMAP_ORACLE_LIB: a library built elsewhere from a modified copy of
            # the source (the planted-mistake tests load mutants this way)
            _lib = C.CDLL(os.environ.get("SNNMAP_ORACLE_LIB") or build())
            L = _lib
            vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
            L.orc_build.argtypes = [vp, i32, i32, vp, vp, vp, C.POINTER(vp)]
            L.orc_build.restype = C.c_int
            L.orc_free.argtypes = [vp]
            L.orc_level_dims.argtypes = [vp, vp, vp, vp]
            L.orc_level_copy.argtypes = [vp] + [vp] * 9
            L.orc_affinity.argtypes = [vp, vp, vp, vp, vp]
            L.orc_affinity.restype = C.c_int
            L.orc_cand_one.argtypes = [vp, vp, i32, vp, vp, vp]
            L.orc_cand_one.restype = C.c_int
            L.orc_match.argtypes = [i32, vp, vp, vp]
            L.orc_match.restype = i32
            L.orc_contract.argtypes = [vp, vp, vp, vp, vp, C.POINTER(vp)]
            L.orc_contract.restype = C.c_int
            L.orc_conn.argtypes = [vp, vp]
            L.orc_gp.restype = C.c_int
            L.orc_gp.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
            L.orc_hilbert_order.restype = C.c_int
            L.orc_hilbert_order.argtypes = [i32, i32, vp]
            L.orc_initial_sequence.restype = C.c_int
            L.orc_initial_sequence.argtypes = [i32, i32, vp, vp, vp, vp]
            L.orc_place_trd.restype = C.c_int64
            L.orc_place_trd.argtypes = [i32, i32, vp, vp, vp, i32, vp]
            L.orc_place_refine.restype = C.c_int32
            L.orc_place_refine.argtypes = [i32, i32, vp, vp, vp, i32, i32, vp, i32, vp, vp, vp,
                                           vp, i32]
            L.orc_conn.restype = i64
            L.orc_refine.argtypes = [vp, i32, vp, vp, i32, vp, i32, vp, vp]
            L.orc_refine.restype = i32
            L.orc_partition.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, i32, vp,
                                        vp, i32, vp]
            L.orc_partition.restype = C.c_int
        return _lib


def params(omega, delta, phi, max_levels=1024, max_refine_rounds=16,
           refine_nonpositive=0) -> Params:
    return Params(int(omega), int(delta), int(phi), int(max_levels), int(max_refine_rounds),
                  int(refine_nonpositive))


def params_of(h, **kw) -> Params:
    return params(h.omega, h.delta, h.phi, **kw)


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle error {code}")
        self.code = code


class Level:
    """One level of the oracle's hierarchy (owns a C ``orc_level``)."""

    def __init__(self, handle):
        self._h = C.c_void_p(handle)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_free(self._h)
            self._h = None

    @classmethod
    def build(cls, V, off, pins, w, prm: Params) -> "Level":
        off = np.ascontiguousarray(off, np.int64)
        pins = np.ascontiguousarray(pins, np.int32)
        w = np.ascontiguousarray(w, np.int32)
        h = C.c_void_p()
        rc = lib().orc_build(C.byref(prm), int(V), int(off.shape[0] - 1), _ptr(off), _ptr(pins),
                             _ptr(w), C.byref(h))
        if rc != OK:
            raise OracleError(rc)
        return cls(h.value)

    @classmethod
    def from_hypergraph(cls, hg, prm: Params | None = None) -> "Level":
        return cls.build(hg.V, hg.off, hg.pins, hg.w, prm or params_of(hg))

    def dims(self):
        V, E, P = C.c_int32(), C.c_int32(), C.c_int64()
        lib().orc_level_dims(self._h, C.byref(V), C.byref(E), C.byref(P))
        return V.value, E.value, P.value

    def arrays(self) -> dict:
        V, E, P = self.dims()
        d = {"off": np.empty(E + 1, np.int64), "pins": np.empty(P, np.int32),
             "w": np.empty(E, np.int64), "k": np.empty(E, np.int32),
             "selfdst": np.empty(E, np.uint8), "size": np.empty(V, np.int32),
             "inpins": np.empty(V, np.int32), "in_count": np.empty(V, np.int32),
             "in_internal": np.empty(V, np.int32)}
        lib().orc_level_copy(self._h, *[_ptr(d[k]) for k in
                                        ("off", "pins", "w", "k", "selfdst", "size", "inpins",
                                         "in_count", "in_internal")])
        d["V"], d["E"], d["P"] = V, E, P
        return d

    def affinity(self, prm: Params):
        V = self.dims()[0]
        cand = np.empty(V, np.int32)
        cscore = np.empty(V, np.int64)
        cov = np.empty(V, np.int32)
        rc = lib().orc_affinity(self._h, C.byref(prm), _ptr(cand), _ptr(cscore), _ptr(cov))
        if rc != OK:
            raise OracleError(rc)
        return cand, cscore, cov

    def cand_one(self, n, prm: Params):
        c, s, o = C.c_int32(), C.c_int64(), C.c_int32()
        rc = lib().orc_cand_one(self._h, C.byref(prm), int(n), C.byref(c), C.byref(s), C.byref(o))
        if rc != OK:
            raise OracleError(rc)
        return c.value, s.value, o.value

    def contract(self, match, cand, cov):
        V = self.dims()[0]
        match = np.ascontiguousarray(match, np.int32)
        cand = np.ascontiguousarray(cand, np.int32)
        cov = np.ascontiguousarray(cov, np.int32)
        cid = np.empty(V, np.int32)
        h = C.c_void_p()
        rc = lib().orc_contract(self._h, _ptr(match), _ptr(cand), _ptr(cov), _ptr(cid),
                                C.byref(h))
        if rc != OK:
            raise OracleError(rc)
        return Level(h.value), cid

    def conn(self, rho) -> int:
        rho = np.ascontiguousarray(rho, np.int32)
        return int(lib().orc_conn(self._h, _ptr(rho)))

    def partition_graph(self, rho):
        """G_P of a partition of this level (R18): dict(off, pins, eta,
        axons, internal), hyperedges in canonical order."""
        V, E, P = self.dims()
        rho = np.ascontiguousarray(rho, dtype=np.int32)
        off = np.zeros(E + 1, np.int64)
        pins = np.zeros(max(P, 1), np.int32)
        eta = np.zeros(max(E, 1), np.int64)
        axons = np.zeros(max(E, 1), np.int32)
        ne, npins, inw = C.c_int32(), C.c_int64(), C.c_int64()
        rc = _lib.orc_gp(self._h, _ptr(rho), _ptr(off), _ptr(pins), _ptr(eta), _ptr(axons),
                         C.byref(ne), C.byref(npins), C.byref(inw))
        if rc:
            raise OracleError(rc)
        e, p = ne.value, npins.value
        return {"off": off[:e + 1], "pins": pins[:p], "eta": eta[:e], "axons": axons[:e],
                "internal": inw.value}

    def refine(self, K, rho, prm: Params, level=0, log_cap=4096):
        """Refines ``rho`` in place; returns (rounds, moves, round logs)."""
        assert rho.dtype == np.int32 and rho.flags.c_contiguous
        logs = (RoundLog * log_cap)()
        n = C.c_int32(0)
        moves = C.c_int64(0)
        r = lib().orc_refine(self._h, int(K), _ptr(rho), C.byref(prm), int(level), logs,
                             log_cap, C.byref(n), C.byref(moves))
        if r < 0:
            raise OracleError(r)
        return r, moves.value, [_round(logs[i]) for i in range(n.value)]


def match(cand, cscore):
    cand = np.ascontiguousarray(cand, np.int32)
    cscore = np.ascontiguousarray(cscore, np.int64)
    V = cand.shape[0]
    out = np.empty(V, np.int32)
    pairs = lib().orc_match(V, _ptr(cand), _ptr(cscore), _ptr(out))
    return out, int(pairs)


def _round(r):
    return {"level": r.level, "round": r.round, "n_props": r.n_props, "istar": r.istar,
            "gain": r.gain}


def partition(hg, prm: Params | None = None, log_cap=1 << 14):
    """Full pass. Returns (rho, cost, stats dict, level logs, round logs)."""
    prm = prm or params_of(hg)
    off = np.ascontiguousarray(hg.off, np.int64)
    pins = np.ascontiguousarray(hg.pins, np.int32)
    w = np.ascontiguousarray(hg.w, np.int32)
    rho = np.empty(hg.V, np.int32)
    cost = C.c_int64()
    st = Stats()
    llog = (LevelLog * log_cap)()
    rlog = (RoundLog * log_cap)()
    nl, nr = C.c_int32(), C.c_int32()
    rc = lib().orc_partition(C.byref(prm), int(hg.V), int(off.shape[0] - 1), _ptr(off),
                             _ptr(pins), _ptr(w), _ptr(rho), C.byref(cost), C.byref(st),
                             llog, log_cap, C.byref(nl), rlog, log_cap, C.byref(nr))
    if rc != OK:
        raise OracleError(rc)
    stats = {f: getattr(st, f) for f, _ in Stats._fields_}
    levels = [{"V": g.V, "E": g.E, "P": g.P, "n_cand": g.n_cand, "n_pairs": g.n_pairs}
              for g in llog[:nl.value]]
    return rho, cost.value, stats, levels, [_round(r) for r in rlog[:nr.value]]


def place_trd(n_nodes, off, pins, eta, width, gamma) -> int:
    """Total residual distance of a placement (reading RP6)."""
    lib()
    off = np.ascontiguousarray(off, np.int64)
    pins = np.ascontiguousarray(pins, np.int32)
    eta = np.ascontiguousarray(eta, np.int64)
    gamma = np.ascontiguousarray(gamma, np.int32)
    return int(_lib.orc_place_trd(int(n_nodes), int(len(off) - 1), _ptr(off), _ptr(pins),
                                  _ptr(eta), int(width), _ptr(gamma)))


def place_refine(n_nodes, off, pins, eta, width, height, gamma, max_rounds=1000, log_cap=4096):
    """Swap refinement of a placement of G_P (Sec. 4.2; readings RP1-RP6).
    Returns (gamma, logs) with one dict per round."""
    lib()
    off = np.ascontiguousarray(off, np.int64)
    pins = np.ascontiguousarray(pins, np.int32)
    eta = np.ascontiguousarray(eta, np.int64)
    g = np.array(gamma, dtype=np.int32, copy=True)
    lp = np.zeros(log_cap, np.int32)
    ls = np.zeros(log_cap, np.int32)
    la = np.zeros(log_cap, np.int32)
    lg = np.zeros(log_cap, np.int64)
    r = _lib.orc_place_refine(int(n_nodes), int(len(off) - 1), _ptr(off), _ptr(pins), _ptr(eta),
                              int(width), int(height), _ptr(g), int(max_rounds), _ptr(lp),
                              _ptr(ls), _ptr(la), _ptr(lg), int(log_cap))
    if r < 0:
        raise OracleError(-r)
    logs = [{"props": int(lp[i]), "swaps": int(ls[i]), "applied": int(la[i]),
             "gain": int(lg[i])} for i in range(min(r, log_cap))]
    return g, logs


def hilbert_order(width, height):
    """Cores of a width x height lattice in Hilbert order (reading RI1)."""
    lib()
    out = np.zeros(max(width * height, 1), np.int32)
    rc = _lib.orc_hilbert_order(int(width), int(height), _ptr(out))
    if rc:
        raise OracleError(rc)
    return out[:width * height]


def initial_sequence(n_nodes, off, pins, eta, seq0):
    """Node order of one start of the initial placement (readings RI2-RI4)
    from the initial order seq0."""
    lib()
    off = np.ascontiguousarray(off, np.int64)
    pins = np.ascontiguousarray(pins, np.int32)
    eta = np.ascontiguousarray(eta, np.int64)
    seq = np.array(seq0, dtype=np.int32, copy=True)
    rc = _lib.orc_initial_sequence(int(n_nodes), int(len(off) - 1), _ptr(off), _ptr(pins),
                                   _ptr(eta), _ptr(seq))
    if rc:
        raise OracleError(rc)
    return seq


def initial_placement(n_nodes, off, pins, eta, width, height, seq0):
    """gamma of one start: the i-th node of the sequence on the i-th core in
    Hilbert order."""
    seq = initial_sequence(n_nodes, off, pins, eta, seq0)
    order = hilbert_order(width, height)
    gamma = np.zeros(n_nodes, np.int32)
    gamma[seq] = order[:n_nodes]
    return gamma
