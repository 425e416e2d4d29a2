"""ctypes binding of libsnnmap (include/snnmap.h): the same entry points,
argument marshalling only. Every step of the partitioning pass runs in the
library's CUDA kernels; there is no Python or CPU fallback, and loading
fails loudly if the library has not been built."""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsnnmap.so")

OK, ERR_INVALID, ERR_INFEASIBLE, ERR_OOM, ERR_DEVICE_TIMEOUT, ERR_CUDA, ERR_STATE = range(7)


class Params(C.Structure):
    _fields_ = [("omega", C.c_int32), ("delta", C.c_int32), ("phi", C.c_int32),
                ("max_levels", C.c_int32), ("max_refine_rounds", C.c_int32),
                ("refine_nonpositive", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("levels", C.c_int32), ("n_parts", C.c_int32), ("nonempty_parts", C.c_int32),
                ("rounds", C.c_int32), ("moves", C.c_int64), ("cost_initial", C.c_int64),
                ("cost", C.c_int64), ("pins_total", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class RoundLog(C.Structure):
    _fields_ = [("level", C.c_int32), ("round", C.c_int32), ("n_props", C.c_int32),
                ("istar", C.c_int32), ("n_active", C.c_int32), ("rows", C.c_int32),
                ("gain", C.c_int64)]


class LevelLog(C.Structure):
    _fields_ = [("V", C.c_int32), ("E", C.c_int32), ("P", C.c_int64), ("n_cand", C.c_int32),
                ("n_pairs", C.c_int32), ("pair_terms", C.c_int64), ("n_block", C.c_int32),
                ("n_global", C.c_int32), ("carried", C.c_int32), ("n_full", C.c_int32),
                ("hist_work", C.c_int64)]


class StageTime(C.Structure):
    _fields_ = [("name", C.c_char_p), ("calls", C.c_int64), ("ms", C.c_double)]


class Job(C.Structure):
    """snnmap_job: one independent mapping job of the batched/served forms."""
    _fields_ = [("params", Params), ("n_vertices", C.c_int32), ("n_hedges", C.c_int32),
                ("offsets", C.c_void_p), ("pins", C.c_void_p), ("w", C.c_void_p),
                ("rho_out", C.c_void_p), ("on_host", C.c_int32), ("keep_hierarchy", C.c_int32),
                ("status", C.c_int32), ("slot", C.c_int32), ("cost", C.c_int64),
                ("stats", Stats), ("footprint", C.c_int64), ("peak_bytes", C.c_int64),
                ("t_submit_ms", C.c_double), ("t_start_ms", C.c_double),
                ("t_end_ms", C.c_double), ("error", C.c_char * 128)]


class ServeOpts(C.Structure):
    _fields_ = [("slots", C.c_int32), ("dry_run_us", C.c_int32), ("mem_budget", C.c_int64)]


class PlaceLog(C.Structure):
    """snnmap_place_log: one round of placement swap refinement."""
    _fields_ = [("props", C.c_int32), ("swaps", C.c_int32), ("applied", C.c_int32),
                ("reserved", C.c_int32), ("gain", C.c_int64)]


class SnnmapError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"snnmap error {code}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()

# name -> (restype, argtypes)
_vp, _i32, _i64 = C.c_void_p, C.c_int32, C.c_int64
_SIGS = {
    "snnmap_default_params": (Params, [_i32, _i32, _i32]),
    "snnmap_build_hgraph": (C.c_int, [C.POINTER(Params), _i32, _i32, _vp, _vp, _vp, _vp,
                                      C.POINTER(_vp)]),
    "snnmap_coarsen_level": (C.c_int, [_vp, _vp, C.POINTER(_i32), C.POINTER(_i32)]),
    "snnmap_contract": (C.c_int, [_vp, _vp, C.POINTER(_i32), C.POINTER(_i32), C.POINTER(_i64)]),
    "snnmap_num_levels": (C.c_int, [_vp, C.POINTER(_i32)]),
    "snnmap_level_dims": (C.c_int, [_vp, _i32, C.POINTER(_i32), C.POINTER(_i32), C.POINTER(_i64)]),
    "snnmap_project": (C.c_int, [_vp, _i32, _vp, _vp, _vp]),
    "snnmap_refine": (C.c_int, [_vp, _i32, _i32, _vp, _vp, C.POINTER(_i64)]),
    "snnmap_partition": (C.c_int, [_vp, _vp, _vp, C.POINTER(_i64), C.POINTER(Stats)]),
    "snnmap_connectivity": (C.c_int, [_vp, _i32, _vp, _vp, C.POINTER(_i64)]),
    "snnmap_partition_host": (C.c_int, [C.POINTER(Params), _i32, _i32, _vp, _vp, _vp, _vp,
                                        C.POINTER(_i64), C.POINTER(Stats), _vp]),
    "snnmap_level_copy": (C.c_int, [_vp, _i32] + [_vp] * 9 + [_vp]),
    "snnmap_last_matching": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "snnmap_level_cid": (C.c_int, [_vp, _i32, _vp, _vp]),
    "snnmap_round_logs": (C.c_int, [_vp, _vp, _i32, C.POINTER(_i32)]),
    "snnmap_level_logs": (C.c_int, [_vp, _vp, _i32, C.POINTER(_i32)]),
    "snnmap_device_bytes": (C.c_int, [_vp, C.POINTER(_i64)]),
    "snnmap_profile": (C.c_int, [_vp, _i32]),
    "snnmap_stage_times": (C.c_int, [_vp, _vp, _i32, C.POINTER(_i32)]),
    "snnmap_launch_count": (_i64, []),
    "snnmap_set_level_budget": (C.c_int, [_vp, _i64]),
    "snnmap_set_row_budget": (C.c_int, [_vp, _i64]),
    "snnmap_set_coarsen_mode": (C.c_int, [_vp, _i32]),
    "snnmap_hist_ceiling": (C.c_int, [_i32, _i32, _vp, C.POINTER(C.c_double)]),
    "snnmap_set_histogram_tiers": (C.c_int, [_vp, _i64, _i64, _i64]),
    "snnmap_set_tier_table": (C.c_int, [_i32, _vp, _vp, _vp, _vp]),
    "snnmap_partition_graph": (C.c_int, [_vp, _i32, _vp, _vp, C.POINTER(_i32), C.POINTER(_i64),
                                         C.POINTER(_i64)]),
    "snnmap_partition_graph_copy": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "snnmap_connectivity_noalloc": (C.c_int, [_i32, _i32, _vp, _vp, _vp, _vp, _i32, _vp, _vp]),
    "snnmap_peak_bytes": (C.c_int, [_vp, C.POINTER(_i64)]),
    "snnmap_job_footprint": (C.c_int, [_i32, _i32, _i64, _i32, C.POINTER(_i64)]),
    "snnmap_serve_create": (C.c_int, [C.POINTER(ServeOpts), C.POINTER(_vp)]),
    "snnmap_serve_submit": (C.c_int, [_vp, C.POINTER(Job), C.POINTER(_i64)]),
    "snnmap_serve_wait": (C.c_int, [_vp, _i64, C.c_double, C.POINTER(_i32)]),
    "snnmap_serve_hgraph": (C.c_int, [_vp, _i64, C.POINTER(_vp)]),
    "snnmap_serve_release": (C.c_int, [_vp, _i64]),
    "snnmap_serve_info": (C.c_int, [_vp, C.POINTER(_i32), C.POINTER(_i32), C.POINTER(_i64)]),
    "snnmap_serve_destroy": (C.c_int, [_vp]),
    "snnmap_batch_partition": (C.c_int, [C.POINTER(Job), _i32, C.POINTER(ServeOpts)]),
    "snnmap_place_refine": (C.c_int, [_i32, _i32, _vp, _vp, _vp, _i32, _i32, _i32, _vp, _i32,
                                      _vp, _vp, _vp, _i32]),
    "snnmap_place_trd": (C.c_int, [_i32, _i32, _vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp, _vp]),
    "snnmap_place_best": (C.c_int, [_i32, _i32, _vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp,
                                    C.POINTER(_i32), C.POINTER(_i64), _vp]),
    "snnmap_place_initial": (C.c_int, [_i32, _i32, _vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp,
                                       _vp, _vp]),
    "snnmap_hilbert_order": (C.c_int, [_i32, _i32, _vp, _vp]),
    "snnmap_free": (None, [_vp]),
    "snnmap_last_error": (C.c_char_p, []),
}


def lib():
    """Loads libsnnmap.so; raises if it is missing (build it first). On first
    load, installs the autotuned histogram tier table if the package has one
    (autotune.load_table)."""
    global _lib
    fresh = False
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build the CUDA library first "
                    "(python -c 'import __graft_entry__ as g; g.build()')")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
            fresh = True
    if fresh:
        from .autotune import load_table
        load_table()
    return _lib


def check(rc):
    if rc != OK:
        raise SnnmapError(rc, lib().snnmap_last_error().decode())
    return rc


def _p(x):
    """Device pointer of a torch tensor, or an int address, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


# --- the C entry points under their own names --------------------------------

def snnmap_default_params(omega, delta, phi):
    return lib().snnmap_default_params(int(omega), int(delta), int(phi))


def snnmap_build_hgraph(params, n_vertices, n_hedges, d_offsets, d_pins, d_w, stream=None):
    h = C.c_void_p()
    check(lib().snnmap_build_hgraph(C.byref(params), int(n_vertices), int(n_hedges), _p(d_offsets),
                                    _p(d_pins), _p(d_w), _stream(stream), C.byref(h)))
    return h


def snnmap_coarsen_level(h, stream=None):
    nc, npairs = C.c_int32(), C.c_int32()
    check(lib().snnmap_coarsen_level(h, _stream(stream), C.byref(nc), C.byref(npairs)))
    return nc.value, npairs.value


def snnmap_contract(h, stream=None):
    V, E, P = C.c_int32(), C.c_int32(), C.c_int64()
    check(lib().snnmap_contract(h, _stream(stream), C.byref(V), C.byref(E), C.byref(P)))
    return V.value, E.value, P.value


def snnmap_num_levels(h):
    n = C.c_int32()
    check(lib().snnmap_num_levels(h, C.byref(n)))
    return n.value


def snnmap_level_dims(h, level):
    V, E, P = C.c_int32(), C.c_int32(), C.c_int64()
    check(lib().snnmap_level_dims(h, int(level), C.byref(V), C.byref(E), C.byref(P)))
    return V.value, E.value, P.value


def snnmap_project(h, level, d_rho_coarse, d_rho_fine, stream=None):
    check(lib().snnmap_project(h, int(level), _p(d_rho_coarse), _p(d_rho_fine), _stream(stream)))


def snnmap_refine(h, level, n_parts, d_rho, stream=None):
    c = C.c_int64()
    check(lib().snnmap_refine(h, int(level), int(n_parts), _p(d_rho), _stream(stream), C.byref(c)))
    return c.value


def snnmap_partition(h, d_rho_out, stream=None):
    c = C.c_int64()
    st = Stats()
    check(lib().snnmap_partition(h, _stream(stream), _p(d_rho_out), C.byref(c), C.byref(st)))
    return c.value, st.as_dict()


def snnmap_connectivity(h, n_parts, d_rho, stream=None):
    c = C.c_int64()
    check(lib().snnmap_connectivity(h, int(n_parts), _p(d_rho), _stream(stream), C.byref(c)))
    return c.value


def snnmap_partition_host(params, n_vertices, n_hedges, h_offsets, h_pins, h_w, h_rho_out,
                          stream=None):
    """Host buffers: numpy arrays or pinned torch CPU tensors (int64/int32)."""
    def hp(a):
        if a is None:
            return None
        if hasattr(a, "ctypes"):
            return a.ctypes.data
        return a.data_ptr()
    c = C.c_int64()
    st = Stats()
    check(lib().snnmap_partition_host(C.byref(params), int(n_vertices), int(n_hedges),
                                      hp(h_offsets), hp(h_pins), hp(h_w), hp(h_rho_out),
                                      C.byref(c), C.byref(st), _stream(stream)))
    return c.value, st.as_dict()


def snnmap_level_copy(h, level, d_off=None, d_pins=None, d_w=None, d_k=None, d_selfdst=None,
                      d_size=None, d_inpins=None, d_in_count=None, d_in_internal=None,
                      stream=None):
    check(lib().snnmap_level_copy(h, int(level), _p(d_off), _p(d_pins), _p(d_w), _p(d_k),
                                  _p(d_selfdst), _p(d_size), _p(d_inpins), _p(d_in_count),
                                  _p(d_in_internal), _stream(stream)))


def snnmap_last_matching(h, d_cand=None, d_cscore=None, d_cov=None, d_match=None, stream=None):
    check(lib().snnmap_last_matching(h, _p(d_cand), _p(d_cscore), _p(d_cov), _p(d_match),
                                     _stream(stream)))


def snnmap_level_cid(h, level, d_cid, stream=None):
    check(lib().snnmap_level_cid(h, int(level), _p(d_cid), _stream(stream)))


def snnmap_round_logs(h):
    n = C.c_int32()
    check(lib().snnmap_round_logs(h, None, 0, C.byref(n)))
    buf = (RoundLog * max(1, n.value))()
    check(lib().snnmap_round_logs(h, buf, n.value, C.byref(n)))
    return [{f: getattr(buf[i], f) for f, _ in RoundLog._fields_} for i in range(n.value)]


def snnmap_level_logs(h):
    n = C.c_int32()
    check(lib().snnmap_level_logs(h, None, 0, C.byref(n)))
    buf = (LevelLog * max(1, n.value))()
    check(lib().snnmap_level_logs(h, buf, n.value, C.byref(n)))
    return [{f: getattr(buf[i], f) for f, _ in LevelLog._fields_} for i in range(n.value)]


def snnmap_device_bytes(h):
    b = C.c_int64()
    check(lib().snnmap_device_bytes(h, C.byref(b)))
    return b.value


def snnmap_profile(h, on):
    check(lib().snnmap_profile(h, 1 if on else 0))


def snnmap_stage_times(h):
    n = C.c_int32()
    buf = (StageTime * 32)()
    check(lib().snnmap_stage_times(h, buf, 32, C.byref(n)))
    return {buf[i].name.decode(): {"calls": buf[i].calls, "ms": buf[i].ms} for i in range(n.value)}


def snnmap_connectivity_noalloc(n_vertices, n_hedges, d_offsets, d_pins, d_w, d_rho, n_parts,
                                d_cost_out, stream=None):
    """Allocation-free connectivity; the result lands in d_cost_out (device)."""
    check(lib().snnmap_connectivity_noalloc(int(n_vertices), int(n_hedges), _p(d_offsets),
                                            _p(d_pins), _p(d_w), _p(d_rho), int(n_parts),
                                            _p(d_cost_out), _stream(stream)))


def snnmap_set_level_budget(h, nbytes):
    check(lib().snnmap_set_level_budget(h, int(nbytes)))


def snnmap_peak_bytes(h):
    b = C.c_int64()
    check(lib().snnmap_peak_bytes(h, C.byref(b)))
    return b.value


def snnmap_job_footprint(n_vertices, n_hedges, n_pins, on_host=False):
    b = C.c_int64()
    check(lib().snnmap_job_footprint(int(n_vertices), int(n_hedges), int(n_pins),
                                     1 if on_host else 0, C.byref(b)))
    return b.value


def snnmap_serve_create(slots=0, mem_budget=0, dry_run_us=0):
    o = ServeOpts(int(slots), int(dry_run_us), int(mem_budget))
    s = C.c_void_p()
    check(lib().snnmap_serve_create(C.byref(o), C.byref(s)))
    return s


def snnmap_serve_submit(s, job):
    """job: a Job struct the caller keeps alive (with its buffers) until done."""
    t = C.c_int64()
    check(lib().snnmap_serve_submit(s, C.byref(job), C.byref(t)))
    return t.value


def snnmap_serve_wait(s, ticket, timeout_ms=-1.0):
    d = C.c_int32()
    check(lib().snnmap_serve_wait(s, int(ticket), float(timeout_ms), C.byref(d)))
    return bool(d.value)


def snnmap_serve_hgraph(s, ticket):
    h = C.c_void_p()
    check(lib().snnmap_serve_hgraph(s, int(ticket), C.byref(h)))
    return h


def snnmap_serve_release(s, ticket):
    check(lib().snnmap_serve_release(s, int(ticket)))


def snnmap_serve_info(s):
    q, r, b = C.c_int32(), C.c_int32(), C.c_int64()
    check(lib().snnmap_serve_info(s, C.byref(q), C.byref(r), C.byref(b)))
    return q.value, r.value, b.value


def snnmap_serve_destroy(s):
    check(lib().snnmap_serve_destroy(s))


def snnmap_batch_partition(jobs, slots=0, mem_budget=0, dry_run_us=0):
    """jobs: a ctypes array of Job. Returns the library's return code (job
    statuses are in the structs)."""
    o = ServeOpts(int(slots), int(dry_run_us), int(mem_budget))
    return lib().snnmap_batch_partition(jobs, len(jobs), C.byref(o))


def snnmap_partition_graph(h, n_parts, d_rho, stream=None):
    """Computes G_P; returns (n_hedges, n_pins, internal_weight)."""
    e, p, w = C.c_int32(), C.c_int64(), C.c_int64()
    check(lib().snnmap_partition_graph(h, int(n_parts), _p(d_rho), _stream(stream), C.byref(e),
                                       C.byref(p), C.byref(w)))
    return e.value, p.value, w.value


def snnmap_partition_graph_copy(h, d_offsets=None, d_pins=None, d_eta=None, d_axons=None,
                                stream=None):
    check(lib().snnmap_partition_graph_copy(h, _p(d_offsets), _p(d_pins), _p(d_eta), _p(d_axons),
                                            _stream(stream)))


def snnmap_place_refine(n_nodes, n_hedges, d_offsets, d_pins, d_eta, width, height, n_starts,
                        d_gamma, max_rounds, stream=None, log_cap=0):
    """Refines n_starts placements of G_P in d_gamma (device int32[n_starts *
    n_nodes]) in place; returns (rounds per start, logs per start as lists
    of dicts, up to log_cap rounds each)."""
    S = int(n_starts)
    rounds = (C.c_int32 * max(S, 1))()
    cap = max(int(log_cap), 0)
    logs = (PlaceLog * max(S * cap, 1))()
    check(lib().snnmap_place_refine(int(n_nodes), int(n_hedges), _p(d_offsets), _p(d_pins),
                                    _p(d_eta), int(width), int(height), S, _p(d_gamma),
                                    int(max_rounds), _stream(stream), rounds,
                                    logs if cap else None, cap))
    out = []
    for i in range(S):
        n = min(rounds[i], cap)
        out.append([{"props": L.props, "swaps": L.swaps, "applied": L.applied, "gain": L.gain}
                    for L in logs[i * cap:i * cap + n]])
    return [rounds[i] for i in range(S)], out


def snnmap_place_trd(n_nodes, n_hedges, d_offsets, d_pins, d_eta, width, height, n_starts,
                     d_gamma, stream=None):
    """Total residual distance of each start's placement (list of ints)."""
    S = int(n_starts)
    out = (C.c_int64 * max(S, 1))()
    check(lib().snnmap_place_trd(int(n_nodes), int(n_hedges), _p(d_offsets), _p(d_pins),
                                 _p(d_eta), int(width), int(height), S, _p(d_gamma),
                                 _stream(stream), out))
    return [out[i] for i in range(S)]


def snnmap_place_best(n_nodes, n_hedges, d_offsets, d_pins, d_eta, width, height, n_starts,
                      d_gamma, stream=None):
    """The start of smallest total residual distance (lowest on ties):
    (start, its distance, every start's distance as a list)."""
    S = int(n_starts)
    out = (C.c_int64 * max(S, 1))()
    best, trd = C.c_int32(), C.c_int64()
    check(lib().snnmap_place_best(int(n_nodes), int(n_hedges), _p(d_offsets), _p(d_pins),
                                  _p(d_eta), int(width), int(height), S, _p(d_gamma),
                                  _stream(stream), C.byref(best), C.byref(trd), out))
    return best.value, trd.value, [out[i] for i in range(S)]


def snnmap_place_initial(n_nodes, n_hedges, d_offsets, d_pins, d_eta, width, height, n_starts,
                         d_seq0, d_gamma_out, d_seq_out=None, stream=None):
    """Initial placements of n_starts starts from their initial orders
    d_seq0 (device int32[n_starts * n_nodes]) into d_gamma_out (and the
    final sequences into d_seq_out if given)."""
    check(lib().snnmap_place_initial(int(n_nodes), int(n_hedges), _p(d_offsets), _p(d_pins),
                                     _p(d_eta), int(width), int(height), int(n_starts),
                                     _p(d_seq0), _p(d_seq_out), _p(d_gamma_out),
                                     _stream(stream)))


def snnmap_hilbert_order(width, height, d_order_out, stream=None):
    """Cores of a width x height lattice in Hilbert order (device int32)."""
    check(lib().snnmap_hilbert_order(int(width), int(height), _p(d_order_out), _stream(stream)))


def snnmap_set_row_budget(h, nbytes):
    check(lib().snnmap_set_row_budget(h, int(nbytes)))


def snnmap_hist_ceiling(distinct_keys=1024, rounds=64, stream=None):
    """On-chip ceiling of the neighbour-histogram insert (updates/s)."""
    r = C.c_double()
    check(lib().snnmap_hist_ceiling(int(distinct_keys), int(rounds), _stream(stream),
                                    C.byref(r)))
    return r.value


def snnmap_set_coarsen_mode(h, mode):
    check(lib().snnmap_set_coarsen_mode(h, int(mode)))


def snnmap_set_tier_table(rows):
    """rows: [(max_pins, wwork, bwork, gwork), ...] in increasing max_pins
    (empty: built-in defaults)."""
    n = len(rows)
    arr = [(C.c_int64 * max(n, 1))(*[int(r[i]) for r in rows]) for i in range(4)]
    check(lib().snnmap_set_tier_table(n, *[C.cast(a, C.c_void_p) for a in arr]))


def snnmap_set_histogram_tiers(h, wwork=-1, bwork=-1, gwork=-1):
    check(lib().snnmap_set_histogram_tiers(h, int(wwork), int(bwork), int(gwork)))


def snnmap_launch_count():
    return int(lib().snnmap_launch_count())


def snnmap_free(h):
    if h:
        lib().snnmap_free(h)


def snnmap_last_error():
    return lib().snnmap_last_error().decode()
