"""Convenience layer over the C ABI: device tensors from torch, a handle
object that frees itself, and one-call partitioning."""
from __future__ import annotations

import numpy as np
import torch

from . import _native as N


def params_for(omega, delta, phi, max_levels=1024, max_refine_rounds=16,
               refine_nonpositive=0) -> N.Params:
    return N.Params(int(omega), int(delta), int(phi), int(max_levels), int(max_refine_rounds),
                    int(refine_nonpositive))


def to_device(hg, device="cuda"):
    """(off, pins, w) of a snngen.Hypergraph as device tensors."""
    off = torch.from_numpy(np.ascontiguousarray(hg.off, np.int64)).to(device)
    pins = torch.from_numpy(np.ascontiguousarray(hg.pins, np.int32)).to(device)
    w = torch.from_numpy(np.ascontiguousarray(hg.w, np.int32)).to(device)
    return off, pins, w


class HGraph:
    """Owns an snnmap handle built from device tensors."""

    def __init__(self, params, V, off, pins, w, stream=None):
        self.V = int(V)
        self.params = params
        self.stream = stream
        self._h = N.snnmap_build_hgraph(params, V, off.shape[0] - 1, off, pins, w, stream)

    @classmethod
    def from_hypergraph(cls, hg, params=None, device="cuda", stream=None, **kw):
        off, pins, w = to_device(hg, device)
        params = params or params_for(hg.omega, hg.delta, hg.phi, **kw)
        return cls(params, hg.V, off, pins, w, stream)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            N.snnmap_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def partition(self, rho_out=None):
        if rho_out is None:
            rho_out = torch.empty(self.V, dtype=torch.int32, device="cuda")
        cost, stats = N.snnmap_partition(self._h, rho_out, self.stream)
        return rho_out, cost, stats

    def coarsen_level(self):
        return N.snnmap_coarsen_level(self._h, self.stream)

    def contract(self):
        return N.snnmap_contract(self._h, self.stream)

    def num_levels(self):
        return N.snnmap_num_levels(self._h)

    def level_dims(self, level):
        return N.snnmap_level_dims(self._h, level)

    def level_arrays(self, level):
        """Copies of one level's arrays as host numpy arrays."""
        V, E, P = self.level_dims(level)
        dev = "cuda"
        t = {
            "off": torch.empty(E + 1, dtype=torch.int64, device=dev),
            "pins": torch.empty(max(P, 1), dtype=torch.int32, device=dev),
            "w": torch.empty(max(E, 1), dtype=torch.int64, device=dev),
            "k": torch.empty(max(E, 1), dtype=torch.int32, device=dev),
            "selfdst": torch.empty(max(E, 1), dtype=torch.uint8, device=dev),
            "size": torch.empty(max(V, 1), dtype=torch.int32, device=dev),
            "inpins": torch.empty(max(V, 1), dtype=torch.int32, device=dev),
            "in_count": torch.empty(max(V, 1), dtype=torch.int32, device=dev),
            "in_internal": torch.empty(max(V, 1), dtype=torch.int32, device=dev),
        }
        N.snnmap_level_copy(self._h, level, t["off"], t["pins"], t["w"], t["k"], t["selfdst"],
                            t["size"], t["inpins"], t["in_count"], t["in_internal"], self.stream)
        sizes = {"off": E + 1, "pins": P, "w": E, "k": E, "selfdst": E, "size": V, "inpins": V,
                 "in_count": V, "in_internal": V}
        out = {k: v.cpu().numpy()[:sizes[k]] for k, v in t.items()}
        out.update(V=V, E=E, P=P)
        return out

    def last_matching(self):
        V = self.level_dims(self.num_levels() - 1)[0]
        t = [torch.empty(max(V, 1), dtype=d, device="cuda")
             for d in (torch.int32, torch.int64, torch.int32, torch.int32)]
        N.snnmap_last_matching(self._h, *t, stream=self.stream)
        return [x.cpu().numpy()[:V] for x in t]

    def level_cid(self, level):
        V = self.level_dims(level)[0]
        t = torch.empty(max(V, 1), dtype=torch.int32, device="cuda")
        N.snnmap_level_cid(self._h, level, t, self.stream)
        return t.cpu().numpy()[:V]

    def trace(self, path, extra=None):
        """Appends this handle's trace to a JSONL file (write_trace): stage
        times (when profiling was on), one line per level and one per
        refinement round."""
        write_trace(path, self.stage_times(), self.level_logs(), self.round_logs(), extra)

    def dump_hierarchy(self, path):
        """Writes every level's arrays (level_arrays) and the cid maps between
        them to one .npz (save_hierarchy), for triage of a mismatch against
        the oracle offline."""
        n = self.num_levels()
        save_hierarchy(path, [self.level_arrays(l) for l in range(n)],
                       [self.level_cid(l) for l in range(n - 1)])

    def refine(self, level, n_parts, rho):
        return N.snnmap_refine(self._h, level, n_parts, rho, self.stream)

    def project(self, level, rho_coarse, rho_fine):
        N.snnmap_project(self._h, level, rho_coarse, rho_fine, self.stream)

    def round_logs(self):
        return N.snnmap_round_logs(self._h)

    def level_logs(self):
        return N.snnmap_level_logs(self._h)

    def partition_graph(self, rho, n_parts):
        """G_P of a level-0 partition (device tensor rho) as numpy arrays:
        dict(off, pins, eta, axons, internal)."""
        E, P, internal = N.snnmap_partition_graph(self._h, n_parts, rho, self.stream)
        off = torch.empty(E + 1, dtype=torch.int64, device="cuda")
        pins = torch.empty(max(P, 1), dtype=torch.int32, device="cuda")
        eta = torch.empty(max(E, 1), dtype=torch.int64, device="cuda")
        axons = torch.empty(max(E, 1), dtype=torch.int32, device="cuda")
        N.snnmap_partition_graph_copy(self._h, off, pins, eta, axons, self.stream)
        return {"off": off.cpu().numpy(), "pins": pins[:P].cpu().numpy(),
                "eta": eta[:E].cpu().numpy(), "axons": axons[:E].cpu().numpy(),
                "internal": internal}

    def set_row_budget(self, nbytes):
        """Bytes for refinement connection rows (-1 default, 0 none)."""
        N.snnmap_set_row_budget(self._h, nbytes)

    def set_level_budget(self, nbytes):
        N.snnmap_set_level_budget(self._h, nbytes)

    def set_coarsen_mode(self, mode):
        """0 auto, 1 full neighbour histograms, 2 carried candidates wherever
        possible (results never depend on it)."""
        N.snnmap_set_coarsen_mode(self._h, mode)

    def set_histogram_tiers(self, wwork=-1, bwork=-1, gwork=-1):
        """Work thresholds of the histogram tiers (results never depend on
        them; -1 keeps a value)."""
        N.snnmap_set_histogram_tiers(self._h, wwork, bwork, gwork)

    def profile(self, on=True):
        N.snnmap_profile(self._h, on)

    def stage_times(self):
        return N.snnmap_stage_times(self._h)

    def device_bytes(self):
        return N.snnmap_device_bytes(self._h)


def write_trace(path, stage_times, level_logs, round_logs, extra=None):
    """Appends one pass's trace to a JSONL file: a "pass" line (extra fields
    and the stage times: calls and ms per stage), then one "level" line per
    level (sizes, candidates, pairs, histogram pair terms) and one "round"
    line per refinement round (level, round, proposals, enacted prefix,
    gain). Returns the number of lines written."""
    import json
    lines = [dict({"kind": "pass", "stages": stage_times}, **(extra or {}))]
    lines += [dict({"kind": "level", "level": i}, **lv) for i, lv in enumerate(level_logs)]
    lines += [dict({"kind": "round"}, **r) for r in round_logs]
    with open(path, "a") as f:
        for line in lines:
            f.write(json.dumps(line) + "\n")
    return len(lines)


def save_hierarchy(path, levels, cids):
    """One .npz holding level dicts (as from HGraph.level_arrays) under keys
    L<l>_<name> and the cid map of level l (onto level l+1) as L<l>_cid."""
    arrays = {"n_levels": np.int64(len(levels))}
    for l, lv in enumerate(levels):
        for k, v in lv.items():
            arrays[f"L{l}_{k}"] = np.asarray(v)
    for l, c in enumerate(cids):
        arrays[f"L{l}_cid"] = np.asarray(c)
    np.savez_compressed(path, **arrays)


def load_hierarchy(path):
    """Inverse of save_hierarchy: (levels as dicts, cid maps)."""
    with np.load(path) as z:
        n = int(z["n_levels"])
        levels, cids = [], []
        for l in range(n):
            pre = f"L{l}_"
            d = {k[len(pre):]: z[k] for k in z.files if k.startswith(pre) and k != pre + "cid"}
            for k in ("V", "E", "P"):
                if k in d:
                    d[k] = int(d[k])
            levels.append(d)
            if pre + "cid" in z.files:
                cids.append(z[pre + "cid"])
    return levels, cids


def partition(hg, device="cuda", **kw):
    """One call: build from a snngen.Hypergraph, partition, return (rho numpy,
    cost, stats)."""
    g = HGraph.from_hypergraph(hg, device=device, **kw)
    try:
        rho, cost, stats = g.partition()
        return rho.cpu().numpy(), cost, stats
    finally:
        g.close()


def lattice_for(n_nodes):
    """The smallest near-square lattice (width, height) with at least
    n_nodes cores: width = ceil(sqrt(n)), height = ceil(n / width)."""
    width = max(1, int(np.ceil(np.sqrt(max(n_nodes, 1)))))
    return width, max(1, -(-int(n_nodes) // width))


def place(n_nodes, off, pins, eta, width=None, height=None, n_starts=64, seed=0,
          max_rounds=1000, stream=None):
    """Placement of G_P on a width x height lattice (Sec. 4.2): n_starts
    initial placements from random node orders (numpy PCG64 seeded by
    `seed`, one permutation per start, drawn here and passed to the
    library), all refined by swaps in the same launches, and the start with
    the smallest total residual distance kept (the lowest start on ties).
    off, pins, eta: G_P as numpy arrays or device tensors (e.g. from
    HGraph.partition_graph). Returns dict(gamma: numpy int32[n_nodes],
    trd, start, trds: per start after refinement, trds_initial, rounds,
    logs)."""
    K = int(n_nodes)
    if width is None or height is None:
        width, height = lattice_for(K)
    S = int(n_starts)

    def dev(a, dt):
        if isinstance(a, torch.Tensor):
            return a.to(device="cuda", dtype=dt).contiguous()
        return torch.from_numpy(np.ascontiguousarray(a).astype(
            np.int64 if dt == torch.int64 else np.int32)).cuda()

    d_off, d_pins, d_eta = dev(off, torch.int64), dev(pins, torch.int32), dev(eta, torch.int64)
    E = int(d_off.numel()) - 1
    rng = np.random.Generator(np.random.PCG64(seed))
    seq0 = np.concatenate([rng.permutation(K).astype(np.int32) for _ in range(S)]) if K else \
        np.zeros(0, np.int32)
    d_seq0 = torch.from_numpy(seq0).cuda()
    gamma = torch.zeros(S * K, dtype=torch.int32, device="cuda")
    N.snnmap_place_initial(K, E, d_off, d_pins, d_eta, width, height, S, d_seq0, gamma,
                           stream=stream)
    trds0 = N.snnmap_place_trd(K, E, d_off, d_pins, d_eta, width, height, S, gamma, stream)
    rounds, logs = N.snnmap_place_refine(K, E, d_off, d_pins, d_eta, width, height, S, gamma,
                                         max_rounds, stream, log_cap=max_rounds)
    best, trd, trds = N.snnmap_place_best(K, E, d_off, d_pins, d_eta, width, height, S, gamma,
                                          stream)
    g = gamma.view(S, K)[best].cpu().numpy() if K else np.zeros(0, np.int32)
    return {"gamma": g, "trd": trd, "start": best, "trds": trds, "trds_initial": trds0,
            "rounds": rounds, "logs": logs, "width": width, "height": height}
