"""Batched and served forms over the C ABI (snnmap_serve_*,
snnmap_batch_partition): job structs whose buffers stay alive while the
library's worker threads run them, and results read back as numpy."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native as N
from .api import params_for


class JobBuffers:
    """One job: the Job struct plus the tensors its pointers refer to.

    on_host=True keeps inputs and the result in pinned host memory (the
    library copies them in and out on the job's own stream); False puts them
    on the device first."""

    def __init__(self, hg, params=None, on_host=True, keep_hierarchy=False, device="cuda"):
        self.hg = hg
        self.params = params or params_for(hg.omega, hg.delta, hg.phi)
        off = torch.from_numpy(np.ascontiguousarray(hg.off, np.int64))
        pins = torch.from_numpy(np.ascontiguousarray(hg.pins, np.int32))
        w = torch.from_numpy(np.ascontiguousarray(hg.w, np.int32))
        if on_host:
            self.off, self.pins, self.w = off.pin_memory(), pins.pin_memory(), w.pin_memory()
            self.rho = torch.empty(hg.V, dtype=torch.int32).pin_memory()
        else:
            self.off, self.pins, self.w = off.to(device), pins.to(device), w.to(device)
            self.rho = torch.empty(hg.V, dtype=torch.int32, device=device)
        self.job = N.Job()
        j = self.job
        j.params = self.params
        j.n_vertices = int(hg.V)
        j.n_hedges = int(self.off.shape[0] - 1)
        j.offsets = self.off.data_ptr()
        j.pins = self.pins.data_ptr()
        j.w = self.w.data_ptr()
        j.rho_out = self.rho.data_ptr()
        j.on_host = 1 if on_host else 0
        j.keep_hierarchy = 1 if keep_hierarchy else 0

    def result(self):
        j = self.job
        rho = self.rho.cpu().numpy() if self.rho.is_cuda else self.rho.numpy().copy()
        return {"status": j.status, "error": j.error.decode(), "rho": rho, "cost": j.cost,
                "stats": j.stats.as_dict(), "slot": j.slot, "footprint": j.footprint,
                "peak_bytes": j.peak_bytes, "t_submit_ms": j.t_submit_ms,
                "t_start_ms": j.t_start_ms, "t_end_ms": j.t_end_ms}


class Server:
    """A continuous-batching server: jobs are admitted as slots and memory
    free up, and run concurrently on the slots' streams."""

    def __init__(self, slots=8, mem_budget=0, dry_run_us=0):
        self._s = N.snnmap_serve_create(slots, mem_budget, dry_run_us)
        self._jobs = {}

    def submit(self, hg, params=None, on_host=True, keep_hierarchy=False):
        jb = JobBuffers(hg, params, on_host, keep_hierarchy)
        t = N.snnmap_serve_submit(self._s, jb.job)
        self._jobs[t] = jb
        return t

    def submit_buffers(self, jb):
        t = N.snnmap_serve_submit(self._s, jb.job)
        self._jobs[t] = jb
        return t

    def wait(self, ticket, timeout_ms=-1.0):
        """Result dict once done (None on timeout)."""
        if not N.snnmap_serve_wait(self._s, ticket, timeout_ms):
            return None
        return self._jobs[ticket].result()

    def hgraph(self, ticket):
        return N.snnmap_serve_hgraph(self._s, ticket)

    def release(self, ticket):
        N.snnmap_serve_release(self._s, ticket)
        self._jobs.pop(ticket, None)

    def info(self):
        return N.snnmap_serve_info(self._s)

    def close(self):
        if getattr(self, "_s", None):
            N.snnmap_serve_destroy(self._s)
            self._s = None
            self._jobs.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_partition(hgs, slots=8, on_host=False, mem_budget=0, buffers=None):
    """Partitions every hypergraph of `hgs` in one batched call; returns
    (return code, list of result dicts in input order). `buffers` may pass
    prepared JobBuffers to keep their setup out of a timed region."""
    bufs = buffers or [JobBuffers(hg, on_host=on_host) for hg in hgs]
    arr = (N.Job * len(bufs))(*[b.job for b in bufs])
    rc = N.snnmap_batch_partition(arr, slots, mem_budget)
    for b, j in zip(bufs, arr):
        ctypes.memmove(ctypes.addressof(b.job), ctypes.addressof(j), ctypes.sizeof(j))
    return rc, [b.result() for b in bufs]
