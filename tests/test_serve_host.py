"""Host logic of the batched/served scheduler, run on the CPU through the
library's dry-run mode (worker threads hold their slot for a time instead of
touching a GPU): FIFO starts, slot limit, admission by footprint, release,
shutdown, batch order, and the footprint model."""
import ctypes as C

import numpy as np
import pytest

import paper_2609_07577_gb300 as P
from paper_2609_07577_gb300 import _native as N


def lib_or_skip():
    from paper_2609_07577_gb300 import _build
    try:
        _build.build()
    except RuntimeError as e:
        pytest.skip(f"cannot build here: {e}")
    return N.lib()


class HostJob:
    """A job over numpy host arrays: one hyperedge per vertex pair chain."""

    def __init__(self, V, pins_per_edge=2, omega=4):
        E = max(V - 1, 0)
        self.off = np.arange(E + 1, dtype=np.int64) * pins_per_edge
        self.pins = np.zeros(E * pins_per_edge, dtype=np.int32)
        self.w = np.ones(E, dtype=np.int32)
        self.rho = np.zeros(max(V, 1), dtype=np.int32)
        j = N.Job()
        j.params = P.params_for(omega, 4 * omega, 16 * omega)
        j.n_vertices, j.n_hedges = V, E
        j.offsets = self.off.ctypes.data
        j.pins = self.pins.ctypes.data
        j.w = self.w.ctypes.data
        j.rho_out = self.rho.ctypes.data
        j.on_host = 1
        self.job = j


def run_dry(sizes, slots, budget=0, us=2000, stagger_ms=0.0):
    s = N.snnmap_serve_create(slots, budget, us)
    jobs = [HostJob(v) for v in sizes]
    tickets = []
    try:
        for hj in jobs:
            tickets.append(N.snnmap_serve_submit(s, hj.job))
        for t in tickets:
            assert N.snnmap_serve_wait(s, t, 10_000.0)
        for t in tickets:
            N.snnmap_serve_release(s, t)
        q, r, b = N.snnmap_serve_info(s)
        assert (q, r, b) == (0, 0, 0)
    finally:
        N.snnmap_serve_destroy(s)
    return [hj.job for hj in jobs]


def overlap(a, b):
    return a.t_start_ms < b.t_end_ms and b.t_start_ms < a.t_end_ms


def test_footprint_model():
    lib_or_skip()
    f0 = N.snnmap_job_footprint(1000, 900, 20000)
    assert f0 > 20000 * 8
    assert N.snnmap_job_footprint(1000, 900, 40000) > f0
    assert N.snnmap_job_footprint(1000, 900, 20000, on_host=True) > f0
    with pytest.raises(N.SnnmapError):
        N.snnmap_job_footprint(-1, 0, 0)


def test_single_slot_runs_fifo_without_overlap():
    lib_or_skip()
    jobs = run_dry([50, 40, 30, 20, 10], slots=1)
    for a, b in zip(jobs, jobs[1:]):
        assert a.status == 0 and b.status == 0
        assert b.t_start_ms >= a.t_end_ms
        assert a.t_submit_ms <= b.t_submit_ms


def test_slots_bound_concurrency():
    lib_or_skip()
    jobs = run_dry([100] * 12, slots=4, us=20000)
    # at no instant do more than 4 jobs run
    events = sorted([(j.t_start_ms, 1) for j in jobs] + [(j.t_end_ms, -1) for j in jobs],
                    key=lambda e: (e[0], e[1]))
    live = peak = 0
    for _, d in events:
        live += d
        peak = max(peak, live)
    assert peak <= 4
    assert peak >= 2, "slots never overlapped"
    assert sorted({j.slot for j in jobs}) == [0, 1, 2, 3]


def test_admission_by_footprint():
    lib_or_skip()
    fp = N.snnmap_job_footprint(100, 99, 198, on_host=True)
    # budget for one job at a time: no two jobs overlap even with 4 slots
    jobs = run_dry([100] * 6, slots=4, budget=fp, us=5000)
    for i, a in enumerate(jobs):
        for b in jobs[i + 1:]:
            assert not overlap(a, b)
    # budget for two: never more than two at once
    jobs = run_dry([100] * 8, slots=4, budget=2 * fp, us=20000)
    events = sorted([(j.t_start_ms, 1) for j in jobs] + [(j.t_end_ms, -1) for j in jobs],
                    key=lambda e: (e[0], e[1]))
    live = peak = 0
    for _, d in events:
        live += d
        peak = max(peak, live)
    assert peak == 2


def test_oversized_job_runs_alone():
    lib_or_skip()
    small = N.snnmap_job_footprint(10, 9, 18, on_host=True)
    jobs = run_dry([10, 5000, 10], slots=4, budget=small * 2, us=5000)
    big = jobs[1]
    assert big.status == 0
    assert not overlap(big, jobs[0]) and not overlap(big, jobs[2])


def test_destroy_marks_queued_jobs():
    lib_or_skip()
    s = N.snnmap_serve_create(1, 0, 200000)
    jobs = [HostJob(10) for _ in range(4)]
    for hj in jobs:
        N.snnmap_serve_submit(s, hj.job)
    import time
    t0 = time.time()
    while N.snnmap_serve_info(s)[1] == 0 and time.time() - t0 < 10:
        time.sleep(0.001)       # until the first job runs
    N.snnmap_serve_destroy(s)
    st = [hj.job.status for hj in jobs]
    assert st[0] == 0
    assert all(x == N.ERR_STATE for x in st[1:]), st
    assert b"destroyed" in jobs[-1].job.error


def test_unknown_ticket_and_state_errors():
    lib_or_skip()
    s = N.snnmap_serve_create(1, 0, 1000)
    try:
        with pytest.raises(N.SnnmapError):
            N.snnmap_serve_wait(s, 12345, 0.0)
        with pytest.raises(N.SnnmapError):
            N.snnmap_serve_release(s, 12345)
        hj = HostJob(10)
        t = N.snnmap_serve_submit(s, hj.job)
        assert N.snnmap_serve_wait(s, t, 10_000.0)
        with pytest.raises(N.SnnmapError) as ei:
            N.snnmap_serve_hgraph(s, t)     # no hierarchy kept in a dry run
        assert ei.value.code == N.ERR_STATE
        N.snnmap_serve_release(s, t)
    finally:
        N.snnmap_serve_destroy(s)


def test_batch_runs_largest_first():
    lib_or_skip()
    sizes = [30, 300, 3, 3000, 30000]
    jobs = [HostJob(v) for v in sizes]
    arr = (N.Job * len(jobs))(*[hj.job for hj in jobs])
    rc = N.snnmap_batch_partition(arr, slots=1, dry_run_us=1000)
    assert rc == 0
    starts = [arr[i].t_start_ms for i in range(len(jobs))]
    order = sorted(range(len(jobs)), key=lambda i: starts[i])
    assert [sizes[i] for i in order] == sorted(sizes, reverse=True)
    assert all(arr[i].status == 0 for i in range(len(jobs)))


def test_bad_arguments():
    lib_or_skip()
    with pytest.raises(N.SnnmapError):
        N.snnmap_serve_create(-1, 0, 1000)
    s = N.snnmap_serve_create(1, 0, 1000)
    try:
        j = N.Job()
        j.n_vertices = -1
        with pytest.raises(N.SnnmapError):
            N.snnmap_serve_submit(s, j)
    finally:
        N.snnmap_serve_destroy(s)


def test_row_grant_counts_in_footprint():
    """A job's footprint is the model's plus any larger row grant (a quarter
    of the memory budget shared by the slots)."""
    lib_or_skip()
    base = N.snnmap_job_footprint(100, 99, 198, on_host=True)

    def fp(slots, budget):
        s = N.snnmap_serve_create(slots, budget, 1000)
        try:
            hj = HostJob(100)
            t = N.snnmap_serve_submit(s, hj.job)
            assert N.snnmap_serve_wait(s, t, 10_000.0)
            N.snnmap_serve_release(s, t)
            return hj.job.footprint
        finally:
            N.snnmap_serve_destroy(s)

    B = 1 << 34
    # both shares (2 GiB, 512 MiB) exceed the model's row budget of a tiny job
    assert fp(2, B) - fp(8, B) == B // 8 - B // 32
    assert fp(8, B) > base
    # a share below the model's row budget leaves the model's footprint
    assert fp(8, 1 << 20) == base
