"""Several-rank path on the CPU: two gloo ranks deal the jobs round-robin,
run their shares through the batch scheduler (dry-run mode: no GPU), and
agree on the slowest rank's time and the total work; the shares are
disjoint and cover every job."""
import os
import socket

import pytest
import torch.multiprocessing as mp

N_JOBS = 11


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import numpy as np
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2609_07577_gb300 import _native as N
    from paper_2609_07577_gb300.shard import rank_jobs, max_over_ranks, sum_over_ranks
    mine = rank_jobs(N_JOBS, rank, world)
    keep = []
    jobs = []
    for j in mine:
        V = 10 + 5 * j
        off = np.arange(V, dtype=np.int64) * 2
        pins = np.zeros(2 * (V - 1), np.int32)
        w = np.ones(V - 1, np.int32)
        rho = np.zeros(V, np.int32)
        keep += [off, pins, w, rho]
        jb = N.Job()
        jb.params = N.Params(4, 16, 64, 1024, 16)
        jb.n_vertices, jb.n_hedges = V, V - 1
        jb.offsets, jb.pins, jb.w, jb.rho_out = off.ctypes.data, pins.ctypes.data, w.ctypes.data, rho.ctypes.data
        jb.on_host = 1
        jobs.append(jb)
    arr = (N.Job * len(jobs))(*jobs)
    rc = N.snnmap_batch_partition(arr, slots=2, dry_run_us=500) if jobs else 0
    span = max((arr[i].t_end_ms for i in range(len(jobs))), default=0.0)
    t = max_over_ranks(span)
    total = sum_over_ranks(len(mine))
    got = [None] * world
    dist.all_gather_object(got, mine)
    out.put((rank, rc, span, t, total, got))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_and_agree():
    from paper_2609_07577_gb300 import _build
    try:
        _build.build()
    except RuntimeError as e:
        pytest.skip(f"cannot build here: {e}")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    spans = [r[2] for r in res]
    for rank, rc, span, t, total, got in res:
        assert rc == 0
        assert t == max(spans)
        assert total == N_JOBS
        flat = sorted(j for part in got for j in part)
        assert flat == list(range(N_JOBS))
        assert set(got[0]).isdisjoint(got[1])


def test_rank_jobs_arguments():
    from paper_2609_07577_gb300.shard import rank_jobs
    assert rank_jobs(5, 0, 1) == [0, 1, 2, 3, 4]
    assert rank_jobs(5, 1, 2) == [1, 3]
    with pytest.raises(ValueError):
        rank_jobs(5, 2, 2)
