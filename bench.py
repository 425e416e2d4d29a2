#!/usr/bin/env python3
"""Benchmark of the multilevel hypergraph partitioning pass on GB300.

Metric: pins processed per second by one full pass (level-0 build,
coarsening, contraction, uncoarsening with refinement) on a synthetic SNN
hypergraph, with the inputs resident in device memory; ms_per_step is the
end-to-end partition time. One JSON line on rank 0.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--config cfg2]
    python bench.py --impl reference ...   # the CPU oracle on a bounded sample

A single hypergraph does not shard across GPUs (every level needs global
histograms, matching and contraction), so N>1 runs N independent replicas
of the same job, one per GPU ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import snngen  # noqa: E402

METRIC = "pins/s per multilevel pass + end-to-end partition time (1 GB300)"
UNIT = "pins/s"
L2_BYTES = 129 * 2**20
# The CPU baseline and reference arm run the oracle on this bounded sample
# of the conv-like workload: same generator, receptive window, weights and
# core limits, 4 layers of 32x32x8 neurons.
SAMPLE = dict(layers=4, side=32, channels=8, nrand=4, seed=1, omega=1024, delta=4096, phi=16384)
SAMPLE_DESC = ("conv-like generator, 4 layers of 32x32x8 (32,768 neurons), cfg2's receptive "
               "window, weights and limits; full pass timed end to end")

CONFIGS = {
    "cfg1": ("Tiny feedforward SNN, 4x1024 neurons, 32-window + 8 random pins", snngen.cfg1),
    "cfg2": ("Conv-like layered SNN, 8 layers of 128x128x8 (1,048,576 neurons), 3x3x8 "
             "receptive window + 4 random pins", snngen.cfg2),
    "cfg3": ("Recurrent power-law SNN, 2^23 neurons, Pareto(2.1) fan-out on [8,16384]",
             snngen.cfg3),
    # quarter-width conv workload (profiling captures: inputs still larger than L2)
    "cfg2q": ("Conv-like layered SNN, 8 layers of 64x64x8 (262,144 neurons)",
              lambda: snngen.by_name("cfg2q")),
    "cfg4": ("Batched: independent jobs of 10k-500k neurons (log-uniform), layered and "
             "power-law generators alternating, seed = job index, Omega from {256,1024,4096}",
             None),
    "cfg5": ("Served: Poisson arrivals (200 jobs/s) of jobs of 10k-2M neurons (log-uniform), "
             "conv-like or power-law, admitted by HBM footprint", None),
    "place": ("Placement (Sec. 4.2) of the partition hypergraph G_P of the quarter-width conv "
              "workload's partition (8 layers of 64x64x8) on the smallest near-square lattice: "
              "64 starts, initial placement + swap refinement, best start by total residual "
              "distance", None),
}
BATCH_METRIC = "batched jobs/s (1 GB300)"
SERVE_METRIC = "served jobs/s with p50/p99 latency (1 GB300)"
PLACE_METRIC = "multi-start placements/s of G_P (64 starts, initial placement + swap refinement)"
PLACE_UNIT = "placements/s"
PLACE_STARTS = 64


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="cfg2", choices=sorted(CONFIGS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-clocks", action="store_true",
                    help="do not sample nvidia-smi (for runs under a profiler)")
    ap.add_argument("--jobs", type=int, default=0,
                    help="cfg4/cfg5: jobs in the sample (default 32 / 48)")
    ap.add_argument("--slots", type=int, default=8, help="cfg4/cfg5: concurrent jobs")
    ap.add_argument("--max-neurons", type=int, default=0,
                    help="cfg5: skip stream jobs larger than this (0: keep all)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks

CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    def __init__(self, gpu_id=None):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            self.p = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.p = None

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if r[5 + i].lower() in ("active", "0x1", "1")})
        power = [num(r[3]) for r in rows if num(r[3]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(power) if power else None}


def gpu_uuid(torch, dev):
    try:
        u = torch.cuda.get_device_properties(dev).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        return None


# ---------------------------------------------------------------------------
# algorithmic bytes per stage call (compulsory traffic: every array the
# stage needs read once, every output written once), from level sizes

def onchip_rate(pair_terms, hist_work, affinity_ms, ceiling):
    """Neighbour-histogram throughput beside its on-chip ceiling: the pair
    terms of the levels (sum of |e|(|e|-1), what a full histogram of every
    level would update) and the elements the level histograms actually
    visited (hist_work: carried levels visit fewer), per second of the
    affinity stage, against the measured rate of the same shared-memory
    table insert with no global memory traffic (snnmap_hist_ceiling). None
    without timing."""
    if not affinity_ms or affinity_ms <= 0:
        return None
    out = {"pair_updates_per_s": pair_terms / (affinity_ms / 1e3), "pair_updates": pair_terms,
           "elements_visited": hist_work,
           "elements_per_s": hist_work / (affinity_ms / 1e3), "affinity_ms": affinity_ms}
    if ceiling:
        out.update({"ceiling_updates_per_s": ceiling,
                    "frac": out["elements_per_s"] / ceiling,
                    "ceiling": "snnmap_hist_ceiling: block-tier table insert, 1024 distinct "
                               "keys per table, keys in registers"})
    return out


def traffic_record(stage, bytes_per_step):
    """DRAM traffic of the stage's dominant kernel from the committed ncu
    capture (profiles/roofline_traffic.json): measured bytes per algorithmic
    byte of the captured launch, scaled to the step's algorithmic bytes.
    None when there is no capture for the stage or the kernel's sources have
    changed since it was taken (their sha256 is recorded with it)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None, None
    if rec.get("stage") != stage:
        return None, None
    h = hashlib.sha256()
    for rel in rec.get("sources", []):
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    if h.hexdigest() != rec.get("sources_sha256"):
        return None, "kernel changed since the capture"
    ratio = rec["dram_bytes"] / rec["algorithmic_bytes"]
    return ratio * bytes_per_step, rec.get("kernel")


def stage_bytes(stage, lv):
    V, E, P = lv["V"], lv["E"], lv["P"]
    if stage == "affinity":
        # pins + incidence lists, offsets, hyperedge weight/k/selfdst,
        # vertex state in, candidate/score/shared out
        return 4 * P + 4 * P + 8 * (V + 1) + 8 * (E + 1) + 13 * E + 12 * V + 16 * V
    if stage == "incidence":
        return 4 * P + 4 * P + 8 * (V + 1)
    if stage == "pincount":
        return 4 * P + 4 * P + 8 * (E + 1) + 13 * E + 16 * V
    if stage == "gains":
        return 4 * P + 8 * (V + 1) + 8 * (E + 1) + 13 * E + 12 * P + 16 * V
    if stage == "contract":
        return 4 * P + 4 * P + 8 * (E + 1) + 13 * E + 28 * V
    if stage == "match":
        return 16 * V
    return None


# ---------------------------------------------------------------------------

def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def host_cpu():
    """The host's logical CPU count and CPU model (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu model")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"cpus": os.cpu_count(), "model": model}


class PinnedToOneCore:
    """Runs the enclosed code with the calling thread pinned to one core (the
    last one it may use), restoring its affinity afterwards; the oracle is
    single-threaded and runs in the calling thread."""

    def __enter__(self):
        self.saved = None
        self.cpu = None
        if hasattr(os, "sched_getaffinity"):
            try:
                self.saved = os.sched_getaffinity(0)
                self.cpu = max(self.saved)
                os.sched_setaffinity(0, {self.cpu})
            except OSError:
                self.saved = None
                self.cpu = None
        return self

    def __exit__(self, *exc):
        if self.saved is not None:
            os.sched_setaffinity(0, self.saved)
        return False


def cpu_baseline(warm=0, steps=1):
    """The oracle (single-threaded C) on the bounded sample, pinned to one
    core; pins/s."""
    import oracle
    hg = snngen.conv(**SAMPLE, name="cfg2-sample")
    oracle.build()
    times = []
    with PinnedToOneCore() as pin:
        for _ in range(warm):
            oracle.partition(hg)
        for _ in range(steps):
            t0 = time.perf_counter()
            oracle.partition(hg)
            times.append(time.perf_counter() - t0)
    t = statistics.median(times)
    host = host_cpu()
    return {"value": hg.P / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{SAMPLE_DESC}; P={hg.P}; {t:.2f} s per pass (median of {steps})",
            "s_per_pass": t, "pins": hg.P, "pinned_cpu": pin.cpu,
            "host_cpus": host["cpus"], "host_model": host["model"]}


def place_baseline(budget_s=10.0):
    """The oracle on a bounded sample of the placement workload: whole
    starts (initial placement + swap refinement) on the G_P of the
    scaled-down conv workload's partition, as many as fit budget_s; value =
    64-start placements/s at that rate."""
    import oracle
    hg = snngen.by_name("cfg2s")
    oracle.build()
    rho, _, st, *_ = oracle.partition(hg, oracle.params_of(hg))
    K = int(st["n_parts"])
    gp = oracle.Level.from_hypergraph(hg, oracle.params_of(hg)).partition_graph(rho)
    width = int(math.ceil(math.sqrt(K)))
    height = -(-K // width)
    rng = np.random.Generator(np.random.PCG64(0))
    with PinnedToOneCore():
        n, t0 = 0, time.perf_counter()
        while n < PLACE_STARTS and (n == 0 or time.perf_counter() - t0 < budget_s):
            g0 = oracle.initial_placement(K, gp["off"], gp["pins"], gp["eta"], width, height,
                                          rng.permutation(K))
            oracle.place_refine(K, gp["off"], gp["pins"], gp["eta"], width, height, g0)
            n += 1
        per_start = (time.perf_counter() - t0) / n
    return {"value": 1.0 / (per_start * PLACE_STARTS), "unit": PLACE_UNIT, "cores": 1,
            "kind": "oracle",
            "sample": (f"{n} whole starts on the G_P of the 8192-neuron conv workload's partition "
                       f"(K={K}, {len(gp['pins'])} pins; the timed workload's G_P is beyond the "
                       f"oracle's label propagation); {per_start:.2f} s per start, scaled to 64 "
                       f"starts"),
            "s_per_placement": per_start * PLACE_STARTS}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.config == "place":
        cb = place_baseline()
        line = {"impl": "reference", "metric": PLACE_METRIC, "value": cb["value"],
                "unit": PLACE_UNIT, "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": cb["s_per_placement"] * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int64", "data": "synthetic",
                "config": {"workload": "place", "description": CONFIGS["place"][0],
                           "sample": cb["sample"]},
                "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
                "e2e": {"value": cb["value"], "unit": PLACE_UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    cfg_desc = CONFIGS[args.config][0]
    cb = cpu_baseline(warm=args.warmup, steps=args.steps)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": cb["s_per_pass"] * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": args.config, "description": cfg_desc,
                       "sample": cb["sample"]},
            "cpu_baseline": {"value": cb["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": cb["sample"], "pinned_cpu": cb["pinned_cpu"],
                             "host_cpus": cb["host_cpus"], "host_model": cb["host_model"]},
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    import paper_2609_07577_gb300 as P
    from paper_2609_07577_gb300 import HGraph, params_for

    desc, gen = CONFIGS[args.config]
    hg = gen()
    params = params_for(hg.omega, hg.delta, hg.phi)
    off = torch.from_numpy(hg.off).to(dev)
    pins = torch.from_numpy(hg.pins).to(dev)
    w = torch.from_numpy(hg.w).to(dev)
    rho = torch.empty(hg.V, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(profile=False):
        g = HGraph(params, hg.V, off, pins, w, stream)
        try:
            if profile:
                g.profile(True)
            cost, stats = P.snnmap_partition(g.handle, rho, stream)
            st = g.stage_times() if profile else None
            lv = g.level_logs() if profile else None
            rl = g.round_logs() if profile else None
        finally:
            g.close()
        return cost, stats, st, lv, rl

    for _ in range(args.warmup):
        cost, stats, _, _, _ = step()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    sampler = None if args.no_clocks else ClockSampler(gpu_uuid(torch, local))
    time.sleep(0.3)
    barrier()
    l0 = P.snnmap_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stage_acc = {}
    for _ in range(args.steps):
        cost, stats, st, lv, rl = step(profile=True)
        for k, v in st.items():
            a = stage_acc.setdefault(k, {"calls": 0, "ms": 0.0})
            a["calls"] += v["calls"]
            a["ms"] += v["ms"]
    e1.record(stream)
    barrier()
    launches = P.snnmap_launch_count() - l0
    clocks = sampler.stop() if sampler else {"sm_mhz": None, "sm_max_mhz": None,
                                             "reasons": ["not sampled"]}
    ms = e0.elapsed_time(e1) / args.steps
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * hg.P / (ms / 1e3)

    # dominant stage and its roofline (HBM-bound formulas; algorithmic bytes
    # summed over the levels / rounds the stage ran on in one pass)
    peak, peak_kind = load_peaks()
    per_step = {k: {"calls": v["calls"] / args.steps, "ms": v["ms"] / args.steps}
                for k, v in stage_acc.items()}
    dom = max(per_step, key=lambda k: per_step[k]["ms"])
    levels = lv
    rounds_per_level = {}
    for r in rl:
        rounds_per_level[r["level"]] = rounds_per_level.get(r["level"], 0) + 1
    def bytes_of(stage):
        tot = 0
        for i, g in enumerate(levels):
            b = stage_bytes(stage, g)
            if b is None:
                return None
            if stage in ("affinity", "match"):
                tot += b
            elif stage in ("pincount", "gains"):
                tot += b * rounds_per_level.get(i, 0)
            elif stage in ("contract", "incidence"):
                tot += b if i + 1 < len(levels) else 0
        return tot
    dom_bytes = bytes_of(dom)
    roof = None
    if dom_bytes is not None and per_step[dom]["ms"] > 0:
        calls = per_step[dom]["calls"]
        achieved = dom_bytes / (per_step[dom]["ms"] / 1e3) / 1e9
        traffic, tnote = traffic_record(dom, dom_bytes)
        # the histogram stages are limited on chip (shared-memory table
        # updates, L2 latency), not by HBM: frac is how far below the HBM
        # copy roof they run; "onchip" holds the fraction of their own ceiling
        roof = {"bound": "onchip" if dom in ("affinity", "gains", "rows") else "hbm",
                "kernel_stage": dom, "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
                "traffic": traffic, "traffic_source": tnote, "bytes_per_step": dom_bytes,
                "launches_per_step": calls, "ms_per_step": per_step[dom]["ms"]}
    pair_terms = sum(g["pair_terms"] for g in levels)
    hist_work = sum(g.get("hist_work", 0) for g in levels)
    try:
        ceiling = P.snnmap_hist_ceiling(1024, 64, stream)
    except Exception:
        ceiling = None

    # end to end through the host-buffer entry point (pinned host memory)
    e2e_s = None
    if args.e2e_steps > 0:
        h_off = torch.from_numpy(hg.off).pin_memory()
        h_pins = torch.from_numpy(hg.pins).pin_memory()
        h_w = torch.from_numpy(hg.w).pin_memory()
        h_rho = torch.empty(hg.V, dtype=torch.int32).pin_memory()
        P.snnmap_partition_host(params, hg.V, hg.E, h_off, h_pins, h_w, h_rho, stream)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            c2, _ = P.snnmap_partition_host(params, hg.V, hg.E, h_off, h_pins, h_w, h_rho, stream)
        barrier()
        e2e_s = (time.perf_counter() - t0) / args.e2e_steps
        assert c2 == cost, (c2, cost)
        if world > 1:
            t = torch.tensor([e2e_s], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())

    cb = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(steps=3)   # median of three passes, ~13 s of one core
        cb = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample", "pinned_cpu",
                                 "host_cpus", "host_model")}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64", "data": "synthetic",
            "config": {"workload": args.config, "description": desc, "V": hg.V, "E": hg.E,
                       "P": hg.P, "omega": hg.omega, "delta": hg.delta, "phi": hg.phi,
                       "parallelism": f"replicas{world}",
                       "l2": f"inputs ({(hg.P * 4 + hg.E * 12) / 2**20:.0f} MiB) larger than L2",
                       "levels": stats["levels"], "partitions": stats["nonempty_parts"],
                       "cost": cost, "pins_all_levels": stats["pins_total"],
                       "pair_terms_all_levels": pair_terms},
            "stage_ms_per_step": {k: round(v["ms"], 3) for k, v in per_step.items()},
            "roofline": roof,
            "onchip": onchip_rate(pair_terms, hist_work, per_step.get("affinity", {}).get("ms"),
                                  ceiling),
            "cpu_baseline": cb,
            "e2e": None if e2e_s is None else {
                "value": world * hg.P / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": 8 * (hg.E + 1) + 4 * hg.P + 4 * hg.E,
                "d2h_bytes_per_step": 4 * hg.V, "s_per_step": e2e_s},
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _dist_setup():
    import torch
    import torch.distributed as dist
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    return rank, world, local


def _max_over_ranks(x, world, local):
    """Slowest rank's value (NCCL on the rank's GPU when N > 1)."""
    from paper_2609_07577_gb300.shard import max_over_ranks
    return x if world == 1 else max_over_ranks(x, device=f"cuda:{local}")


def _barrier(world, local):
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize(torch.device("cuda", local))


def run_batch(args):
    """cfg4: every rank partitions its share of the jobs (job j on rank
    j % N, no collective) in one batched call; timed against the same jobs
    run one at a time (one slot)."""
    import torch
    rank, world, local = _dist_setup()
    import __graft_entry__
    __graft_entry__.build()
    import paper_2609_07577_gb300 as P
    from paper_2609_07577_gb300 import JobBuffers
    from paper_2609_07577_gb300.shard import rank_jobs
    n_jobs = args.jobs or 32
    mine = rank_jobs(n_jobs, rank, world)
    t0 = time.perf_counter()
    hgs = [snngen.batch_jobs_one(j) for j in mine]
    gen_s = time.perf_counter() - t0
    dev_bufs = [JobBuffers(hg, on_host=False) for hg in hgs]
    host_bufs = [JobBuffers(hg, on_host=True) for hg in hgs]

    def batch(bufs, slots):
        arr = (P.Job * len(bufs))(*[b.job for b in bufs])
        rc = P.snnmap_batch_partition(arr, slots)
        assert rc == 0, (rc, [arr[i].error for i in range(len(bufs)) if arr[i].status])
        return [(arr[i].cost, arr[i].stats.levels, arr[i].peak_bytes, arr[i].footprint)
                for i in range(len(bufs))]

    # warm-up: the smallest jobs of this rank's share (kernel loading, pools)
    small = sorted(dev_bufs, key=lambda b: b.hg.P)[:max(1, min(8, len(dev_bufs)))]
    for _ in range(args.warmup):
        batch(small, args.slots)
    sampler = None if args.no_clocks else ClockSampler(gpu_uuid(torch, local))
    time.sleep(0.3)
    _barrier(world, local)
    l0 = P.snnmap_launch_count()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        res = batch(dev_bufs, args.slots)
    _barrier(world, local)
    t_batch = (time.perf_counter() - t0) / args.steps
    launches = P.snnmap_launch_count() - l0
    clocks = sampler.stop() if sampler else {"sm_mhz": None, "sm_max_mhz": None,
                                             "reasons": ["not sampled"]}
    t_batch = _max_over_ranks(t_batch, world, local)
    # one job at a time, same jobs
    t0 = time.perf_counter()
    ser = batch(dev_bufs, 1)
    _barrier(world, local)
    t_serial = _max_over_ranks(time.perf_counter() - t0, world, local)
    assert [r[0] for r in ser] == [r[0] for r in res], "batched costs differ from serial"
    # end to end: host inputs and results, copies inside the timed region
    t0 = time.perf_counter()
    eres = batch(host_bufs, args.slots)
    _barrier(world, local)
    t_e2e = _max_over_ranks(time.perf_counter() - t0, world, local)
    assert [r[0] for r in eres] == [r[0] for r in res]
    if rank == 0:
        pins = sum(hg.P for hg in hgs) * world
        line = {
            "metric": BATCH_METRIC, "value": n_jobs / t_batch, "unit": "jobs/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_batch * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": "cfg4", "description": CONFIGS["cfg4"][0], "jobs": n_jobs,
                       "slots": args.slots, "parallelism": f"jobs sharded over {world} GPU(s)",
                       "neurons_rank0": sum(hg.V for hg in hgs), "pins_rank0": sum(hg.P for hg in hgs),
                       "warmup_jobs": "the 8 smallest jobs of the rank's share per warm-up step",
                       "gen_s_rank0": round(gen_s, 1),
                       "l2": "every job's inputs are read once per pass; no flush"},
            "serial": {"value": n_jobs / t_serial, "unit": "jobs/s", "s": t_serial,
                       "speedup_batched": t_serial / t_batch},
            "pins_per_s": pins / t_batch,
            "peak_over_footprint_max": max(r[2] / r[3] for r in res),
            "e2e": {"value": n_jobs / t_e2e, "unit": "jobs/s",
                    "h2d_bytes_per_step": sum(8 * (hg.E + 1) + 4 * hg.P + 4 * hg.E for hg in hgs) * world,
                    "d2h_bytes_per_step": sum(4 * hg.V for hg in hgs) * world},
            "gpu_launches": launches, "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_serve(args):
    """cfg5: replay a Poisson arrival stream into a server (jobs admitted by
    footprint as slots free up); latency = completion - arrival. Compared
    with the same stream served one job at a time."""
    import torch
    rank, world, local = _dist_setup()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2609_07577_gb300 import JobBuffers, Server
    n_jobs = args.jobs or 48
    stream = snngen.serve_stream(n_jobs)
    if args.max_neurons:
        stream = [d for d in stream if d["n"] <= args.max_neurons]
    from paper_2609_07577_gb300.shard import rank_jobs
    mine = [stream[i] for i in rank_jobs(len(stream), rank, world)]
    t0 = time.perf_counter()
    bufs = [JobBuffers(snngen.serve_job(d), on_host=True) for d in mine]
    gen_s = time.perf_counter() - t0
    t_arr = [d["t"] for d in mine]

    def replay(slots):
        with Server(slots=slots) as S:
            base = time.perf_counter()
            tickets = []
            for b, ta in zip(bufs, t_arr):
                dt = ta - (time.perf_counter() - base)
                if dt > 0:
                    time.sleep(dt)
                tickets.append((S.submit_buffers(b), ta))
            t_sub0 = None
            out = []
            for t, ta in tickets:
                r = S.wait(t)
                assert r["status"] == 0, r["error"]
                out.append(r)
            # latency from the scheduled arrival: the server clock starts at
            # creation, just before `base`
            lat = [r["t_end_ms"] / 1e3 - ta for r, (_, ta) in zip(out, tickets)]
            span = max(r["t_end_ms"] for r in out) / 1e3
            for t, _ in tickets:
                S.release(t)
        return out, lat, span

    # warm-up: the smallest job, alone
    small = min(bufs, key=lambda b: b.hg.P)
    for _ in range(args.warmup):
        with Server(slots=1) as S:
            S.wait(S.submit_buffers(small))
    sampler = None if args.no_clocks else ClockSampler(gpu_uuid(torch, local))
    _barrier(world, local)
    out, lat, span = replay(args.slots)
    clocks = sampler.stop() if sampler else {"sm_mhz": None, "sm_max_mhz": None,
                                             "reasons": ["not sampled"]}
    out1, lat1, span1 = replay(1)
    assert [r["cost"] for r in out] == [r["cost"] for r in out1], "served costs differ from serial"
    span = _max_over_ranks(span, world, local)
    span1 = _max_over_ranks(span1, world, local)
    if rank == 0:
        q = lambda xs, p: float(np.percentile(np.array(xs) * 1e3, p))
        line = {
            "metric": SERVE_METRIC, "value": len(stream) / span, "unit": "jobs/s",
            "n_gpus": world, "steps": 1, "warmup": args.warmup, "ms_per_step": span * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": "cfg5", "description": CONFIGS["cfg5"][0],
                       "jobs": len(stream), "slots": args.slots, "rate_jobs_per_s": 200.0,
                       "max_neurons": args.max_neurons or None,
                       "neurons_rank0": sum(b.hg.V for b in bufs),
                       "pins_rank0": sum(b.hg.P for b in bufs), "gen_s_rank0": round(gen_s, 1),
                       "parallelism": f"jobs sharded over {world} GPU(s)",
                       "inputs": "pinned host memory, copied in and out by the server"},
            "latency_ms": {"p50": q(lat, 50), "p99": q(lat, 99), "max": q(lat, 100)},
            "serial": {"value": len(stream) / span1, "unit": "jobs/s",
                       "latency_ms": {"p50": q(lat1, 50), "p99": q(lat1, 99)}},
            "e2e": {"value": len(stream) / span, "unit": "jobs/s",
                    "h2d_bytes_per_step": sum(8 * (b.hg.E + 1) + 4 * b.hg.P + 4 * b.hg.E for b in bufs) * world,
                    "d2h_bytes_per_step": sum(4 * b.hg.V for b in bufs) * world},
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_place(args):
    """Placement of a G_P in the size range of the paper's (16 to 1.7k
    nodes; cfg2's own has about 4.5k): the quarter-width conv workload is
    partitioned once (untimed setup);
    each step is one 64-start placement (paper_2609_07577_gb300.place) on
    device-resident G_P arrays; e2e repeats it from host arrays."""
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2609_07577_gb300 as P
    from paper_2609_07577_gb300 import HGraph

    hg = snngen.by_name("cfg2q")
    G = HGraph.from_hypergraph(hg, device=dev)
    try:
        rho, _, st = G.partition()
        K = int(st["n_parts"])
        gp = G.partition_graph(rho, K)
    finally:
        G.close()
    E, Pgp = len(gp["eta"]), len(gp["pins"])
    d = {k: torch.from_numpy(np.ascontiguousarray(gp[k])).to(dev) for k in ("off", "pins", "eta")}
    width, height = P.lattice_for(K)

    def step(i, arrays):
        return P.place(K, arrays["off"], arrays["pins"], arrays["eta"], width, height,
                       n_starts=PLACE_STARTS, seed=i)

    for i in range(args.warmup):
        res = step(i, d)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    sampler = None if args.no_clocks else ClockSampler(gpu_uuid(torch, local))
    time.sleep(0.3)
    barrier()
    l0 = P.snnmap_launch_count()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        res = step(args.warmup + i, d)
    e1.record(stream)
    barrier()
    launches = P.snnmap_launch_count() - l0
    clocks = sampler.stop() if sampler else {"sm_mhz": None, "sm_max_mhz": None,
                                             "reasons": ["not sampled"]}
    ms = e0.elapsed_time(e1) / args.steps
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())

    e2e_s = None
    if args.e2e_steps > 0:
        barrier()
        t0 = time.perf_counter()
        for i in range(args.e2e_steps):
            step(i, gp)
        barrier()
        e2e_s = (time.perf_counter() - t0) / args.e2e_steps
        if world > 1:
            t = torch.tensor([e2e_s], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())

    cb = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = place_baseline()
        cb = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
    if rank == 0:
        line = {
            "metric": PLACE_METRIC, "value": world / (ms / 1e3), "unit": PLACE_UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": "place", "description": CONFIGS["place"][0], "K": K,
                       "hyperedges": E, "pins": Pgp, "width": width, "height": height,
                       "starts": PLACE_STARTS, "parallelism": f"replicas{world}",
                       "l2": "G_P fits L2: placement kernels run from L1/L2",
                       "trd_best": res["trd"],
                       "trd_initial_best": min(res["trds_initial"])},
            "roofline": None,
            "roofline_note": "placement kernels not yet captured with ncu",
            "cpu_baseline": cb,
            "e2e": None if e2e_s is None else {
                "value": world / e2e_s, "unit": PLACE_UNIT,
                "h2d_bytes_per_step": 8 * (E + 1) + 4 * Pgp + 8 * E + 4 * PLACE_STARTS * K,
                "d2h_bytes_per_step": 4 * K, "s_per_step": e2e_s},
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "place":
        run_place(args)
    elif args.config == "cfg4":
        run_batch(args)
    elif args.config == "cfg5":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
