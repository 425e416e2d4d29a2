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
}


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


def cpu_baseline(warm=0, steps=1):
    """The oracle (single-threaded C) on the bounded sample; pins/s."""
    import oracle
    hg = snngen.conv(**SAMPLE, name="cfg2-sample")
    oracle.build()
    for _ in range(warm):
        oracle.partition(hg)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        oracle.partition(hg)
        times.append(time.perf_counter() - t0)
    t = statistics.median(times)
    return {"value": hg.P / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{SAMPLE_DESC}; P={hg.P}; {t:.2f} s per pass",
            "s_per_pass": t, "pins": hg.P}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
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
                             "sample": cb["sample"]},
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
        roof = {"bound": "hbm", "kernel_stage": dom, "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
                "traffic": None, "bytes_per_step": dom_bytes, "launches_per_step": calls,
                "ms_per_step": per_step[dom]["ms"]}
    pair_terms = sum(g["pair_terms"] for g in levels)

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
        cb = cpu_baseline()
        cb = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}

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


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
