#!/usr/bin/env python3
"""Throughput of the PIC/MCC hot path (arXiv 2109.04469 §2 steps 1-6) on GB300.

One "step" is one pass of the whole per-timestep path (field solve, particle pass with
gather/push/walls/MCC/deposit, compaction) over the synthetic workload
``ccp_1pa_300v_400c``: 2.5 cm argon CCP, 1 Pa, 300 V, 13.56 MHz, 400 cells,
dt = T_RF/3000, 2e6 superparticles per species, R = 0.2, gamma = 0.1.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank runs an independent replica
(instance = rank): weak scaling, no data-path collective.  ``--impl reference`` times the FP64
CPU oracle (the checker, plain C, one thread) on the same workload and metric.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (push+MCC+deposit), FP32/batched vs FP64 plain; % of HBM peak"
UNIT = "particle-steps/s"
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 256 << 20
PROFILE_DIR = os.path.join(ROOT, "profiles")
PUSH_SOURCES = ("paper_2109_04469_gb300/csrc/pic_fp64.cu", "paper_2109_04469_gb300/csrc/pic_dev.cuh")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default="ccp_1pa_300v_400c")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-steps", type=int, default=30)
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def source_hash(paths) -> str:
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, if the kernel source is unchanged."""
    path = os.path.join(PROFILE_DIR, f"{kernel}_{workload}.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_sha256_16") != source_hash(PUSH_SOURCES):
        return None
    try:
        return float(vals["dram_bytes_per_launch_full_workload"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.out = None

    def start(self):
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        self.out.flush()
        self.out.seek(0)
        sm, smax, reasons, power = [], [], set(), []
        for line in self.out.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for name, flag in zip(self.NAMES, parts[4:8]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.out.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_baseline(cfg: dict, steps: int) -> dict:
    """The FP64 oracle as it stands, one thread, on the full workload for a bounded window."""
    from oracle import oracle as O

    sim = O.OracleSim(cfg)
    sim.step(2)
    n0 = sim.count(0) + sim.count(1)
    t = time.perf_counter()
    parts = 0
    for _ in range(steps):
        parts += sim.count(0) + sim.count(1)
        sim.step(1)
    dt = time.perf_counter() - t
    return {"value": parts / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{cfg.get('name', '')} full population ({n0} superparticles), {steps} "
                      f"steps after 2 warm-up steps, plain C FP64, 1 thread, {dt:.1f} s"}


def run_reference(args, cfg):
    rank, _, world = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O

    est_s_per_step = 4e6 * 2.5e-8
    budget = 150.0
    scale = min(1.0, budget / max(1e-9, (args.steps + args.warmup) * est_s_per_step))
    c = dict(cfg)
    if scale < 1.0:
        c["init_per_species"] = max(1000, int(cfg["init_per_species"] * scale))
    sim = O.OracleSim(c)
    sim.step(args.warmup)
    parts = 0
    t = time.perf_counter()
    for _ in range(args.steps):
        parts += sim.count(0) + sim.count(1)
        sim.step(1)
    el = time.perf_counter() - t
    v = parts / el
    sample = (f"{args.workload}: {c['init_per_species']} initial superparticles per species, "
              f"{args.warmup} warm-up + {args.steps} timed steps, plain C FP64, 1 thread")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "particles_per_species": c["init_per_species"],
                       "n_cells": c["n_cells"], "precision": "fp64"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    from paper_2109_04469_gb300 import workloads

    cfg = workloads.params(args.workload)
    cfg["name"] = args.workload
    if args.impl == "reference":
        run_reference(args, cfg)
        return
    import torch

    rank, local_rank, world = dist_env()
    assert world == args.gpus or world == 1, "launch N>1 with torchrun --nproc-per-node N"
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    from paper_2109_04469_gb300 import pic

    cfg["instance"] = rank  # independent replica per rank
    pcfg = {k: v for k, v in cfg.items() if k != "name"}
    sim = pic.Simulation(pcfg)
    stream = sim.stream
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    sim.step(args.warmup)
    sim.sync()
    c0 = sim.accum()["counters"].astype(np.int64)
    d = sim.derived()
    try:
        uuid = str(torch.cuda.get_device_properties(local_rank).uuid)
        uuid = uuid if uuid.startswith("GPU-") else f"GPU-{uuid}"
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    ms2 = np.zeros(2)  # particle pass, compaction (+ next field solve beside it)
    step_ms = 0.0
    parts = 0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(k)  # L2 flush between timed steps (outside the events)
            ne, ni = sim.counts()
            parts += ne + ni
            ev0.record(stream)
            sim.step_profiled(1, ms2)
            ev1.record(stream)
            ev1.synchronize()
            step_ms += ev0.elapsed_time(ev1)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    # the field solve on its own (it runs beside the compaction inside each step)
    field_ms = 0.0
    with torch.cuda.stream(stream):
        for k in range(10):
            ev0.record(stream)
            sim.solve_field()
            ev1.record(stream)
            ev1.synchronize()
            field_ms += ev0.elapsed_time(ev1) / 10
    status = sim.status()
    c1 = sim.accum()["counters"].astype(np.int64)
    dc = c1 - c0
    # algorithmic bytes of the particle pass (per particle-step: x, vx r/w + id read = 36 B;
    # candidates r/w vy, vz 32 B; removed and born particles move one 36 B record)
    turnover = int(dc[0] + dc[1] + dc[2] + dc[3] + 2 * dc[8] + dc[5])
    alg_bytes = 36.0 * parts + 32.0 * float(dc[11] + dc[12]) + 36.0 * turnover
    total_ms = step_ms
    total_parts = parts
    if dist:
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        p = torch.tensor([float(total_parts)], dtype=torch.float64, device="cuda")
        dist.all_reduce(p, op=dist.ReduceOp.SUM)
        total_parts = int(p.item())
    value = total_parts / (total_ms / 1e3)
    push_ms = ms2[0] / args.steps
    compact_ms = ms2[1] / args.steps
    peak, peak_src = measured_peak()
    achieved = (alg_bytes / args.steps) / (push_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": peak_src,
            "traffic": profiled_traffic("push_fp64", args.workload),
            "kernel": "k_push_fp64", "alg_bytes_per_launch": alg_bytes / args.steps,
            "launch_ms": push_ms}

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(sim, args, torch)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "particles_per_species": cfg["init_per_species"],
                       "n_cells": cfg["n_cells"], "steps_per_rf": cfg["steps_per_rf"],
                       "precision": "fp64", "parallelism": f"replicas x{world}",
                       "l2": "flushed (256 MiB write) between timed steps"},
            "roofline": roof,
            "kernel_ms_per_step": {"particles": push_ms, "compaction_and_next_field": compact_ms,
                                   "field_alone": field_ms},
            "poisson_share": field_ms / (total_ms / args.steps),
            "compaction_share": compact_ms / (total_ms / args.steps),
            "gpu_launches": 2 * args.steps,
            "clocks": clocks, "status": status}
    if e2e:
        line["e2e"] = e2e
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(pcfg | {"name": args.workload}, args.cpu_steps)
    if rank == 0:
        print(json.dumps(line), flush=True)
    sim.close()
    if dist:
        dist.destroy_process_group()


def run_e2e(sim, args, torch):
    """End to end through the C-ABI with host buffers: each step uploads the particle state
    from pinned host memory (pic_set_particles), advances one step (pic_step) and reads the
    diagnostics back (pic_diag)."""
    host = []
    h2d = 0
    for s in (0, 1):
        p = sim.particles(s)
        pinned = {}
        for k, a in p.items():
            t = torch.empty(a.shape, dtype=torch.float64 if a.dtype == np.float64 else torch.int32,
                            pin_memory=True)
            arr = t.numpy().view(a.dtype)
            arr[...] = a
            pinned[k] = (t, arr)
        host.append(pinned)
        h2d += len(p["x"]) * 36
    nx = sim.nx
    c = sim.cfg
    d2h = 8 * (2 * nx + c["eepf_bins"] + 2 * c["fedf_bins"] + 16) + 72
    parts = 0
    times = []
    for _ in range(args.e2e_steps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        for s in (0, 1):
            a = host[s]
            n = len(a["x"][1])
            sim.set_particles(s, a["x"][1], a["vx"][1], a["vy"][1], a["vz"][1], a["id"][1], n)
        sim.step(1)
        sim.diag()
        times.append(time.perf_counter() - t)
        parts += len(host[0]["x"][1]) + len(host[1]["x"][1])
    total = sum(times)
    return {"value": parts / total, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "steps": args.e2e_steps,
            "note": "wall clock per step: H2D of the full particle state from pinned memory, "
                    "one step, pic_diag read-back"}


if __name__ == "__main__":
    main()
