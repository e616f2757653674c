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

  python bench.py --profile-case fp32|fp64|ens|mlp

runs one small, self-contained case of a kernel family (a few launches) and exits: the
command lines that the ncu summaries under profiles/ were taken with.
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
PUSH_SOURCES = ("paper_2109_04469_gb300/csrc/pic_fp64.cu", "paper_2109_04469_gb300/csrc/pic_dev.cuh",
                "paper_2109_04469_gb300/csrc/pic_common.cuh")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default="ccp_1pa_300v_400c")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-stress", action="store_true")
    ap.add_argument("--stress-steps", type=int, default=10)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-steps", type=int, default=100)
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--ensemble-members", type=int, default=64)
    ap.add_argument("--ensemble-steps", type=int, default=20,
                    help="timed ensemble steps (members grow from their uniform load; the "
                         "capacity of workloads.ensemble_members holds about 45 steps)")
    ap.add_argument("--ensemble-warmup", type=int, default=3)
    ap.add_argument("--profile-case", choices=("fp32", "fp64", "ens", "mlp"), default=None)
    ap.add_argument("--precisions", default="fp32,fp64",
                    help="comma list; the first is the headline, the others are reported beside it")
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


def profiled_value(kernel: str, workload: str, key: str):
    """A figure from a committed ncu summary (profiles/<kernel>_<workload>.txt), if the sources
    it was taken on are unchanged (their hash is recorded in the summary)."""
    path = os.path.join(PROFILE_DIR, f"{kernel}_{workload}.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    srcs = tuple(s.strip() for s in vals.get("sources", ",".join(PUSH_SOURCES)).split(","))
    if vals.get("source_sha256_16") != source_hash(srcs):
        return None
    try:
        return float(vals[key].split()[0])
    except (KeyError, ValueError, IndexError):
        return None


def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, if the kernel source is unchanged."""
    return profiled_value(kernel, workload, "dram_bytes_per_launch_full_workload")


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


BAD_CLOCK_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def clocks_rejected(c: dict) -> bool:
    """A timed region whose clock samples show a hardware or thermal slowdown, or an SM clock
    well below its maximum with no reason given (a leftover clock lock), is not kept
    (sw_power_cap is kept and noted)."""
    if any(r in c.get("reasons", []) for r in BAD_CLOCK_REASONS):
        return True
    sm, smax = c.get("sm_mhz"), c.get("sm_max_mhz")
    return bool(sm and smax and sm < 0.9 * smax and not c.get("reasons"))


def cpu_baseline(cfg: dict, steps: int, warmup: int = 2) -> dict:
    """The FP64 oracle as it stands, one thread, on the full workload for a bounded window."""
    from oracle import oracle as O

    sim = O.OracleSim(cfg)
    sim.step(warmup)
    n0 = sim.count(0) + sim.count(1)
    t = time.perf_counter()
    parts = 0
    for _ in range(steps):
        parts += sim.count(0) + sim.count(1)
        sim.step(1)
    dt = time.perf_counter() - t
    return {"value": parts / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{cfg.get('name', '')} full population ({n0} superparticles), {steps} "
                      f"steps after {warmup} warm-up steps, plain C FP64, 1 thread, {dt:.1f} s"}


def ensemble_cpu_baseline(members: int, budget_s: float = 10.0) -> dict:
    """The oracle on the batched scan: one member per host core, all cores stepping their
    member concurrently (the C oracle releases the interpreter lock), for about budget_s of
    wall time; the aggregate particle-steps/s over all threads.  The members are spread over
    the scan (every members/cores-th one), so the sample mixes its sizes and pressures."""
    import os
    import threading

    from oracle import oracle as O
    from paper_2109_04469_gb300 import workloads

    scan = workloads.ensemble_members(members)
    cores = max(1, min(os.cpu_count() or 1, len(scan)))
    pick = [scan[(i * len(scan)) // cores][0] for i in range(cores)]
    done = [0] * cores
    start = threading.Barrier(cores + 1)

    def run(i: int, t_end: list):
        sim = O.OracleSim(dict(pick[i]))  # loaded in this thread, outside the window
        sim.step(1)  # warm-up step
        start.wait()
        while time.perf_counter() < t_end[0]:
            done[i] += sim.count(0) + sim.count(1)
            sim.step(1)

    t_end = [float("inf")]
    threads = [threading.Thread(target=run, args=(i, t_end)) for i in range(cores)]
    for th in threads:
        th.start()
    start.wait()
    t0 = time.perf_counter()
    t_end[0] = t0 + budget_s
    for th in threads:
        th.join()
    wall = time.perf_counter() - t0
    return {"value": sum(done) / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} of the {len(scan)} scan members (every {len(scan) // cores}-th), "
                      f"one per host thread, stepped concurrently for {wall:.1f} s after one "
                      f"warm-up step each; plain C FP64"}


def arm_config(args, cfg: dict, world: int) -> dict:
    """The workload keys of the JSON line, the same for this implementation and the reference
    arm (the oracle): what is simulated, not how."""
    return {"workload": args.workload, "particles_per_species": cfg["init_per_species"],
            "n_cells": cfg["n_cells"], "steps_per_rf": cfg["steps_per_rf"],
            "pressure_pa": cfg["pressure_pa"], "v_rf_amp_v": cfg["v_rf_amp_v"],
            "parallelism": f"replicas x{world}",
            "initial_state": "uniform Maxwellian load (reading C-22), not a converged discharge",
            "l2": "flushed between timed steps: 256 MiB written, then 256 MiB read"}


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
    sample = (f"{args.workload}: {c['init_per_species']} initial superparticles per species "
              f"(the workload's {cfg['init_per_species']} scaled to the time budget)"
              if scale < 1.0 else f"{args.workload}: the full population")
    sample += (f", {args.warmup} warm-up + {args.steps} timed steps, plain C FP64 oracle, "
               f"1 host thread (rank 0 only)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": arm_config(args, cfg, world),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


BYTES_PER_PARTICLE = {  # algorithmic bytes of the particle pass per particle-step
    # FP64: x, vx read and written (32 B) + id read (4 B); a candidate also reads and writes
    # vy, vz (32 B); a removed or born particle moves one 36 B record
    "fp64": (36.0, 32.0, 36.0),
    # FP32 cell + offset: (offset, vx) read and written (16 B) + the cell read and written
    # (4 B) + id read (4 B) = 24 B; candidates r/w vy, vz (16 B); a moved record is 24 B
    "fp32": (24.0, 16.0, 24.0),
}
# the FP32 layout's own bytes: the null-collision countdown shares a u32 with the cell, so the
# cell word is 4 B each way (28 B per particle-step)
FP32_LAYOUT_BYTES = 28.0


def alg_bytes(precision: str, parts: int, dc, per=None) -> float:
    """Algorithmic bytes of the particle passes of a run: `parts` particle-steps, the collision
    candidates and the records moved (removed + born) from the counter deltas dc."""
    p0, cand, rec = BYTES_PER_PARTICLE[precision]
    turnover = int(dc[0] + dc[1] + dc[2] + dc[3] + 2 * dc[8] + dc[5])
    return (p0 if per is None else per) * parts + cand * float(dc[11] + dc[12]) + rec * turnover


class L2Flush:
    """Evict the simulation's data from L2 between timed steps: write one buffer larger than
    L2, then read a second one, so L2 is left holding clean lines of the second buffer and
    the timed step pays neither for hits nor for write-backs of the flush's dirty lines."""

    def __init__(self, torch):
        self.w = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
        self.r = torch.ones(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")

    def __call__(self, k: int):
        self.w.fill_(k)
        self.sink = self.r.sum()


def measure(pcfg: dict, precision: str, args, torch, dist, local_rank: int,
            with_e2e: bool) -> dict:
    """Time args.steps steps of one precision (CUDA events on the library's stream, L2
    flushed between steps, clocks sampled during the timed region)."""
    from paper_2109_04469_gb300 import pic

    cfg = dict(pcfg)
    cfg["precision"] = pic.PIC_FP32 if precision == "fp32" else pic.PIC_FP64
    sim = pic.Simulation(cfg)
    stream = sim.stream
    flush = L2Flush(torch)
    sim.step(args.warmup)
    sim.sync()
    c0 = sim.accum()["counters"].astype(np.int64)
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
    # Every step is enqueued without a host wait, so the host stays ahead of the GPU and no
    # launch latency falls between a step's events: L2 flush, event, the step's two
    # launches, event, copy of the counts after the step (pinned host memory).  Step k
    # processes the counts left by step k - 1.
    counts = torch.zeros((args.steps + 1, 2), dtype=torch.int64, pin_memory=True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        sim.counts_async(counts[0])
        for k in range(args.steps):
            flush(k)  # outside the events
            evs[k][0].record(stream)
            sim.step(1)  # the step's two launches, nothing else between the events
            evs[k][1].record(stream)
            sim.counts_async(counts[k + 1])
    torch.cuda.synchronize()
    step_ms = float(sum(a.elapsed_time(b) for a, b in evs))
    parts = int(counts[:args.steps].sum().item())
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    dc = sim.accum()["counters"].astype(np.int64) - c0  # events of the timed steps
    # per-launch split from a second pass with events around each launch
    ms2 = np.zeros(2)  # particle pass, placement (+ next field solve beside it)
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush(k)
            sim.step_profiled(1, ms2)
    ev0, ev1 = evs[0]
    field_ms = 0.0  # the field solve on its own (it runs beside the placement in a step)
    with torch.cuda.stream(stream):
        for k in range(10):
            ev0.record(stream)
            sim.solve_field()
            ev1.record(stream)
            ev1.synchronize()
            field_ms += ev0.elapsed_time(ev1) / 10
    status = sim.status()
    ab = alg_bytes(precision, parts, dc)
    ab_layout = alg_bytes(precision, parts, dc, FP32_LAYOUT_BYTES) if precision == "fp32" else ab
    per_step = sorted(float(a.elapsed_time(b)) for a, b in evs)
    out = dict(step_ms=step_ms, parts=parts, push_ms=ms2[0] / args.steps,
               place_ms=ms2[1] / args.steps, field_ms=field_ms,
               alg_bytes_per_launch=ab / args.steps,
               layout_bytes_per_launch=ab_layout / args.steps, clocks=clocks, status=status,
               step_ms_quantiles=[per_step[len(per_step) // 10], statistics.median(per_step),
                                  per_step[(9 * len(per_step)) // 10]])
    if with_e2e:
        out["e2e"] = run_e2e(sim, args, torch)
    sim.close()
    return out


def fp64_pipe_roofline(parts_per_launch: float, launch_ms: float, workload: str) -> dict:
    """The FP64 particle pass against the axis that bounds it on GB300: FP64 operations per
    second (DADD + DMUL + 2 DFMA per particle-step, from the committed ncu counters of the
    unchanged kernel) over the pipe rate measured live by pic_fp64_rate (separate multiplies
    and adds, the FP64 path's own mix)."""
    from paper_2109_04469_gb300 import pic

    peak_mix, peak_fma = pic.fp64_rate()
    inst = profiled_value("push_fp64", workload, "fp64_pipe_inst_per_particle_step")
    ops = profiled_value("push_fp64", workload, "fp64_ops_per_particle_step")
    out = {"bound": "fp64", "peak": peak_mix, "peak_fma_flops": peak_fma,
           "unit": "FP64-pipe instructions/s",
           "peak_source": "measured live (pic_fp64_rate: separate multiplies and adds)",
           "inst_per_particle_step": inst, "flops_per_particle_step": ops}
    if inst is not None and ops is not None:
        rate = parts_per_launch / (launch_ms / 1e3)
        out["achieved"] = inst * rate
        out["frac"] = out["achieved"] / peak_mix
        out["flops_frac"] = ops * rate / peak_mix
    else:
        out["achieved"] = out["frac"] = None
        out["note"] = "no ncu count of FP64 instructions for the current kernel sources"
    return out


def measure_ensemble(args, torch, dist, rank: int) -> dict:
    """The batched FP32 scan: args.ensemble_members uneven simulations (workloads.
    ensemble_members) advanced by one graph-replayed launch per step.  Its state is many GB,
    far beyond L2, so steps run back to back; each step is bracketed by CUDA events, with the
    members' counts copied to pinned memory outside the events."""
    from paper_2109_04469_gb300 import pic, workloads

    members = workloads.ensemble_members(args.ensemble_members)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sims = []
        for c, _ in members:
            c = dict(c, precision=pic.PIC_FP32, instance=c["instance"] + 1000 * rank)
            sims.append(pic.Simulation(c))
        ens = pic.Ensemble(sims, [t for _, t in members])
        chosen = ens.autotune(2)
        ens.step(args.ensemble_warmup)
    try:
        ens.sync()
    except pic.PicError:
        pass  # a sticky member status is reported after the timed steps
    c0 = sum(s.accum()["counters"].astype(np.int64) for s in sims)
    n = len(sims)
    steps = args.ensemble_steps
    counts = torch.zeros((steps + 1, n, 2), dtype=torch.int64, pin_memory=True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for i, sim in enumerate(sims):
            sim.counts_async(counts[0, i])
        for k in range(steps):
            evs[k][0].record(stream)
            ens.step(1)
            evs[k][1].record(stream)
            for i, sim in enumerate(sims):
                sim.counts_async(counts[k + 1, i])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    try:
        status = ens.sync()
    except pic.PicError as e:  # reported in the line (e.g. births dropped at capacity)
        status = e.code
    step_ms = float(sum(a.elapsed_time(b) for a, b in evs))
    parts = int(counts[:steps].sum().item())
    dc = sum(s.accum()["counters"].astype(np.int64) for s in sims) - c0
    info = ens.info()
    grow = counts[steps].double() / counts[0].double().clamp(min=1)
    out = dict(step_ms=step_ms, parts=parts, alg_bytes=alg_bytes("fp32", parts, dc),
               layout_bytes=alg_bytes("fp32", parts, dc, FP32_LAYOUT_BYTES), status=status,
               steps=steps, max_growth=float(grow.max().item()),
               members=n, particles=int(counts[0].sum().item()),
               schedule={"unit": chosen[0], "blocks_per_sm": chosen[1], "grid": info["grid"],
                         "graph": bool(info["graph"])})
    ens.close()
    del sims
    return out


def measure_stress(args, torch, dist, local_rank: int, rank: int, peak: float,
                   world: int = 1) -> dict:
    """The stress workload (5e7 + 5e7 superparticles, 1025 nodes): both precisions, the split
    of a step between the particle launch, the placement launch and the field solve, and the
    field solve's share of the step."""
    import types

    from paper_2109_04469_gb300 import workloads

    name = "ccp_20pa_500v_1024c"
    scfg = workloads.params(name)
    scfg["instance"] = rank
    sargs = types.SimpleNamespace(**vars(args))
    sargs.steps, sargs.warmup = args.stress_steps, 3
    out = {"workload": name + ": 3 cm, 1024 cells, 20 Pa, 500 V, N_t 4000, 5e7 + 5e7 "
                              "superparticles, R 0.2, gamma 0.2",
           "l2": "state of several GB, larger than L2 (the flush between steps is kept)"}
    for prec in ("fp32", "fp64"):
        r = measure(scfg, prec, sargs, torch, dist, local_rank, with_e2e=False)
        t, p = reduce_ranks(torch, dist, r["step_ms"], r["parts"])
        ms = t / sargs.steps
        out[prec] = {"value": p / (t / 1e3), "unit": UNIT, "ms_per_step": ms,
                     "particles_ms": r["push_ms"], "placement_and_next_field_ms": r["place_ms"],
                     "field_alone_ms": r["field_ms"], "poisson_share": r["field_ms"] / ms,
                     "roofline_frac_hbm": r["alg_bytes_per_launch"] / (r["push_ms"] / 1e3)
                     / 1e9 / peak,
                     "bytes_per_particle_step": BYTES_PER_PARTICLE[prec][0],
                     "status": r["status"], "clocks": r["clocks"]}
        if prec == "fp32":
            out[prec]["roofline_frac_hbm_layout_28b"] = (
                r["layout_bytes_per_launch"] / (r["push_ms"] / 1e3) / 1e9 / peak)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(dict(scfg, name=name), 2, warmup=1)
    return out


def measure_surrogate(torch) -> dict:
    """The surrogate network of the parameter scans: a 2000-setting scan run by the FP32
    ensemble (2 RF periods from the load, then averages over 2 more), the network trained on
    1800 settings by the tensor-core kernels, judged on the 200 held-out settings by the plain
    method's profiles; plus the tensor-core rate of its forward pass at batch 1024."""
    from paper_2109_04469_gb300 import pic, surrogate as S

    settings = S.sample_settings(2000, seed=11)
    X, Y, D, pic_s = S.run_scan(settings, warm_cycles=2.0, avg_cycles=2.0)
    tr, te = np.arange(1800), np.arange(1800, 2000)
    sur = S.Surrogate(batch_max=512, seed=4)
    t = time.perf_counter()
    losses = sur.fit(X[tr], Y[tr], epochs=300)
    torch.cuda.synchronize()
    fit_s = time.perf_counter() - t
    t = time.perf_counter()
    P = sur.predict(X[te])
    net_s = time.perf_counter() - t
    err = S.profile_error(P, Y[te])
    base = S.profile_error(np.repeat(Y[tr].mean(axis=0, keepdims=True), len(te), 0), Y[te])
    agree = (S.accuracy_flags([settings[i] for i in te], P) ==
             S.pic_flags([D[i] for i in te])).mean(axis=0)
    # tensor-core rate of the network's forward pass at batch 1024 (three GEMMs and their
    # epilogues, enqueued back to back; events around 50 passes)
    net = pic.Mlp(1024, seed=1)
    xb = torch.randn(1024, 7, device="cuda")
    net.forward(xb)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(50):
        net.forward(xb)
    e1.record()
    e1.synchronize()
    fwd_ms = e0.elapsed_time(e1) / 50
    fwd_flop = 2.0 * 1024 * (16 * 256 + 256 * 256 + 256 * 192)
    return {"settings": len(settings), "held_out": len(te),
            "held_out_profile_error_mean": float(err.mean()),
            "held_out_profile_error_median": float(np.median(err)),
            "training_mean_error": float(base.mean()),
            "flag_agreement": [float(v) for v in agree],
            "scan_gpu_s_per_setting": pic_s / len(settings),
            "network_s_per_setting": net_s / len(te), "fit_s": fit_s,
            "final_loss": float(losses[-1]),
            "forward_1024_us": fwd_ms * 1e3,
            "forward_tflops": fwd_flop / (fwd_ms * 1e-3) / 1e12,
            "held_out_dx_flag_positives": int(S.pic_flags([D[i] for i in te])[:, 1].sum()),
            "note": "scan runs are 4 RF periods from a uniform load (not converged "
                    "discharges); the network is tiny, so its kernels are launch and latency "
                    "bound, far from the tensor-core peak"}


def reduce_ranks(torch, dist, step_ms: float, parts: int, device: str = "cuda"):
    """Whole-job figures of the replicas: the slowest rank's time, every rank's particles."""
    if not dist:
        return step_ms, parts
    t = torch.tensor([step_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    p = torch.tensor([int(parts)], dtype=torch.int64, device=device)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t.item()), int(p.item())


def profile_case(mode: str) -> None:
    """Small, self-contained launches of one kernel family for ncu: the FP32 or FP64 particle
    pass on the production workload (5 steps), a 16-member ensemble (5 steps) and the
    surrogate network's training GEMMs (3 Adam steps at batch 1024)."""
    import torch

    from paper_2109_04469_gb300 import pic, workloads

    if mode in ("fp32", "fp64"):
        prec = pic.PIC_FP32 if mode == "fp32" else pic.PIC_FP64
        sim = pic.Simulation(workloads.params("ccp_1pa_300v_400c", precision=prec))
        for k in range(5):  # particles each step's pass starts from (for per-particle counts)
            print("step", k, "particles", sum(sim.counts()))
            sim.step(1)
        print("status", sim.sync())
    elif mode == "ens":  # 16 scan members (2.5e5-1e6 superparticles each)
        members = workloads.ensemble_members(16, per_run=(2.5e5, 1.0e6))
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            sims = [pic.Simulation(dict(c, precision=pic.PIC_FP32)) for c, _ in members]
            ens = pic.Ensemble(sims, [10**9] * len(sims))
            ens.configure(2048, 2, True)
            ens.step(5)
        print("status", ens.sync())
    else:  # mlp
        net = pic.Mlp(1024, seed=1)
        x = torch.randn(1024, 7, device="cuda")
        t = torch.randn(1024, 192, device="cuda")
        for _ in range(3):
            net.train_step(x, t, 1e-3, want_loss=False)
        torch.cuda.synchronize()
        print("ok")


def main():
    args = parse()
    if args.profile_case:
        profile_case(args.profile_case)
        return
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
    cfg["instance"] = rank  # independent replica per rank
    pcfg = {k: v for k, v in cfg.items() if k != "name"}
    runs = {}
    for prec in args.precisions.split(","):
        e2e = prec == args.precisions.split(",")[0] and not args.no_e2e
        r = measure(pcfg, prec, args, torch, dist, local_rank, with_e2e=e2e)
        bad = clocks_rejected(r["clocks"])
        if dist:  # every rank measures again if any rank's clocks were off
            flag = torch.tensor([int(bad)], device="cuda")
            dist.all_reduce(flag, op=dist.ReduceOp.MAX)
            bad = bool(flag.item())
        if bad:  # measured again once; the line says so
            r = measure(pcfg, prec, args, torch, dist, local_rank, with_e2e=e2e)
            r["clocks"]["remeasured"] = True
        r["clocks"]["rejected"] = clocks_rejected(r["clocks"])
        runs[prec] = r
    head_prec = args.precisions.split(",")[0]
    head = runs[head_prec]
    total_ms, total_parts = reduce_ranks(torch, dist, head["step_ms"], head["parts"])
    value = total_parts / (total_ms / 1e3)
    peak, peak_src = measured_peak()
    achieved = head["alg_bytes_per_launch"] / (head["push_ms"] / 1e3) / 1e9
    achieved_layout = head["layout_bytes_per_launch"] / (head["push_ms"] / 1e3) / 1e9
    kname = "k_push_fp32" if head_prec == "fp32" else "k_push_fp64"
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": peak_src,
            "traffic": profiled_traffic(f"push_{head_prec}", args.workload),
            "kernel": kname, "alg_bytes_per_launch": head["alg_bytes_per_launch"],
            "bytes_per_particle_step": BYTES_PER_PARTICLE[head_prec][0],
            "launch_ms": head["push_ms"]}
    if head_prec == "fp32":
        roof["frac_layout_28b"] = achieved_layout / peak
    ms_step = total_ms / args.steps
    q = head["step_ms_quantiles"]
    parts_per_step = total_parts / args.steps
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if head_prec == "fp32" else "f64", "data": "synthetic",
            "config": arm_config(args, cfg, world),
            "per_step_spread": {"value_p10": parts_per_step / world / (q[2] / 1e3),
                                "value_median": parts_per_step / world / (q[1] / 1e3),
                                "value_p90": parts_per_step / world / (q[0] / 1e3),
                                "note": "rank-0 per-step event times (10 %, 50 %, 90 % "
                                        "quantiles of the rate)"},
            "roofline": roof,
            "kernel_ms_per_step": {"particles": head["push_ms"],
                                   "placement_and_next_field": head["place_ms"],
                                   "field_alone": head["field_ms"]},
            "poisson_share": head["field_ms"] / ms_step,
            "compaction_share": max(0.0, head["place_ms"] - head["field_ms"]) / ms_step,
            "gpu_launches": 2 * args.steps,
            "precision": head_prec + (" particles, fp64 field" if head_prec == "fp32" else ""),
            "clocks": head["clocks"], "status": head["status"]}
    for prec, r in runs.items():
        if prec == head_prec:
            continue
        t, p = reduce_ranks(torch, dist, r["step_ms"], r["parts"])
        line[f"{prec}_plain"] = {
            "value": p / (t / 1e3), "ms_per_step": t / args.steps, "particles_ms": r["push_ms"],
            "roofline_frac_hbm": r["alg_bytes_per_launch"] / (r["push_ms"] / 1e3) / 1e9 / peak,
            "clocks": r["clocks"]}
        if prec == "fp64":
            line["fp64_plain"]["roofline_fp64_pipe"] = fp64_pipe_roofline(
                r["parts"] / args.steps, r["push_ms"], args.workload)
        line[f"speedup_vs_{prec}"] = value / (p / (t / 1e3))
    if not args.no_ensemble:
        er = measure_ensemble(args, torch, dist, rank)
        et, ep = reduce_ranks(torch, dist, er["step_ms"], er["parts"])
        ev = ep / (et / 1e3)
        eb = er["alg_bytes"] / (er["step_ms"] / 1e3) / 1e9  # the launch is the whole step
        ebl = er["layout_bytes"] / (er["step_ms"] / 1e3) / 1e9
        ok = er["status"] == 0
        line["ensemble"] = {
            # a run that dropped births no longer follows §2 step 6: no value is reported
            "value": ev if ok else None, "unit": UNIT,
            "ms_per_step": et / er["steps"], "steps": er["steps"],
            "warmup": args.ensemble_warmup,
            "members": er["members"], "particles_per_step": er["particles"],
            "max_population_growth": er["max_growth"],
            "workload": "64 uneven ccp scans (workloads.ensemble_members): p 1-20 Pa, "
                        "V 100-500 V, N_t 500-4000, 100-800 cells, 2.5e5-4e6 superparticles per "
                        "run, R 0-0.7, gamma 0-0.4; uniform Maxwellian loads",
            "l2": "state of many GB, larger than L2: steps back to back",
            "schedule": er["schedule"],
            "roofline": {"bound": "hbm", "achieved": eb, "peak": peak, "unit": "GB/s",
                         "frac": eb / peak, "frac_layout_28b": ebl / peak,
                         "kernel": "k_ensemble_step"},
            "status": er["status"]}
        if not ok:
            line["ensemble"]["refused"] = ("non-zero status: a member dropped births or a wait "
                                          "timed out, so the run is not the method's")
        if ok and "fp64" in runs and "fp64" != head_prec:
            line["ensemble"]["speedup_vs_fp64_plain"] = ev / line["fp64_plain"]["value"]
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            line["ensemble"]["cpu_baseline"] = ensemble_cpu_baseline(args.ensemble_members)
    if not args.no_stress:
        line["stress"] = measure_stress(args, torch, dist, local_rank, rank, peak, world)
    if not args.no_surrogate and rank == 0:
        line["surrogate"] = measure_surrogate(torch)
    if "e2e" in head:
        line["e2e"] = head["e2e"]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(pcfg | {"name": args.workload}, args.cpu_steps)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


E2E_WARMUP = 3  # untimed end-to-end iterations before the timed ones


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
    def e2e_step():
        for s in (0, 1):
            a = host[s]
            n = len(a["x"][1])
            sim.set_particles(s, a["x"][1], a["vx"][1], a["vy"][1], a["vz"][1], a["id"][1], n)
        sim.step(1)
        sim.diag()

    for _ in range(E2E_WARMUP):  # untimed, like every other measurement's warm-up
        e2e_step()
    parts = 0
    times = []
    for _ in range(args.e2e_steps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        e2e_step()
        times.append(time.perf_counter() - t)
        parts += len(host[0]["x"][1]) + len(host[1]["x"][1])
    total = sum(times)
    return {"value": parts / total, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "steps": args.e2e_steps, "warmup": E2E_WARMUP,
            "note": "wall clock per step: H2D of the full particle state from pinned memory, "
                    "one step, pic_diag read-back"}


if __name__ == "__main__":
    main()
