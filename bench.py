#!/usr/bin/env python
"""Reweighted events/s for g g -> t t~ g on B300: 2^20 events x 16 parameter points per GPU.

One step = one pass of the whole hot path (momenta -> wavefunctions -> currents ->
jamps -> colour sum -> helicity sum -> w*|M'|^2/|M|^2) over one batch: a single
rex_reweight call on 2^20 seeded RAMBO events (sqrt(s_hat) log-uniform in
[400, 4000] GeV, mt = 173) to 16 points (mt in linspace(171, 175, 4) x alphas in
linspace(0.112, 0.124, 4)), original point (mt = 173, alphas = 0.118).

  python bench.py [--gpus N --steps K --warmup W] [--mode fp64|mixed] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): every rank reweights its own 2^20 events
(seed 3 + rank); no data-path collective, weak scaling.  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
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

from paper_2510_05100_b300 import dist as rdist  # noqa: E402
from paper_2510_05100_b300 import phase_space as ps  # noqa: E402

METRIC = "reweighted events/sec (events x param points), gg->tt~g, 1 B300, at stated rel. error"
UNIT = "events*points/s"
PROC = "gg_ttxg"
NEV = 1 << 20
ORIGINAL = dict(mt=173.0, wt=0.0, alphas=0.118)
SEED = 3
# relative error of a new weight vs the FP64 oracle, per mode (tests/test_gpu_parity.py)
STATED_ERROR = {"fp64": 1e-12, "mixed": 1e-3, "df64": 1e-12}

# Peaks for an ALU-bound kernel, derived from unit counts and the maximum SM clock
# (148 SMs, 2032 MHz): FP32 = 148 x 128 lanes x 2 flop x 2.032 GHz.  The FP64 figure
# uses the FP64 FMA issue rate per SM measured by rex_probe_fma (2 DFMA per clock per SM).
SM_COUNT = 148
SM_MAX_MHZ = 2032.0
FP32_PEAK = SM_COUNT * 128 * 2 * SM_MAX_MHZ * 1e6
FP64_FMA_PER_SM_CLK = 2         # rex_probe_fma: 1.18 TFLOP/s at 2032 MHz on 148 SMs -> 1.96

def _measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


PEAKS = _measured_peaks()

# DRAM traffic per launch from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum) of the dominant kernel, scaled to the full launch;
# only reported while the kernel sources still hash to the captured version.
TRAFFIC = {
    # ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum of profile_case at 2^19
    # events (FP64, scaled x2 by events) and 2^20 events (mixed); summaries of the
    # captures are under profiles/
    ("gg_ttxg", "fp64"): {"bytes_per_launch": 2 * (91.167232e6 + 34.621440e6), "source_hash": "fb0176ae6762d5e1"},
    ("gg_ttxg", "mixed"): {"bytes_per_launch": 176.708608e6 + 104.756992e6, "source_hash": "fb0176ae6762d5e1"},
}


def kernel_source_hash() -> str:
    """Hash of what the g g -> t t~ g kernel is compiled from: its own sources and, from the
    shared launch header, the launch-table struct and its size constants (declarations of
    other processes there do not change this kernel)."""
    import re
    h = hashlib.sha256()
    for rel in ("paper_2510_05100_b300/csrc/qcd_kernel.cuh", "paper_2510_05100_b300/csrc/kernels_gg_ttxg.cu",
                "paper_2510_05100_b300/csrc/helas.cuh", "paper_2510_05100_b300/csrc/colour_tc.cuh",
                "paper_2510_05100_b300/csrc/fpconv.cuh", "paper_2510_05100_b300/csrc/df64.cuh",
                "paper_2510_05100_b300/csrc/gg_ttxg_df64.cuh",
                "paper_2510_05100_b300/csrc/generated/qcd_amplitudes.cuh"):
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    with open(os.path.join(ROOT, "paper_2510_05100_b300/csrc/rex_internal.cuh")) as f:
        text = f.read()
    for pat in (r"constexpr int MAX_MASS = \d+;", r"constexpr int MAX_POINTS = \d+;", r"struct QcdLaunch \{.*?\n\};"):
        h.update(re.search(pat, text, re.S).group(0).encode())
    return h.hexdigest()[:16]


# ----------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, on the host cores, on a bounded sample
# ----------------------------------------------------------------------------
def _oracle_chunk(args):
    mom, pts = args
    from oracle import reweight as orw
    orw.reweight(PROC, mom, np.ones(mom.shape[0]), ORIGINAL, pts)
    return mom.shape[0]


def oracle_throughput(mom_all: np.ndarray, pts, ntasks: int, chunk: int, cores: int, pool=None):
    """Events*points/s of the oracle over ntasks chunks of ``chunk`` events."""
    import multiprocessing as mp
    tasks = [(mom_all[(i * chunk) % (mom_all.shape[0] - chunk):][:chunk].copy(), pts) for i in range(ntasks)]
    own = pool is None
    if own:
        pool = mp.get_context("spawn").Pool(cores)
    t0 = time.perf_counter()
    done = sum(pool.map(_oracle_chunk, tasks, chunksize=1))
    dt = time.perf_counter() - t0
    if own:
        pool.close()
        pool.join()
    return done * len(pts) / dt, done, dt


def _cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _start_pool(cores):
    import multiprocessing as mp
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    os.environ.setdefault("MKL_NUM_THREADS", "1")
    return mp.get_context("spawn").Pool(cores)


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = bus_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.bus_id:
            cmd += ["-i", self.bus_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_median": statistics.median(power) if power else None}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--nev", type=int, default=NEV)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra-modes", action="store_true")
    ap.add_argument("--no-multi", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-xsec", action="store_true")
    ap.add_argument("--no-lhe", action="store_true")
    ap.add_argument("--no-qq", action="store_true", help="skip the q q~ -> t t~ (g) and p p -> t t~ legs")
    ap.add_argument("--no-helicity", action="store_true", help="skip the helicity-exclusive leg")
    args = ap.parse_args()
    world, rank, local = rdist.env()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_ours(args, world, rank, local)


def grid():
    return ps.grid_gg_ttxg()


def config_block(args, world):
    return {"workload": f"{PROC}: g g -> t t~ g, {args.nev} events/GPU x 16 param points",
            "process": PROC, "events_per_gpu": args.nev, "param_points": 16,
            "grid": "mt in linspace(171,175,4) x alphas in linspace(0.112,0.124,4), mt-major",
            "original": ORIGINAL, "events": "seeded massive RAMBO, sqrt(s_hat) log-uniform [400, 4000] GeV",
            "seed": f"{SEED} + rank", "mode": args.mode,
            "l2": "inputs larger than L2 (momenta 160 MiB + w_out 128 MiB per GPU > 126 MB)",
            "parallelism": f"replicas x{world} (events sharded per GPU, no collective)"}


def run_reference(args, world, rank):
    """The oracle (FP64, numpy, CPU) timed on the host cores: --impl reference."""
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    pool = _start_pool(cores)
    mom = ps.make_events(PROC, 1 << 14, SEED)
    pts = grid()
    chunk = 256
    for _ in range(args.warmup):
        oracle_throughput(mom, pts, cores, chunk, cores, pool)
    t_total = 0.0
    n_total = 0
    for _ in range(args.steps):
        _, n, dt = oracle_throughput(mom, pts, cores, chunk, cores, pool)
        t_total += dt
        n_total += n
    pool.close()
    pool.join()
    value = n_total * len(pts) / t_total
    sample = f"{args.steps} steps x {cores} chunks x {chunk} events of the {PROC} workload, 16 points each"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_block(args, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


MULTI_BATCHES = (("ee_mumu", 10_000, 41), ("gg_ttx", 1_000_000, 42), ("gg_ttxg", 500_000, 43),
                 ("gg_ttxgg", 100_000, 44))


def multi_amp_flops(spec, pts):
    """Counted FP32 amplitude flops of one mixed multi-process step (for the time-weighted
    fraction of a batch: all its processes' flops over one time and the FP32 peak).
    spec: (process, events); crossed q q~ -> t t~ g channels count as q q~ -> t t~ g; the
    e+e- batch runs in FP64 and is left out."""
    from paper_2510_05100_b300 import flops as flopmod
    nmass = 1 + len({p["mt"] for p in pts} - {ORIGINAL["mt"]})
    total = 0
    for proc, n in spec:
        kind = "qq_ttxg" if proc in ("qxq_ttxg", "qg_ttxq", "gq_ttxq", "qxg_ttxqx", "gqx_ttxqx") else proc
        if kind == "ee_mumu":
            continue
        total += n * flopmod.per_event(kind, 1 if kind == "qq_ttx" else nmass)["amp"]
    return total


def time_weighted(fl, ms):
    return {"bound": "alu", "pipe": "FP32 FMA (counted amplitude flops of every batch over the step)",
            "achieved": fl / (ms * 1e-3) / 1e12, "peak": FP32_PEAK / 1e12, "unit": "TFLOP/s",
            "frac": fl / (ms * 1e-3) / FP32_PEAK}


def run_multi_leg(dev, stream, steps, world, barrier, max_over_ranks):
    """Mixed batch of four subprocesses x 64 points in one persistent, graph-captured launch
    (mixed precision), against the same work as four sequential single-process launches."""
    import torch
    from paper_2510_05100_b300 import rex

    pts = [dict(p, **ps.EE_NEW) for p in ps.grid_64()]
    batches = []
    for proc, n, seed in MULTI_BATCHES:
        prec = rex.FP64 if proc == "ee_mumu" else rex.MIXED
        h = rex.Process(proc, prec)
        h.set_params(ps.EE_ORIGINAL if proc == "ee_mumu" else ORIGINAL)
        mom = torch.from_numpy(ps.make_events(proc, n, seed)).to(dev)
        batches.append((h, mom, torch.ones(n, dtype=torch.float64, device=dev),
                        torch.empty((n, len(pts)), dtype=torch.float64, device=dev)))
    m = rex.Multi(rex.MIXED)          # ee_mumu (FP64 only) joins the mixed launch
    tune = m.autotune(batches, pts, stream=stream)   # slot groups by measurement
    m.capture(batches, pts)
    ms_streams = rex.Multi(rex.MIXED, rex.MULTI_STREAMS)   # one launch per batch, forked streams
    ms_streams.capture(batches, pts)
    units = sum(b[1].shape[0] for b in batches) * len(pts)

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize(dev)
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(steps):
            fn()
        t1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        return max_over_ranks(t0.elapsed_time(t1)) / steps

    def graph_step():
        m.replay(stream)

    def sequential_step():
        for h, mom, w, wo in batches:
            h.reweight(mom, w, pts, w_out=wo, stream=stream)

    ms_graph = timed(graph_step)
    ms_seq = timed(sequential_step)
    ms_str = timed(lambda: ms_streams.replay(stream))
    m_groups = m.slot_groups
    tile_us = {proc: m.tile_cost(b[0]) for (proc, _, _), b in zip(MULTI_BATCHES, batches)}
    m.close()
    fl = multi_amp_flops([(proc, n) for proc, n, _ in MULTI_BATCHES], pts)
    ms_streams.close()
    return {"workload": "10k ee_mumu (FP64) + 1M gg_ttx + 500k gg_ttxg + 100k gg_ttxgg (mixed) x 64 points",
            "value": rdist.job_throughput(units, world, ms_graph * 1e-3), "unit": UNIT,
            "ms_per_step": ms_graph, "graph_launches_per_step": 1, "slot_groups": m_groups,
            "autotune_ms_per_launch": dict(zip((1, 2, 3, 4, 6, 8), tune)),
            "measured_tile_us": tile_us,   # one block's time per tile: the order of the work items
            "kernel_launches_per_step": 3,   # one persistent kernel per register class present
            "sequential_value": rdist.job_throughput(units, world, ms_seq * 1e-3),
            "sequential_ms_per_step": ms_seq,
            "streams_graph_value": rdist.job_throughput(units, world, ms_str * 1e-3),
            "streams_graph_ms_per_step": ms_str,
            "roofline": time_weighted(fl, ms_graph),
            "sequential_roofline_frac": time_weighted(fl, ms_seq)["frac"],
            "streams_graph_roofline_frac": time_weighted(fl, ms_str)["frac"],
            "note": "value: one captured graph of persistent kernels, one per register class present; "
                    "sequential: one single-process launch per batch; streams_graph: one graph of "
                    "per-process launches on forked streams",
            "steps": steps}


# many channels of small event counts: the regime where one launch per subprocess leaves
# the GPU latency bound (paper Sec. 4.2); crossed channels use the q q~ -> t t~ g events
SMALL_MULTI_BATCHES = (("gg_ttx", 8000, 71, "gg_ttx"), ("gg_ttxg", 4000, 72, "gg_ttxg"),
                       ("gg_ttxgg", 1000, 73, "gg_ttxgg"), ("qq_ttx", 8000, 74, "qq_ttx"),
                       ("qq_ttxg", 3000, 75, "qq_ttxg"), ("qg_ttxq", 2000, 76, "qq_ttxg"),
                       ("gq_ttxq", 2000, 77, "qq_ttxg"), ("qxg_ttxqx", 1000, 78, "qq_ttxg"))


def run_small_multi_leg(dev, stream, steps, world, barrier, max_over_ranks):
    """Eight subprocess batches of 10^3 - 10^4 events x 64 points (mixed precision): one
    graph of persistent kernels (one per register class present) against a graph of one
    single-process launch per batch (captured with the same stream), the streams mode's
    graph of per-process launches on forked streams, and plain sequential launches."""
    import torch
    from paper_2510_05100_b300 import rex

    pts = ps.grid_64()
    batches = []
    for proc, n, seed, gen in SMALL_MULTI_BATCHES:
        h = rex.Process(proc, rex.MIXED)
        h.set_params(ORIGINAL)
        mom = torch.from_numpy(ps.make_events(gen, n, seed)).to(dev)
        batches.append((h, mom, torch.ones(n, dtype=torch.float64, device=dev),
                        torch.empty((n, len(pts)), dtype=torch.float64, device=dev)))
    units = sum(b[1].shape[0] for b in batches) * len(pts)
    m = rex.Multi(rex.MIXED)
    tune = m.autotune(batches, pts, stream=stream)   # slot groups by measurement
    m.capture(batches, pts)
    ms_streams = rex.Multi(rex.MIXED, rex.MULTI_STREAMS)
    ms_streams.capture(batches, pts)

    def sequential_step(st=stream):
        for h, mom, w, wo in batches:
            h.reweight(mom, w, pts, w_out=wo, stream=st)

    # the same per-batch launches captured into one CUDA graph
    cap = torch.cuda.Stream(dev)
    cap.wait_stream(torch.cuda.current_stream(dev))
    sequential_step(cap)
    torch.cuda.synchronize(dev)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=cap):
        sequential_step(cap)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(steps):
            fn()
        t1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        return max_over_ranks(t0.elapsed_time(t1)) / steps

    ms_persistent = timed(lambda: m.replay(stream))
    groups = m.slot_groups
    m.slot_groups = 1
    m.capture(batches, pts)
    ms_persistent1 = timed(lambda: m.replay(stream))
    ms_seq_graph = timed(lambda: g.replay())
    ms_streams_graph = timed(lambda: ms_streams.replay(stream))
    ms_seq = timed(sequential_step)
    tile_us = {proc: m.tile_cost(b[0]) for (proc, _, _, _), b in zip(SMALL_MULTI_BATCHES, batches)}
    m.close()
    ms_streams.close()
    for b in batches:
        b[0].close()
    desc = " + ".join(f"{n} {proc}" for proc, n, _, _ in SMALL_MULTI_BATCHES)
    val = lambda ms: rdist.job_throughput(units, world, ms * 1e-3)   # noqa: E731
    fl = multi_amp_flops([(proc, n) for proc, n, _, _ in SMALL_MULTI_BATCHES], pts)
    frac = lambda ms: time_weighted(fl, ms)["frac"]   # noqa: E731
    return {"workload": f"{desc}, 64 points each, mixed precision", "unit": UNIT, "steps": steps,
            "roofline": time_weighted(fl, ms_persistent),
            "fracs": {"persistent_graph": frac(ms_persistent), "per_process_graph": frac(ms_seq_graph),
                      "streams_graph": frac(ms_streams_graph), "sequential_launches": frac(ms_seq)},
            "persistent_graph": {"value": val(ms_persistent), "ms_per_step": ms_persistent,
                                 "slot_groups": groups, "autotune_ms_per_launch": dict(zip((1, 2, 3, 4, 6, 8), tune)),
                                 "without_slot_groups_ms_per_step": ms_persistent1, "measured_tile_us": tile_us},
            "per_process_graph": {"value": val(ms_seq_graph), "ms_per_step": ms_seq_graph},
            "streams_graph": {"value": val(ms_streams_graph), "ms_per_step": ms_streams_graph},
            "sequential_launches": {"value": val(ms_seq), "ms_per_step": ms_seq},
            "note": "persistent_graph: one graph of persistent kernels, one per register class present; "
                    "per_process_graph: one single-process launch per batch, captured; streams_graph: "
                    "per-process launches on forked streams, captured; sequential_launches: per-process "
                    "launches from the host"}


def run_qqg_leg(dev, stream, pts, steps, nev=NEV):
    """q q~ -> t t~ g (the quark-initiated p p -> t t~ + jet channel) on the headline's
    points: nev events per launch in FP64, mixed precision and double-float, CUDA-event
    timed, with the roofline of each kernel against its arithmetic pipe (counted flops)."""
    import torch
    from paper_2510_05100_b300 import flops as flopmod
    from paper_2510_05100_b300 import rex
    k = len(pts)
    mom = torch.from_numpy(ps.make_events("qq_ttxg", nev, SEED + 200)).to(dev)
    w_in = torch.ones(nev, dtype=torch.float64, device=dev)
    w_out = torch.empty((nev, k), dtype=torch.float64, device=dev)
    nmass = 1 + len({p["mt"] for p in pts} - {ORIGINAL["mt"]})
    fl = flopmod.per_event("qq_ttxg", nmass)["amp"] * nev
    p64 = SM_COUNT * FP64_FMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6
    out = {"workload": f"q q~ -> t t~ g, {nev} events x {k} points ({nmass} mass slots), the headline's grid",
           "flops_per_launch": fl}
    fl_df = flopmod.per_event("qq_ttxg_df64", nmass)["amp"] * nev   # FP32 flops of the double-float code
    for name, prec, peak, pipe in (("fp64", rex.FP64, p64, "FP64 FMA"), ("mixed", rex.MIXED, FP32_PEAK, "FP32 FMA"),
                                   ("double_float", rex.DF64, FP32_PEAK, "FP32 FMA (double-float operations)")):
        proc = rex.Process("qq_ttxg", prec)
        proc.set_params(ORIGINAL)
        for _ in range(3):
            proc.reweight(mom, w_in, pts, w_out=w_out, stream=stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize(dev)
        for a, b in ev:
            a.record(stream)
            proc.reweight(mom, w_in, pts, w_out=w_out, stream=stream)
            b.record(stream)
        torch.cuda.synchronize(dev)
        proc.close()
        t = statistics.mean(a.elapsed_time(b) for a, b in ev) * 1e-3
        f = fl_df if prec == rex.DF64 else fl
        out[name] = {"value": nev * k / t, "unit": UNIT, "ms_per_launch": t * 1e3,
                     "roofline": {"bound": "alu", "pipe": pipe, "achieved": f / t / 1e12, "peak": peak / 1e12,
                                  "unit": "TFLOP/s", "frac": f / t / peak}}
    return out


# multi-channel p p -> t t~ (+ jet) samples of 2^20 events: g g and q q~ initial states
# 7 : 1 for t t~; g g, q g, q~ g and q q~ 12 : 2 : 1 : 1 for t t~ + jet
PP_TTX_BATCHES = (("gg_ttx", 917504, 11), ("qq_ttx", 131072, 12))
PP_TTXJ_BATCHES = (("gg_ttxg", 786432, 13), ("qg_ttxq", 131072, 15), ("qxg_ttxqx", 65536, 16),
                   ("qq_ttxg", 65536, 14))


def run_pp_ttx_leg(dev, stream, pts, steps, world, barrier, max_over_ranks, spec=PP_TTX_BATCHES):
    """The p p -> t t~ (+ jet) channels (one batch per initial state of one sample)
    reweighted to the headline's points: one graph-captured persistent multi-process launch against one
    launch per channel, in FP64 and in mixed precision."""
    import torch
    from paper_2510_05100_b300 import rex

    units = sum(n for _, n, _ in spec) * len(pts)

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize(dev)
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(steps):
            fn()
        t1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        return max_over_ranks(t0.elapsed_time(t1)) / steps

    desc = " + ".join(f"{n} {proc}" for proc, n, _ in spec)
    out = {"workload": f"{len(spec)}-channel sample of 2^20 events: {desc}, {len(pts)} points", "unit": UNIT,
           "steps": steps}
    results = {}
    for name, prec in (("fp64", rex.FP64), ("mixed", rex.MIXED)):
        batches = []
        for proc, n, seed in spec:
            h = rex.Process(proc, prec)
            h.set_params(ORIGINAL)
            mom = torch.from_numpy(ps.make_events(proc, n, seed)).to(dev)
            batches.append((h, mom, torch.ones(n, dtype=torch.float64, device=dev),
                            torch.empty((n, len(pts)), dtype=torch.float64, device=dev)))
        m = rex.Multi(prec)
        m.capture(batches, pts)

        def sequential():
            for h, mom, w, wo in batches:
                h.reweight(mom, w, pts, w_out=wo, stream=stream)

        ms_multi = timed(lambda: m.replay(stream))
        ms_seq = timed(sequential)
        m.replay(stream)
        torch.cuda.synchronize(dev)
        results[name] = [b[3].clone() for b in batches]
        m.close()
        for b in batches:
            b[0].close()
        out[name] = {"value": rdist.job_throughput(units, world, ms_multi * 1e-3), "ms_per_step": ms_multi,
                     "kernel_launches_per_step": 1,
                     "sequential_value": rdist.job_throughput(units, world, ms_seq * 1e-3),
                     "sequential_ms_per_step": ms_seq}
    # accuracy of the mixed mode on this sample: per channel, against the FP64 weights
    acc = {}
    for (proc, _, _), wm, wd in zip(spec, results["mixed"], results["fp64"]):
        # relative error where the FP64 weight is non-zero; a weight that is zero in one
        # mode and not in the other (or NaN) is counted apart instead of turning the max NaN
        nz = wd != 0
        err = torch.where(nz, (wm / torch.where(nz, wd, torch.ones_like(wd)) - 1.0).abs(), torch.zeros_like(wd))
        bad = ((wd == 0) != (wm == 0)) | torch.isnan(wm) | torch.isnan(wd)
        err = torch.where(bad, torch.zeros_like(err), err).amax(dim=1)
        acc[proc] = {"max_rel_err": float(err.max()), "frac_events_above_1e-4": float((err > 1e-4).double().mean()),
                     "weights_zero_or_nan_in_one_mode_only": int(bad.sum())}
    out["mixed"]["vs_fp64"] = acc
    return out


def _soft_collinear_y(mom):
    """min over i in {1, 2, t, t~} of 2 k.p_i / s_hat for the final gluon k (torch, [n, 5, 4]),
    the variable of the surrogate's fallback guard."""
    import torch

    def dot(a, b):
        return a[:, 0] * b[:, 0] - (a[:, 1:] * b[:, 1:]).sum(1)
    shat = dot(mom[:, 0] + mom[:, 1], mom[:, 0] + mom[:, 1])
    return 2.0 * torch.stack([dot(mom[:, 4], mom[:, i]) for i in range(4)]).min(dim=0).values / shat


def run_surrogate_leg(dev, stream, world, max_over_ranks, bound=3e-2, max_escape_cal=5e-4):
    """Surrogate with exact fallback for g g -> t t~ g, with a stated error bound.

    Train on exact FP64 ratios of 500k events x 64 random points (30000 Adam steps of
    8192, learning rate 1e-3 -> 3e-4 -> 1e-4; the alphas^3 part of the ratio exact).
    Calibrate on a held-out set (131072 events, seed 54, the 64 grid points): pick
    the fallback threshold tau on the error head and the soft/collinear guard that
    keep the most events with at most max_escape_cal of the kept pairs off by more
    than the bound in log weight.  Then reweight 4M other events (seed 53) x 64 grid
    points, falling back to the exact mixed-precision kernel (its own bound 1e-3 is
    below the surrogate's), and measure against the FP64 kernel (equal to the oracle
    to 1e-12 by the parity tests): the escape rate of the kept pairs, the fallback
    rate and the largest error kept."""
    import torch
    from paper_2510_05100_b300 import rex

    g = np.random.default_rng(52)
    train_pts = [dict(mt=float(m), wt=0.0, alphas=float(a))
                 for m, a in zip(g.uniform(170.0, 176.0, 64), g.uniform(0.110, 0.126, 64))]
    exact64 = rex.Process(PROC, rex.FP64)
    exact64.set_params(ORIGINAL)
    ntr = 500_000
    mom_tr = torch.from_numpy(ps.make_events(PROC, ntr, 51)).to(dev)
    ratio = exact64.reweight(mom_tr, torch.ones(ntr, dtype=torch.float64, device=dev), train_pts, stream=stream)
    sur = rex.Surrogate(5)
    sur.set_exact_alphas(ORIGINAL["alphas"], 3)
    phases = [(16000, 1e-3), (8000, 3e-4), (6000, 1e-4)]
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    losses = np.concatenate([sur.train(mom_tr, ratio, train_pts, steps=st, batch=8192, lr=lr, seed=7, stream=stream)
                             for st, lr in phases])
    t_train = time.perf_counter() - t0
    del mom_tr, ratio

    pts = ps.grid_64()
    ncal = 131072
    mom_cal = torch.from_numpy(ps.make_events(PROC, ncal, 54)).to(dev)
    cal = sur.calibrate(exact64, mom_cal, pts, bound, max_escape_cal, stream=stream)
    del mom_cal
    tau = cal["tau"]

    nin = 4_000_000
    mom = torch.from_numpy(ps.make_events(PROC, nin, 53)).to(dev)
    w = torch.ones(nin, dtype=torch.float64, device=dev)
    out = torch.empty((nin, len(pts)), dtype=torch.float64, device=dev)
    err = torch.empty((nin, len(pts)), dtype=torch.float32, device=dev)
    mixed = rex.Process(PROC, rex.MIXED)
    mixed.set_params(ORIGINAL)

    def timed(fn):
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        r = fn()
        torch.cuda.synchronize(dev)
        return max_over_ranks(time.perf_counter() - t), r

    sur.reweight(mom[:8192], w[:8192], pts, tau=tau, exact=mixed, w_out=out[:8192], stream=stream)   # warm-up
    t_sur, nfb = timed(lambda: sur.reweight(mom, w, pts, tau=tau, exact=mixed, w_out=out, err=err, stream=stream))
    # the network alone (fused tcgen05 kernel, no fallback), timed with CUDA events on the stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tmp = torch.empty_like(out)
    e0.record(stream)
    sur.reweight(mom, w, pts, w_out=tmp, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t_net = e0.elapsed_time(e1) * 1e-3
    ref = torch.empty_like(out)
    t_fp64, _ = timed(lambda: exact64.reweight(mom, w, pts, w_out=ref, stream=stream))
    mixed.reweight(mom[:8192], w[:8192], pts, w_out=tmp[:8192], stream=stream)
    t_mix, _ = timed(lambda: mixed.reweight(mom, w, pts, w_out=tmp, stream=stream))
    dlog = (out / ref).log().abs()
    flagged = (err > tau).any(dim=1) | ~(_soft_collinear_y(mom) >= cal["guard"])
    kept = dlog[~flagged]
    units = nin * len(pts) * world
    net_flops = nin * len(pts) * 2 * (32 * 256 + 3 * 256 * 256 + 256 * 2)
    peak = PEAKS.get("bf16_tflops")
    res = {"workload": f"{PROC}: train 32M exact samples (500k events x 64 random points, "
                       f"{sum(p[0] for p in phases)} Adam steps of 8192), calibrate on 131072 held-out events x 64 "
                       f"grid points, reweight {nin} other events x 64 grid points with exact mixed-precision fallback",
           "value": units / t_sur, "unit": UNIT,
           "stated_bound": {"abs_log_weight": bound, "max_escape_rate": 1e-3,
                            "meaning": "at most 1e-3 of the pairs the network keeps are off by more than the bound "
                                       "in |log w| against the FP64 oracle; fallback pairs carry the mixed kernel's 1e-3"},
           "calibration": {"tau": tau, "guard_y_min": cal["guard"], "fallback_rate": cal["fallback_rate"],
                           "escape_rate": cal["escape_rate"], "target_escape": max_escape_cal, "events": ncal,
                           "seed": 54},
           "escape_rate": float((kept > bound).double().mean()) if kept.numel() else 0.0,
           "fallback_rate": nfb / nin, "kept_max_abs_err_log_weight": float(kept.max()) if kept.numel() else 0.0,
           "abs_err_log_weight": {"max": float(dlog.max()), "median": float(dlog.flatten()[::16].median())},
           "network_only": {"value": units / t_net, "unit": UNIT, "kernel": "fused tcgen05 (BF16, FP32 accumulation)",
                            "tensor_tflops": net_flops / t_net / 1e12,
                            "frac_of_bf16_peak": (net_flops / t_net / 1e12) / peak if peak else None,
                            "peak_tflops": peak, "peak_source": "MEASURED_PEAKS bf16_tflops (burst, of measured)"},
           "exact_fp64_value": units / t_fp64, "exact_mixed_value": units / t_mix,
           "train_seconds": t_train, "final_loss": float(losses[-50:].mean()),
           "note": "the exact mixed kernel is faster than the network on B300 (4.1e5 tensor flops per pair against "
                   "about 1e4 FP32 flops of amplitudes) and more accurate; the surrogate's value is its bounded error, "
                   "not its speed"}
    sur.close()
    return res


def run_lhe_leg(dev, stream, pts, nev=100_000):
    """The front-end around the path, file to file: read a synthetic LHE file of
    g g -> t t~ g events (interleaved with other processes), extract the process,
    reweight it to the points on the GPU (FP64, host buffers through the device),
    append one weight per point and write the file."""
    import tempfile
    import torch
    from paper_2510_05100_b300 import lhe_synth
    from paper_2510_05100_b300 import rex

    k = len(pts)
    with tempfile.TemporaryDirectory() as tmp:
        src, dst = os.path.join(tmp, "in.lhe"), os.path.join(tmp, "out.lhe")
        lhe_synth.write_lhe(src, {PROC: nev, "gg_ttx": nev // 4}, seed=9)
        size = os.path.getsize(src)
        proc = rex.Process(PROC, rex.FP64)
        proc.set_params(ORIGINAL)
        pin, pout = lhe_synth.PROCESSES[PROC]
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        L = rex.Lhe(src)
        t1 = time.perf_counter()
        mom, w, idx = L.extract(pin, pout)
        t2 = time.perf_counter()
        w_out = proc.reweight(torch.from_numpy(mom).to(dev), torch.from_numpy(w).to(dev), pts,
                              stream=stream).cpu().numpy()
        t3 = time.perf_counter()
        for j, pt in enumerate(pts):
            L.set_weights("mt%.2f_as%.4f" % (pt["mt"], pt["alphas"]), idx, w_out[:, j])
        L.write(dst)
        t4 = time.perf_counter()
        nfile = L.num_events
        L.close()
        proc.close()
    n = mom.shape[0]
    return {"workload": f"synthetic LHE v3 file of {nfile} events ({n} g g -> t t~ g, {nfile - n} g g -> t t~), "
                        f"{size / 1e6:.0f} MB; {k} weights appended per g g -> t t~ g event",
            "value": n * k / (t4 - t0), "unit": UNIT, "seconds": t4 - t0,
            "read_events_per_s": nfile / (t1 - t0), "extract_events_per_s": nfile / (t2 - t1),
            "reweight_seconds": t3 - t2, "write_events_per_s": nfile / (t4 - t3),
            "threads": os.cpu_count(), "note": "file to file through the public API; read/extract/write on the host"}


def run_qq_leg(dev, stream, pts, steps, nev=NEV):
    """q q~ -> t t~, the other leading-order channel of p p -> t t~, on the headline's
    points: nev events per launch in FP64 and in mixed precision, each timed with CUDA
    events on the launching stream, with its roofline (FP64 pipe / HBM)."""
    import torch
    from paper_2510_05100_b300 import flops as flopmod
    from paper_2510_05100_b300 import rex
    k = len(pts)
    mom = torch.from_numpy(ps.make_events("qq_ttx", nev, SEED + 100)).to(dev)
    w_in = torch.ones(nev, dtype=torch.float64, device=dev)
    w_out = torch.empty((nev, k), dtype=torch.float64, device=dev)
    # counted flops: the per-event constants, their normalisation by the original
    # point (polynomial, reciprocal, three products) and per point the polynomial and
    # the weight product; FP64 in the FP64 mode, FP32 in the mixed mode
    amp = flopmod.per_event("qq_ttx", 1)["amp"] + 8
    per_point = 6
    nbytes = nev * (16 * 8 + 8 + 8 * k)           # momenta + w_in read, w_out written
    p64 = SM_COUNT * FP64_FMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6
    out = {"workload": f"q q~ -> t t~, {nev} events x {k} points (the headline's grid and original point); "
                       "inputs + outputs exceed L2"}
    for name, prec in (("fp64", rex.FP64), ("mixed", rex.MIXED)):
        proc = rex.Process("qq_ttx", prec)
        proc.set_params(ORIGINAL)
        for _ in range(3):
            proc.reweight(mom, w_in, pts, w_out=w_out, stream=stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize(dev)
        for a, b in ev:
            a.record(stream)
            proc.reweight(mom, w_in, pts, w_out=w_out, stream=stream)
            b.record(stream)
        torch.cuda.synchronize(dev)
        proc.close()
        t = statistics.mean(a.elapsed_time(b) for a, b in ev) * 1e-3
        hbm = nbytes / t / 1e9
        fl = (amp + per_point * k) * nev
        if prec == rex.FP64:
            roof = {"bound": "alu", "pipe": "FP64 FMA", "achieved": fl / t / 1e12, "peak": p64 / 1e12,
                    "unit": "TFLOP/s", "frac": fl / t / p64, "flops_per_launch": fl}
        else:
            roof = {"bound": "hbm", "achieved": hbm, "peak": PEAKS.get("hbm_gbs"), "unit": "GB/s",
                    "frac": hbm / PEAKS["hbm_gbs"] if PEAKS.get("hbm_gbs") else None,
                    "fp32_flops_per_launch": fl, "fp32_tflops": fl / t / 1e12}
        roof["algorithmic_bytes_per_launch"] = nbytes
        out[name] = {"value": nev * k / t, "unit": UNIT, "ms_per_launch": t * 1e3, "roofline": roof}
    return out


HEL_SEED = SEED + 200   # helicity configurations of the exclusive leg's events


def helicity_inputs(nev=NEV):
    """The exclusive leg's events: the headline sample, each with a random configuration
    of its five helicities (+1/-1, int8 [nev][5])."""
    mom = ps.make_events(PROC, nev, SEED)
    hel = np.random.default_rng(HEL_SEED).choice(np.array([-1, 1], dtype=np.int8), size=(nev, 5))
    return mom, hel


def run_helicity_leg(dev, stream, pts, steps, nev=NEV):
    """Helicity-exclusive reweighting (rex_reweight_helicity) of the headline workload:
    each event reweighted with its own helicity configuration, FP64 and mixed, beside the
    helicity-summed launch on the same events.  Counted flops: the exclusive tile's
    amplitude arithmetic (its lanes evaluate the quark line for the event's antitop
    helicity only)."""
    import torch
    from paper_2510_05100_b300 import flops as flopmod
    from paper_2510_05100_b300 import rex
    k = len(pts)
    mom_np, hel_np = helicity_inputs(nev)
    mom = torch.from_numpy(mom_np).to(dev)
    hel = torch.from_numpy(hel_np).to(dev)
    w_in = torch.ones(nev, dtype=torch.float64, device=dev)
    w_out = torch.empty((nev, k), dtype=torch.float64, device=dev)
    nmass = 1 + len({p["mt"] for p in pts} - {ORIGINAL["mt"]})
    p64 = SM_COUNT * FP64_FMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6
    out = {"workload": f"{PROC}, {nev} events x {k} points, each event with a random helicity configuration "
                       "(the headline's sample and grid)",
           "stated_rel_error": {"fp64": 1e-12, "mixed": 1e-3, "double_float": 1e-12}}

    def timed(fn):
        for _ in range(2):
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize(dev)
        for a, b in ev:
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize(dev)
        return statistics.mean(a.elapsed_time(b) for a, b in ev) * 1e-3

    for name, prec in (("fp64", rex.FP64), ("mixed", rex.MIXED), ("double_float", rex.DF64)):
        proc = rex.Process(PROC, prec)
        proc.set_params(ORIGINAL)
        t = timed(lambda: proc.reweight_helicity(mom, hel, w_in, pts, w_out=w_out, stream=stream))
        t_sum = timed(lambda: proc.reweight(mom, w_in, pts, w_out=w_out, stream=stream))
        proc.close()
        cnt = flopmod.per_event(PROC, nmass, exclusive=True)
        if prec == rex.FP64:
            fl, pk, pipe = cnt["total"] * nev, p64, "FP64 FMA"
        elif prec == rex.DF64:
            fl = flopmod.per_event(PROC + "_df64", nmass, exclusive=True)["amp"] * nev
            pk, pipe = FP32_PEAK, "FP32 FMA (double-float operations; lane shuffles not counted)"
        else:
            fl, pk, pipe = cnt["amp"] * nev, FP32_PEAK, "FP32 FMA (amplitudes; FP64 invariants not counted)"
        out[name] = {"value": nev * k / t, "unit": UNIT, "ms_per_launch": t * 1e3,
                     "helicity_summed_ms_per_launch": t_sum * 1e3, "exclusive_over_summed_time": t / t_sum,
                     "roofline": {"bound": "alu", "pipe": pipe, "achieved": fl / t / 1e12, "peak": pk / 1e12,
                                  "unit": "TFLOP/s", "frac": fl / t / pk, "flops_per_launch": fl}}
    return out


def run_small_configs_leg(dev, stream, steps):
    """The two single-process workloads beside the headline.

    e+e- -> mu+mu- (gamma + Z): 4096 events (seed 1), one new electroweak point, FP64.
    4096 events fill 28 per SM, so one launch is bound by launch latency and the
    kernel's fixed cost, not by a pipe; reported with its time per launch.

    g g -> t t~: 2^20 events (seed 2) x 8 points (mt in linspace(171,175,4) x
    alphas in {0.112, 0.124}), in FP64, in mixed precision with the scalar FP32 colour
    sum (the default variant) and with the colour sum on tensor cores (the tensor-core
    variants, which need 8 lanes per event: the antitop helicity split over lanes);
    each with its roofline fraction (FP64 / FP32 FMA pipe, counted amplitude flops)."""
    import torch
    from paper_2510_05100_b300 import flops as flopmod
    from paper_2510_05100_b300 import rex

    def time_launches(proc, mom, w_in, pts, w_out, reps):
        for _ in range(3):
            proc.reweight(mom, w_in, pts, w_out=w_out, stream=stream)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            proc.reweight(mom, w_in, pts, w_out=w_out, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) * 1e-3 / reps

    out = {}
    # ---- e+e- -> mu+mu-
    nee = 4096
    mom = torch.from_numpy(ps.make_events("ee_mumu", nee, 1)).to(dev)
    w_in = torch.ones(nee, dtype=torch.float64, device=dev)
    w_out = torch.empty((nee, 1), dtype=torch.float64, device=dev)
    proc = rex.Process("ee_mumu", rex.FP64)
    proc.set_params(ps.EE_ORIGINAL)
    t = time_launches(proc, mom, w_in, [ps.EE_NEW], w_out, 200)
    # the same launches replayed from a CUDA graph: device time without the host's call overhead
    cap = torch.cuda.Stream(dev)
    cap.wait_stream(torch.cuda.current_stream(dev))
    proc.reweight(mom, w_in, [ps.EE_NEW], w_out=w_out, stream=cap)
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=cap):
        for _ in range(50):
            proc.reweight(mom, w_in, [ps.EE_NEW], w_out=w_out, stream=cap)
    graph.replay()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(4):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t_graph = e0.elapsed_time(e1) * 1e-3 / 200
    proc.close()
    out["ee_mumu"] = {"workload": "e+ e- -> mu+ mu- (gamma + Z), sqrt(s) = 500 GeV, 4096 events x 1 point "
                                  "(mZ 91.1876 -> 91.0, wZ 2.4952 -> 2.6, sin2thetaW 0.2312 -> 0.2300), FP64",
                      "value": nee / t, "unit": UNIT, "us_per_launch": t * 1e6, "launches_timed": 200,
                      "graph_replay": {"value": nee / t_graph, "us_per_launch": t_graph * 1e6,
                                       "note": "50 launches captured in one CUDA graph, replayed 4 times"},
                      "stated_rel_error": 1e-12,
                      "roofline": {"bound": "latency", "note": "28 events per SM: one launch is its fixed cost "
                                   "(launch, one block wave, the epilogue), no pipe is the limit"}}
    # ---- g g -> t t~
    n = 1 << 20
    pts = ps.grid_gg_ttx()
    k = len(pts)
    mom = torch.from_numpy(ps.make_events("gg_ttx", n, 2)).to(dev)
    w_in = torch.ones(n, dtype=torch.float64, device=dev)
    w_out = torch.empty((n, k), dtype=torch.float64, device=dev)
    nmass = 1 + len({p["mt"] for p in pts} - {ORIGINAL["mt"]})
    cnt = flopmod.per_event("gg_ttx", nmass)
    p64 = SM_COUNT * FP64_FMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6
    gg = {"workload": f"g g -> t t~, {n} events x {k} points (mt in linspace(171,175,4) x alphas in "
                      "{0.112, 0.124}); inputs + outputs exceed L2", "unit": UNIT}
    ref = None
    for name, prec, variants in (("fp64", rex.FP64, ["tuned"]), ("double_float", rex.DF64, ["tuned"]),
                                 ("mixed_scalar_colour", rex.MIXED, ["tuned"]),
                                 ("mixed_tensor_core_colour", rex.MIXED, [6, 8])):
        best = None
        for v in variants:
            proc = rex.Process("gg_ttx", prec)
            proc.set_params(ORIGINAL)
            if v == "tuned":   # rex_autotune: every variant timed on these events, the fastest kept
                tuned_ms = proc.autotune(mom, w_in, pts, w_out)
                if prec == rex.MIXED and proc.variant >= 5:   # the scalar colour form's best
                    proc.variant = int(np.argmin(tuned_ms[:5]))
            else:
                proc.variant = v
            t = time_launches(proc, mom, w_in, pts, w_out, steps)
            variant = proc.variant
            proc.close()
            if name == "fp64":
                ref = w_out.clone()
            err = None if name == "fp64" else float(((w_out / ref) - 1.0).abs().max())
            if best is None or t < best[0]:
                best = (t, variant, err)
        t, variant, err = best
        if prec == rex.FP64:
            fl, pk, pipe = cnt["total"] * n, p64, "FP64 FMA"
        elif prec == rex.DF64:
            fl = flopmod.per_event("gg_ttx_df64", nmass)["amp"] * n
            pk, pipe = FP32_PEAK, "FP32 FMA (double-float operations)"
        else:
            fl, pk, pipe = cnt["amp"] * n, FP32_PEAK, "FP32 FMA (amplitudes)"
        gg[name] = {"value": n * k / t, "unit": UNIT, "ms_per_launch": t * 1e3, "variant": variant,
                    "max_rel_err_vs_fp64": err,
                    "roofline": {"bound": "alu", "pipe": pipe, "achieved": fl / t / 1e12, "peak": pk / 1e12,
                                 "unit": "TFLOP/s", "frac": fl / t / pk, "flops_per_launch": fl}}
    out["gg_ttx"] = gg
    return out


def run_ours(args, world, rank, local):
    cpu_pool = None
    cores = os.cpu_count() or 1
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_pool = _start_pool(cores)          # spawn pool, created before any GPU call

    import torch
    from paper_2510_05100_b300 import flops as flopmod
    from paper_2510_05100_b300 import rex

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    pts = grid()
    k = len(pts)
    mom_np = ps.make_events(PROC, args.nev, rdist.rank_seed(SEED, rank))
    mom = torch.from_numpy(mom_np).to(dev)
    w_in = torch.ones(args.nev, dtype=torch.float64, device=dev)
    w_out = torch.empty((args.nev, k), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        return rdist.max_over_ranks(x, device=dev)

    def time_mode(precision: int, flags: int = 0, steps: int = args.steps, warmup: int = args.warmup,
                  sampler=None):
        proc = rex.Process(PROC, precision)
        proc.set_params(ORIGINAL)
        if flags:
            proc.set_flags(flags)
        for _ in range(warmup):
            proc.reweight(mom, w_in, pts, w_out=w_out, stream=stream)
        torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        if sampler:
            sampler.start()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for s in range(steps):
            ev[s][0].record(stream)
            proc.reweight(mom, w_in, pts, w_out=w_out, stream=stream)
            ev[s][1].record(stream)
        t1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        clocks = sampler.stop() if sampler else None
        total_ms = max_over_ranks(t0.elapsed_time(t1))
        per_launch = [a.elapsed_time(b) for a, b in ev]
        proc.close()
        return total_ms, per_launch, clocks

    props = torch.cuda.get_device_properties(dev)
    bus = None
    try:
        bus = f"{props.pci_domain_id:08X}:{props.pci_bus_id:02X}:{props.pci_device_id:02X}.0"
    except AttributeError:
        pass
    sampler = ClockSampler(bus)
    precision = rex.FP64 if args.mode == "fp64" else rex.MIXED
    total_ms, per_launch, clocks = time_mode(precision, sampler=sampler)
    value = rdist.job_throughput(args.nev * k * args.steps, world, total_ms * 1e-3)

    # ---- e2e through the host-buffer entry point (copies inside the timed region)
    h_mom = torch.from_numpy(mom_np).pin_memory()
    h_win = torch.ones(args.nev, dtype=torch.float64).pin_memory()
    h_out = torch.empty((args.nev, k), dtype=torch.float64).pin_memory()
    proc = rex.Process(PROC, precision)
    proc.set_params(ORIGINAL)
    for _ in range(max(1, args.warmup)):
        proc.reweight_host(h_mom, h_win, pts, h_out, stream=stream)
    barrier()
    e2e_steps = max(3, args.steps // 2)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        proc.reweight_host(h_mom, h_win, pts, h_out, stream=stream)
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    barrier()
    proc.close()
    e2e_value = rdist.job_throughput(args.nev * k * e2e_steps, world, e2e_s)
    h2d = h_mom.numel() * 8 + h_win.numel() * 8
    d2h = h_out.numel() * 8

    # ---- other modes on the same workload (reported beside the headline)
    extra = {}
    if not args.no_extra_modes:
        for name, prec, fl in (("fp64", rex.FP64, 0), ("mixed", rex.MIXED, 0), ("df64", rex.DF64, 0),
                               ("fp64_per_point", rex.FP64, rex.FLAG_NO_DEDUPE)):
            if name == args.mode:
                continue
            st = max(2, args.steps // 3)
            tm, per, _ = time_mode(prec, fl, steps=st, warmup=1)
            # counted flops of one launch against the pipe that carries them
            slots = (k + 1) if fl else 1 + len({p["mt"] for p in pts} - {ORIGINAL["mt"]})
            cnt = flopmod.per_event(PROC, slots)
            note = None
            if prec == rex.FP64:
                fpl, pk, pipe = cnt["total"] * args.nev, SM_COUNT * FP64_FMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6, "FP64 FMA"
            elif prec == rex.DF64:
                # the FP32 flops the double-float arithmetic performs (flopcount's df64 costs)
                fpl = flopmod.per_event(PROC + "_df64", slots)["amp"] * args.nev
                pk, pipe = FP32_PEAK, "FP32 FMA (double-float operations; FP64 invariants and ratio not counted)"
                note = {"fp64_equivalent_tflops": cnt["total"] * args.nev / (statistics.mean(per) * 1e-3) / 1e12,
                        "fp32_flops_per_fp64_flop": fpl / (cnt["total"] * args.nev)}
            else:
                fpl, pk, pipe = cnt["amp"] * args.nev, FP32_PEAK, "FP32 FMA (amplitudes; FP64 invariants and sums not counted)"
            ach = fpl / (statistics.mean(per) * 1e-3)
            e2e_mode = None
            if name == "mixed":
                # the same metric through rex_reweight_host (copies overlapped with the kernels)
                hp = rex.Process(PROC, prec)
                hp.set_params(ORIGINAL)
                for _ in range(max(1, args.warmup)):
                    hp.reweight_host(h_mom, h_win, pts, h_out, stream=stream)
                barrier()
                t0 = time.perf_counter()
                for _ in range(e2e_steps):
                    hp.reweight_host(h_mom, h_win, pts, h_out, stream=stream)
                es = max_over_ranks(time.perf_counter() - t0)
                hp.close()
                e2e_mode = {"value": rdist.job_throughput(args.nev * k * e2e_steps, world, es), "unit": UNIT,
                            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                            "entry_point": "rex_reweight_host (pinned host buffers)"}
            extra[name] = {"value": args.nev * k * st * world / (tm * 1e-3), "unit": UNIT, "e2e": e2e_mode,
                           "stated_rel_error": STATED_ERROR.get(name.split("_")[0]), "double_float": note,
                           "roofline": {"bound": "alu", "pipe": pipe, "achieved": ach / 1e12, "peak": pk / 1e12,
                                        "unit": "TFLOP/s", "frac": ach / pk}}

    # ---- roofline of the dominant kernel (the fused gg_ttxg kernel; one launch per step)
    nmass = 1 + len({p["mt"] for p in pts} - {ORIGINAL["mt"]})
    fl = flopmod.per_event(PROC, nmass)
    launch_ms = statistics.mean(per_launch)
    probe64 = rex.probe_fma(True, stream=stream)
    probe32 = rex.probe_fma(False, stream=stream)
    if args.mode == "fp64":
        flops_launch = fl["total"] * args.nev
        fma_per_clk = FP64_FMA_PER_SM_CLK
        peak = SM_COUNT * fma_per_clk * 2 * SM_MAX_MHZ * 1e6
        pipe = "FP64 FMA"
    else:
        flops_launch = fl["amp"] * args.nev
        peak = FP32_PEAK
        pipe = "FP32 FMA"
    achieved = flops_launch / (launch_ms * 1e-3)
    tr = TRAFFIC.get((PROC, args.mode))
    traffic = tr["bytes_per_launch"] if tr and tr["source_hash"] == kernel_source_hash() else None
    roofline = {"bound": "alu", "pipe": pipe, "achieved": achieved / 1e12, "peak": peak / 1e12,
                "unit": "TFLOP/s", "frac": achieved / peak if peak > 0 else None, "traffic": traffic,
                "flops_per_launch": flops_launch, "launch_ms": launch_ms,
                "peak_source": "derived: 148 SMs x FMA issue rate x 2 flop x 2032 MHz (rex_probe_fma measures the issue rate)",
                "probe_fp64_tflops": probe64 / 1e12, "probe_fp32_tflops": probe32 / 1e12,
                "algorithmic_bytes_per_launch": (args.nev * 5 * 4 * 8 + args.nev * 8 + args.nev * k * 8)}

    # ---- reweighted cross sections (Sec. 3.1.2) on the headline's output
    xsec = None
    if not args.no_xsec:
        proc = rex.Process(PROC, rex.FP64)
        proc.set_params(ORIGINAL)
        w_out = torch.empty((args.nev, k), dtype=torch.float64, device=dev)
        proc.reweight(mom, w_in, pts, w_out=w_out, stream=stream)
        proc.close()
        xs = rex.XSec(k)
        for _ in range(3):
            xs.accumulate(w_in, w_out, stream=stream)
        xs.reset(stream=stream)
        reps = 20
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(reps):
            xs.accumulate(w_in, w_out, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        t = e0.elapsed_time(e1) * 1e-3 / reps
        # a sample spread over the ranks: gather and merge the states (the one exchange)
        t0x = time.perf_counter()
        merged = rdist.allgather_merge_xsec_state(xs.get_state(stream=stream), k, rex.xsec_merge_states,
                                                  device=dev)
        xs.set_state(merged, stream=stream)
        t_exchange = time.perf_counter() - t0x
        sig, dsig, fb = xs.result(1.0, 0.01, stream=stream)
        xs.close()
        del w_out
        nbytes = args.nev * 8 + args.nev * k * 8         # w_in + w_out, read once
        hbm = PEAKS.get("hbm_gbs")
        # the per-weight sums run in double-float on the FP32 pipe (FP64 only per thread
        # and per merge): the algorithmic bound of a reduction is the bytes it reads
        xsec = {"workload": f"sigma', dsigma' of {k} points over the headline's {args.nev} events",
                "value": args.nev * k / t, "unit": UNIT, "ms_per_call": t * 1e3, "fallback_points": int(fb.sum()),
                "state_exchange_ms": t_exchange * 1e3, "ranks_merged": world,
                "roofline": {"bound": "hbm", "achieved": nbytes / t / 1e9, "peak": hbm, "unit": "GB/s",
                             "frac": nbytes / t / 1e9 / hbm if hbm else None,
                             "algorithmic_bytes_per_call": nbytes,
                             "peak_source": "MEASURED_PEAKS hbm_gbs (of measured)"}}

    small = None if args.no_qq else run_small_configs_leg(dev, stream, max(5, args.steps // 2))
    lhe_leg = None if args.no_lhe else run_lhe_leg(dev, stream, pts)
    qq_leg = None if args.no_qq else run_qq_leg(dev, stream, pts, max(5, args.steps // 2))
    qqg_leg = None if args.no_qq else run_qqg_leg(dev, stream, pts, max(3, args.steps // 4))
    hel_leg = None if args.no_helicity else run_helicity_leg(dev, stream, pts, max(3, args.steps // 4))
    pp_leg = None if args.no_qq else run_pp_ttx_leg(dev, stream, pts, max(3, args.steps // 4), world, barrier,
                                                     max_over_ranks)
    ppj_leg = None if args.no_qq else run_pp_ttx_leg(dev, stream, pts, 3, world, barrier, max_over_ranks,
                                                      spec=PP_TTXJ_BATCHES)

    multi = None if args.no_multi else run_multi_leg(dev, stream, max(3, args.steps // 2), world, barrier,
                                                     max_over_ranks)
    small_multi = None if args.no_multi else run_small_multi_leg(dev, stream, max(5, args.steps), world, barrier,
                                                                 max_over_ranks)
    surrogate = None if args.no_surrogate else run_surrogate_leg(dev, stream, world, max_over_ranks)

    cpu = None
    if cpu_pool is not None:
        sample_ev = mom_np[: 1 << 14]
        v, n, dt = oracle_throughput(sample_ev, pts, 4 * cores, 256, cores, cpu_pool)
        cpu_pool.close()
        cpu_pool.join()
        # the same oracle on one core, in this process
        t0 = time.perf_counter()
        n1 = sum(_oracle_chunk((mom_np[i * 256:(i + 1) * 256].copy(), pts)) for i in range(2))
        dt1 = time.perf_counter() - t0
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n} events of the workload x {k} points ({4 * cores} chunks of 256), {dt:.1f} s",
               "one_core": {"value": n1 * k / dt1, "unit": UNIT, "sample": f"{n1} events x {k} points, {dt1:.1f} s"},
               "cpu_model": _cpu_model()}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.mode == "fp64" else "f32+f64",
                "data": "synthetic", "stated_rel_error": STATED_ERROR[args.mode],
                "config": config_block(args, world), "clocks": clocks,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                        "entry_point": "rex_reweight_host (pinned host buffers)"},
                "gpu_launches": args.steps, "roofline": roofline, "cpu_baseline": cpu, "modes": extra,
                "multi": multi, "surrogate": surrogate, "xsec": xsec, "lhe": lhe_leg, "qq_ttx": qq_leg,
                "qq_ttxg": qqg_leg, "pp_ttx": pp_leg, "pp_ttxj": ppj_leg, "configs_1_2": small,
                "multi_small_batches": small_multi, "helicity_exclusive": hel_leg}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
