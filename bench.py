#!/usr/bin/env python3
"""Throughput of the fused collide-and-stream update on one (or N) GB300.

Workload (one "step"): one lattice Boltzmann time step (Eq. LB: streaming
with walls, moments, metric equilibrium, improved forcing with Christoffel
symbols and body force, BGK) of every instance of a Dean-number sweep: a
64 x 4 x 256 cylindrical channel (eta = r_i/r_o = 0.975, r_i = 1), 24
instances = 12 Dean numbers in [25, 60] x tau in {0.55, 0.6}, FP32, started
from the laminar curved-channel profile plus +-1e-4 seeded noise. The state
(2 x 258 MB) is larger than L2 (129 MB), so no L2 flush is needed.

Metric: MLUPS (million lattice-node updates per second, whole job).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch with torch.distributed.run; every rank runs the full sweep
on its own GPU (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_UPDATE = {"fp64": 2 * 41 * 8, "fp32": 2 * 41 * 4, "fp16_shifted": 2 * 41 * 2,
                    "bf16_shifted": 2 * 41 * 2}
DTYPE = {"fp64": "f64", "fp32": "f32", "fp16_shifted": "f16 storage / f32 math",
         "bf16_shifted": "bf16 storage / f32 math"}
PROFILE_FILE = os.path.join(ROOT, "profiles", "k_step_split_fp32_cyl64x4x256_b24.md")
KERNEL_SOURCES = ["paper_1411_3133_gb300/csrc/lbm_device.cuh", "paper_1411_3133_gb300/csrc/kernels.cuh",
                  "paper_1411_3133_gb300/csrc/step_launch.cuh", "paper_1411_3133_gb300/csrc/step_f32.cu",
                  "paper_1411_3133_gb300/csrc/lattice.cuh"]
METRIC = "MLUPS and % of HBM roofline at 1 GB300"


FP64_PROFILE_FILE = os.path.join(ROOT, "profiles", "k_step_fp64_cyl64x4x256_b24.md")
# the FP64 step is the plain k_step; its instruction counts depend on the
# kernel body alone
FP64_KERNEL_SOURCES = ["paper_1411_3133_gb300/csrc/lbm_device.cuh", "paper_1411_3133_gb300/csrc/kernels.cuh",
                       "paper_1411_3133_gb300/csrc/step_f64.cu", "paper_1411_3133_gb300/csrc/lattice.cuh"]


def kernel_source_hash(sources=None) -> str:
    h = hashlib.sha256()
    for p in (KERNEL_SOURCES if sources is None else sources):
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profile_value(path, key, sources=None):
    """A figure from a committed ncu summary, if the summary was taken on the
    current kernel source; else None."""
    try:
        text = open(path).read()
    except OSError:
        return None
    m_hash = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", text)
    m_val = re.search(key + r":\s*([0-9.eE+]+)", text)
    if not m_hash or not m_val or m_hash.group(1) != kernel_source_hash(sources):
        return None
    return float(m_val.group(1))


def measured_traffic():
    """DRAM bytes per launch of the FP32 split step (committed ncu summary)."""
    return profile_value(PROFILE_FILE, "dram_bytes_per_launch")


# ncu summaries of the other timed configurations: DRAM bytes of one whole
# step (all its kernels), valid for the step sources of that storage type
STEP_SOURCES = {p: ["paper_1411_3133_gb300/csrc/lbm_device.cuh", "paper_1411_3133_gb300/csrc/kernels.cuh",
                    "paper_1411_3133_gb300/csrc/step_launch.cuh", f"paper_1411_3133_gb300/csrc/step_{t}.cu",
                    "paper_1411_3133_gb300/csrc/lattice.cuh"]
                for p, t in (("fp32", "f32"), ("fp16_shifted", "h16"), ("bf16_shifted", "b16"))}
STEP_PROFILES = {("sweep", "fp16_shifted"): "k_step_split_fp16_cyl64x4x256_b24.md",
                 ("ellipsoid", "fp16_shifted"): "k_step_list_fp16_ell64x4x256_b24.md",
                 ("ellipsoid", "fp32"): "k_step_list_fp32_ell64x4x256_b24.md",
                 ("mixed", "fp32"): "k_step_list_fp32_mixed128.md"}


def step_traffic(workload, precision):
    """DRAM bytes per step of a profiled (workload, precision), else None."""
    name = STEP_PROFILES.get((workload, precision))
    if name is None:
        return None
    return profile_value(os.path.join(ROOT, "profiles", name), "dram_bytes_per_step", STEP_SOURCES[precision])


def measured_fp32_flops():
    """FP32 flops per lattice update of the region-split FP32 step, both
    kernels (ncu FFMA, FADD, FMUL thread-instruction counts, committed
    summary)."""
    return profile_value(PROFILE_FILE, "fp32_flops_per_update")


def measured_fp64_flops():
    """FP64 flops per lattice update executed by k_step<double> (ncu DFMA,
    DADD and DMUL thread-instruction counts, committed summary)."""
    return profile_value(FP64_PROFILE_FILE, "fp64_flops_per_update", FP64_KERNEL_SOURCES)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def workload_desc(precision="fp32"):
    from paper_1411_3133_gb300.workloads import cylinder_sweep
    return cylinder_sweep(precision=precision)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[4:]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        load = [r for r in rows if r[2] > 200.0] or rows
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in load:
            for name, flag in zip(names, r[3][1:]):
                if flag.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r[0] for r in load), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(load),
                "power_w_max": max(r[2] for r in rows)}


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
ORACLE_CHILD = r"""
import json, sys, time
import numpy as np
sys.path.insert(0, {root!r})
from oracle.geometry import Channel
from oracle.lbm import Params, Simulation
from paper_1411_3133_gb300.workloads import cylinder_sweep, noise_field
wl = cylinder_sweep()
ch = Channel(**wl.geometry_kwargs())
sim = Simulation(ch, Params(wl.taus[0], 1e-6))
sim.init_rest(noise_field(wl.seeds[0], ch.ncells, wl.noise_amp))
mode, steps, reps, budget = {mode!r}, {steps}, {reps}, {budget}
if mode == "full":
    sim.step(1)
    out = []
    for _ in range(reps):
        t0 = time.perf_counter()
        sim.step(steps)
        out.append(time.perf_counter() - t0)
    print(json.dumps({{"seconds": out, "cells": ch.ncells * steps}}))
else:
    # each rep updates one contiguous block of m nodes (one step of the
    # oracle restricted to those nodes), m sized so that all reps fit budget
    t0 = time.perf_counter(); sim.step_cells(np.arange(2048)); c = (time.perf_counter() - t0) / 2048
    m = int(min(ch.ncells, max(64, budget / reps / c)))
    cells = np.arange(m)
    out = []
    for _ in range(reps):
        t0 = time.perf_counter()
        sim.step_cells(cells)
        out.append(time.perf_counter() - t0)
    print(json.dumps({{"seconds": out, "cells": m}}))
"""


def time_oracle(mode: str, steps: int = 1, reps: int = 1, budget: float = 120.0):
    """Time the oracle on one instance of the workload, single-threaded BLAS,
    in a fresh process (no CUDA context). mode "full": `reps` timings of
    `steps` whole steps; mode "sample": `reps` one-step updates of a block of
    nodes sized to fit `budget` seconds in total."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    code = ORACLE_CHILD.format(root=ROOT, mode=mode, steps=steps, reps=reps, budget=budget)
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                         timeout=3600)
    if res.returncode != 0:
        raise RuntimeError(res.stderr[-2000:])
    return json.loads(res.stdout.strip().splitlines()[-1])


# ---------------------------------------------------------------------------
# multi-rank aggregation (weak scaling: every rank runs the whole workload)
# ---------------------------------------------------------------------------
def max_over_ranks(x: float, dist, device) -> float:
    """The slowest rank's time (every rank gets it); x itself without a
    process group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(world: int, units_per_rank: int, steps: int, seconds: float) -> float:
    """Node updates of all ranks per second, in millions."""
    return world * units_per_rank * steps / seconds / 1e6


def rank_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s copy of the workload (independent noise)."""
    return base + 1000 * rank


def timed_windows(runner, stream, steps: int, min_seconds: float, min_windows: int):
    """Durations (ms, CUDA events on the launching stream) of back-to-back
    windows of `steps` steps each, until their sum reaches min_seconds and
    there are at least min_windows of them."""
    import torch
    out = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    while len(out) < min_windows or sum(out) < 1e3 * min_seconds:
        ev0.record(stream)
        runner.step(steps)
        ev1.record(stream)
        ev1.synchronize()
        out.append(ev0.elapsed_time(ev1))
    return out


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
class SweepRunner:
    """24 instances of the 64 x 4 x 256 cylinder in one context (k_step)."""
    profiled = True
    launches_per_step = 1

    def __init__(self, args, L, rank):
        self.args, self.L = args, L
        wl = workload_desc(args.precision)
        self.wl = wl
        spec = L.ChannelSpec(**wl.geometry_kwargs())
        desc = spec.desc()
        params = []
        for b in range(wl.batch):
            G = L.lb_force_for_dean("cylindrical", desc, wl.taus[b], wl.deans[b])
            params.append(L.make_params(wl.taus[b], G, False, rank_seed(wl.seeds[b], rank),
                                        wl.noise_amp, True))
        self.ctx = L.LBContext(spec, batch=wl.batch, precision=wl.precision)
        self.ctx.lb_set_option(L.LB_OPT_USE_GRAPH, 1)
        self.ctx.lb_set_option(L.LB_OPT_STEP_KERNEL,
                               {"auto": 0, "plain": 1, "tma": 2, "split": 4, "tiled": 5}[args.step_kernel])
        self.ctx.lb_set_option(L.LB_OPT_BLOCK_THREADS, args.threads)
        self.ctx.lb_init(params)
        self.cells = wl.batch * wl.ncells
        self.stream = self.ctx.stream
        if args.step_kernel == "auto":      # the library's automatic choice for this workload
            args.step_kernel = "plain" if args.precision == "fp64" else "split"
        # 2-byte storage: the split kernels that keep the block's row in shared
        # memory (blocks within one i_r layer: nt n3 a multiple of the block)
        rowsm = "_rowsm" if (args.precision.endswith("_shifted")
                             and (wl.ntheta * wl.n3) % args.threads == 0) else ""
        self.kernel = {"tma": "k_step_tma<KCYL,256>",
                       "split": f"k_step_bulk{rowsm}<{args.precision},KCYL> + k_step_edge{rowsm} "
                                f"({args.threads} threads)"}.get(
            args.step_kernel, f"k_step<{args.precision},KCYL> ({args.threads} threads)")
        self.profiled = args.precision == "fp32" and args.step_kernel == "split"
        self.launches_per_step = 2 if args.step_kernel == "split" else 1

    def warmup(self, n):
        self.ctx.lb_step(n)

    def step(self, n):
        self.ctx.lb_step(n)

    def diagnostics(self):
        return self.ctx.lb_diagnostics()

    def e2e(self, steps):
        import torch
        nbytes = self.ctx.lb_state_bytes()
        host_in = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        host_out = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        self.ctx.lb_get_state(host_in)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            self.ctx.lb_set_state(host_in)
            self.ctx.lb_step(1)
            self.ctx.lb_get_state(host_out)
        torch.cuda.synchronize()
        self.state_bytes = nbytes
        return time.perf_counter() - t0, nbytes, nbytes

    def config(self):
        wl = self.wl
        return {"workload": f"Dean sweep, cylindrical channel {wl.nr}x{wl.ntheta}x{wl.n3}, "
                            f"eta=0.975, {wl.batch} instances (12 De in 25..60 x tau 0.55/0.6), "
                            f"D3Q41, {wl.precision}",
                "cells_per_instance": wl.ncells, "instances": wl.batch, "precision": wl.precision,
                "l2": f"inputs larger than L2: state {2 * self.state_bytes / 1e6:.0f} MB, no flush"}

    def extra(self):
        return {}

    def close(self):
        self.ctx.close()


class EllipsoidRunner(SweepRunner):
    """24 instances of the double-curved channel of Sec. IV.B (R2/R1 = 1,
    64 x 4 x 256, walls on r and phi), De linspace(20, 150, 24) through the
    force of the cylinder of the same streamwise radius and width, tau 0.55,
    from rest plus noise."""

    def __init__(self, args, L, rank):
        from paper_1411_3133_gb300.workloads import ellipsoid_cross_section
        self.args, self.L = args, L
        wl = ellipsoid_cross_section(1.0, precision=args.precision)
        self.wl = wl
        spec = L.ChannelSpec(**wl.geometry_kwargs())
        ref = L.make_desc(1.0, 1.0 + (wl.r_outer - wl.r_inner), wl.nr, wl.ntheta, wl.n3)
        params = [L.make_params(0.55, L.lb_force_for_dean("cylindrical", ref, 0.55, float(de)), False,
                                rank_seed(wl.seeds[0] + b, rank), 1e-4, False)
                  for b, de in enumerate(__import__("numpy").linspace(20, 150, 24))]
        self.batch = 24
        self.ctx = L.LBContext(spec, batch=24, precision=args.precision)
        self.ctx.lb_set_option(L.LB_OPT_USE_GRAPH, 1)
        self.ctx.lb_set_option(L.LB_OPT_STEP_KERNEL,
                               {"auto": 0, "plain": 1, "tma": 2, "split": 4, "tiled": 5}[args.step_kernel])
        self.ctx.lb_set_option(L.LB_OPT_BLOCK_THREADS, args.threads)
        self.ctx.lb_init(params)
        self.cells = 24 * wl.ncells
        self.stream = self.ctx.stream
        if args.step_kernel == "auto":
            args.step_kernel = "plain" if args.precision == "fp64" else "tiled"
        self.kernel = {"tiled": f"k_step_list<{args.precision},KELL> interior + wall tiles ({args.threads} threads)"
                       }.get(args.step_kernel, f"k_step<{args.precision},KELL> ({args.threads} threads)")
        self.profiled = False
        self.launches_per_step = work_lists([wl] * 24) if args.step_kernel == "tiled" else 1

    def config(self):
        wl = self.wl
        return {"workload": f"double-curved channel (ellipsoidal coordinates, R2/R1 = 1, d = R1/40) "
                            f"{wl.nr}x{wl.ntheta}x{wl.n3}, walls on r and phi, 24 instances (De 20..150), "
                            f"D3Q41, {self.args.precision}",
                "cells_per_instance": wl.ncells, "instances": 24, "precision": self.args.precision,
                "l2": f"inputs larger than L2: state {2 * self.state_bytes / 1e6:.0f} MB, no flush"}


def work_lists(channels):
    """Work-list launches of one tiled or batch step over `channels` (objects
    with metric, nr, n3, periodic3 and wall): per metric kind the interior
    tiles and each non-empty wall-node class the library builds -- nodes
    near an r-wall only, near an x3-wall only, and the rest (corners and
    equilibrium walls)."""
    kinds = {}
    for ch in channels:
        lists = kinds.setdefault(ch.metric, set())
        walled3 = not ch.periodic3
        if ch.nr > 6 and (not walled3 or ch.n3 > 6):
            lists.add("interior")
        if getattr(ch, "wall", "bounceback") == "equilibrium":
            lists.add("rest")
            continue
        lists.add("r-layer")
        if walled3:
            lists.update(("x3-layer", "rest"))
    return sum(len(v) for v in kinds.values())


class MixedRunner:
    """128 channels of mixed metric and size (cylinders and double-curved
    channels, N_r in {32, 48, 64}, N_3 in 128..512, De in 20..150) in one
    lb_batch: per metric kind and step, one k_step_list launch over the
    interior tiles and one per wall-node class; autotuned."""
    profiled = False

    def __init__(self, args, L, rank):
        from paper_1411_3133_gb300.sweep import mixed_contexts
        from paper_1411_3133_gb300.workloads import mixed_batch
        self.args, self.L = args, L
        self.insts = mixed_batch(seed=rank_seed(20241111, rank))
        self.launches_per_step = work_lists(self.insts)
        self.ctxs, self.batch = mixed_contexts(self.insts, args.precision)
        self.batch.lb_batch_set_option(L.LB_OPT_USE_GRAPH, 1)
        self.cells = self.batch.lb_batch_nodes()
        self.stream = self.ctxs[0].stream
        self.kernel = f"k_step_list<{args.precision},KCYL|KELL>"
        self.tune = None

    def warmup(self, n):
        self.tune = self.batch.lb_batch_autotune(self.args.tune_steps)
        self.batch.lb_batch_step(n)

    def step(self, n):
        self.batch.lb_batch_step(n)

    def diagnostics(self):
        return [c.lb_diagnostics()[0] for c in self.ctxs]

    def e2e(self, steps):
        import torch
        sizes = [c.lb_state_bytes() for c in self.ctxs]
        host_in = [torch.empty(n, dtype=torch.uint8, pin_memory=True) for n in sizes]
        host_out = [torch.empty(n, dtype=torch.uint8, pin_memory=True) for n in sizes]
        for c, h in zip(self.ctxs, host_in):
            c.lb_get_state(h)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            for c, h in zip(self.ctxs, host_in):
                c.lb_set_state(h)
            self.batch.lb_batch_step(1)
            for c, h in zip(self.ctxs, host_out):
                c.lb_get_state(h)
        torch.cuda.synchronize()
        self.state_bytes = sum(sizes)
        return time.perf_counter() - t0, self.state_bytes, self.state_bytes

    def config(self):
        ncyl = sum(i.metric == "cylindrical" for i in self.insts)
        return {"workload": f"mixed sweep, {len(self.insts)} channels ({ncyl} cylindrical eta=0.975, "
                            f"{len(self.insts) - ncyl} double-curved R2/R1 in 0.25..4), N_r in "
                            "{32,48,64} x 4 x N_3 in 128..512, De in 20..150, tau 0.55, D3Q41, "
                            f"{self.args.precision}, one lb_batch",
                "nodes": self.cells, "instances": len(self.insts), "precision": self.args.precision,
                "l2": f"inputs larger than L2: state {2 * self.state_bytes / 1e6:.0f} MB, no flush"}

    def extra(self):
        best, trials = self.tune
        return {"autotune": {"best": best, "trials": trials}}

    def close(self):
        self.batch.close()
        for c in self.ctxs:
            c.close()


# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--step-kernel", default="auto", choices=["auto", "plain", "tma", "split", "tiled"])
    ap.add_argument("--threads", type=int, default=128, help="threads per block of the step kernel")
    ap.add_argument("--precision", default="fp32", choices=sorted(BYTES_PER_UPDATE))
    ap.add_argument("--workload", default="sweep", choices=["sweep", "mixed", "ellipsoid"],
                    help="sweep: 24-instance 64x4x256 cylinder Dean sweep; mixed: 128 channels "
                         "of mixed metric and size in one lb_batch; ellipsoid: 24 instances of the "
                         "64x4x256 double-curved channel with four walls")
    ap.add_argument("--min-seconds", type=float, default=1.0,
                    help="repeat the K-step window until this much GPU time has accumulated")
    ap.add_argument("--min-windows", type=int, default=5, help="at least this many K-step windows")
    ap.add_argument("--tune-steps", type=int, default=20,
                    help="mixed: steps per autotuner trial (taken inside the warm-up)")
    args = ap.parse_args()
    assert args.warmup >= 3, "at least 3 warm-up steps"

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return reference_arm(args, rank)

    import numpy as np
    import torch

    from paper_1411_3133_gb300 import build as _build
    from paper_1411_3133_gb300 import lbgm as L

    _build.build()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    runner = {"mixed": MixedRunner, "ellipsoid": EllipsoidRunner}.get(args.workload, SweepRunner)(args, L, rank)
    cells = runner.cells
    stream = runner.stream

    # warm-up (the mixed batch's autotuner runs its trials inside it)
    runner.warmup(args.warmup)
    torch.cuda.synchronize()

    # timed region: K steps
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # the K-step window, repeated until at least --min-seconds of GPU time
    # (and --min-windows windows) have accumulated; the median window is the
    # measurement, so a short --steps still gives a stable number
    windows = timed_windows(runner, stream, args.steps, args.min_seconds, args.min_windows)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = statistics.median(windows)
    clocks = sampler.stop() if sampler else None
    d = runner.diagnostics()
    finite = all(x["nonfinite"] == 0 for x in d)
    ms = max_over_ranks(ms, dist, "cuda")
    sec = ms / 1e3
    value = whole_job_mlups(world, cells, args.steps, sec)
    per_launch = sec / args.steps
    bpu = BYTES_PER_UPDATE[args.precision]
    achieved = bpu * cells / per_launch / 1e9
    peak, peak_kind = peaks()
    traffic = measured_traffic() if runner.profiled else step_traffic(args.workload, args.precision)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": traffic, "peak_source": peak_kind,
                "kernel": runner.kernel, "algorithmic_bytes_per_launch": bpu * cells}
    fpu32 = measured_fp32_flops() if runner.profiled else None
    if fpu32 is not None:
        # the other roof: FP32 arithmetic against the FMA peak measured on
        # this GPU (outside the timed region); the HBM roof is the binding one
        alu_peak = L.lb_fma_peak("fp32", stream) / 1e12
        alu = fpu32 * cells / per_launch / 1e12
        roofline["alu"] = {"achieved": round(alu, 3), "peak": round(alu_peak, 3), "unit": "TFLOP/s",
                           "frac": round(alu / alu_peak, 4), "fp32_flops_per_update": fpu32,
                           "peak_source": "measured (lb_fma_peak, FP32 FMA chains on this GPU)"}
    fpu = measured_fp64_flops() if (args.precision == "fp64" and args.step_kernel == "plain"
                                    and args.workload == "sweep") else None
    if fpu is not None:
        # the FP64 step is bound by the FP64 units: report it against the
        # FMA peak measured on this GPU, outside the timed region
        alu_peak = L.lb_fma_peak("fp64", stream) / 1e12
        alu = fpu * cells / per_launch / 1e12
        roofline = {"bound": "alu", "achieved": round(alu, 4), "peak": round(alu_peak, 4),
                    "unit": "TFLOP/s", "frac": round(alu / alu_peak, 4), "traffic": None,
                    "peak_source": "measured (lb_fma_peak, FP64 FMA chains on this GPU)",
                    "kernel": runner.kernel, "fp64_flops_per_update": fpu,
                    "hbm": {"achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                            "frac": round(achieved / peak, 4), "peak_source": peak_kind}}

    # end to end through the C ABI with host buffers: each step uploads the
    # state from pinned host memory, advances it one step and reads it back
    if dist:
        dist.barrier()
    e2e_sec, h2d, d2h = runner.e2e(args.e2e_steps)
    e2e_sec = max_over_ranks(e2e_sec, dist, "cuda")
    e2e_value = whole_job_mlups(world, cells, args.e2e_steps, e2e_sec)
    runner.close()

    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            r = time_oracle("full", steps=args.cpu_steps)
            cpu = {"value": r["cells"] / sum(r["seconds"]) / 1e6, "unit": "MLUPS",
                   "cores": 1, "kind": "oracle",
                   "sample": f"{args.cpu_steps} steps of one 64x4x256 instance of the same sweep "
                             f"(numpy FP64 oracle, single-threaded BLAS, {sum(r['seconds']):.1f} s)"}
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 6),
            "windows": {"count": len(windows), "steps_each": args.steps, "statistic": "median",
                        "ms_min": round(min(windows), 4), "ms_median": round(ms, 4),
                        "ms_max": round(max(windows), 4), "gpu_seconds": round(sum(windows) / 1e3, 3)},
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": dict(runner.config(), bytes_per_update=bpu, parallelism=f"replicas x{world}"),
            "roofline": roofline,
            "e2e": {"value": round(e2e_value, 2), "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": args.e2e_steps},
            "gpu_launches": len(windows) * args.steps * runner.launches_per_step,
            "clocks": clocks,
            "cpu_baseline": cpu,
            "finite": finite,
            "dean_measured": [round(x["dean"], 3) for x in d[:3]],
        }
        line.update(runner.extra())
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def reference_arm(args, rank):
    """The oracle, as it stands, on the host cores. Each step is a bounded
    sample of the workload: one oracle update of a block of nodes of one
    instance, sized so that warm-up and timed steps take about two minutes."""
    if rank != 0:
        return
    r = time_oracle("sample", reps=args.warmup + args.steps, budget=120.0)
    secs = r["seconds"][args.warmup:]
    sec = sum(secs)
    value = r["cells"] * len(secs) / sec / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * sec / len(secs), 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "Dean sweep, cylindrical channel 64x4x256, eta=0.975, D3Q41 "
                               f"(each step: {r['cells']} nodes of one instance)",
                   "parallelism": "host, 1 core"},
        "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS", "cores": 1, "kind": "oracle",
                         "sample": f"{len(secs)} one-step updates of {r['cells']} nodes"},
        "e2e": {"value": round(value, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
