#!/usr/bin/env python
"""Throughput of one evaluation of the 3D placement objective and gradient.

A step is one full pass of the hot path over the synthetic workload: pack the
device-resident positions, then the bistratal WA wirelength with the FD depth
gradient, the fixed-point density scatter (cells + Theorem 1 macros), the
spectral Poisson solve, the field gather and the final gradient assembly.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints ONE JSON line (rank 0).  Under torchrun every rank evaluates its own
copy of the workload (independent placement problems, weak scaling, no
collective on the data path); the timed region is bracketed by barriers and
the slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grad evals/s (WA WL + 3D density fwd+bwd) at 1M cells; % of HBM roofline"
UNIT = "grad evals/s"
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="place3d", choices=["place3d", "reference"])
    ap.add_argument("--workload", default="cells_1m", help="cells_2k|cells_200k|cells_1m|cells_4m_skewed|batch24")
    ap.add_argument("--precision", default="auto", choices=["auto", "fp32_tc", "fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="time separate launches instead of a CUDA graph")
    return ap.parse_args()


# ---------------------------------------------------------------- algorithmic bytes / flops
def algorithmic(prob: dict, precision: str) -> dict:
    """Per-evaluation algorithmic traffic of each stage: every input read once,
    every output written once (FP32 fast path; FP64 doubles the real terms)."""
    n, P, E = prob["n_inst"], prob["n_pin"], prob["n_net"]
    B = prob["nx"] * prob["ny"] * prob["nz"]
    r = 8 if precision == "fp64" else 4
    s = r // 4
    wl = 12 * s * n + (4 + 16 * s) * P + 4 * E + 12 * s * n
    scatter = 28 * s * n + 8 * B
    fwd = 2 * 2 * r * B
    zst = 3 * r * B
    inv = 11 * r * B
    gather = 28 * s * n + 12 * s * B + 12 * s * n
    prefix = 16 * B + r * B
    flops_pass = 2 * B * max(prob["nx"], prob["ny"])  # one x- or y-axis product
    tc_mult = 3 if precision == "fp32_tc" else 1        # split hi/lo: 3 products
    return dict(
        bytes=dict(wirelength=wl, scatter=scatter, prefix_densify=prefix, transform_fwd=fwd,
                   zstage=zst, transform_inv=inv, final=gather, macro_gather=0, norms=16 * s * n, prep=28 * s * n),
        flops=dict(transform_fwd=2 * flops_pass * tc_mult, transform_inv=6 * flops_pass * tc_mult))


# ---------------------------------------------------------------- multi-rank helpers
def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest value over all ranks (the slowest rank's time); identity
    without a process group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, steps: int, total_ms: float) -> float:
    """Whole-job evaluations per second: every rank evaluates `steps` times
    (weak scaling), the job ends with its slowest rank."""
    return world * steps / (total_ms / 1000.0)


# ---------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi samples (SM clock, throttle reasons) during the timed region.

    The sampler polls every 10 ms and is running (first sample seen) before
    start() returns; only samples that arrive between start() and stop()
    count.  start() comes right before the timed steps; mark() right after
    them, and extend_clock_window() then repeats the same step, untimed, until
    the window is MIN_WINDOW_S long, so the clock record holds several samples
    of this workload even when the timed steps take a few milliseconds
    ("samples_in_timed_steps" counts the ones inside the timed steps).  With no
    sample at all, the first one after the window is reported, marked "after"."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 10
    MIN_WINDOW_S = 0.15  # timed steps shorter than this are followed by the same steps, untimed


    def __init__(self, dev: int):
        self.dev = dev
        self.p = None
        self.lines = []  # (arrival time, line)
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", str(self.PERIOD_MS), "-i", str(self.dev)], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            deadline = time.time() + 10.0
            while not self.lines and time.time() < deadline and self.p.poll() is None:
                time.sleep(0.005)
        except OSError:
            self.p = None
        self.t0 = time.time()

    def _read(self):
        for line in self.p.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self):
        """End of the timed steps (samples up to here count as "during")."""
        self.t_mark = time.time()

    def stop(self) -> dict:
        self.t1 = time.time()
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        deadline = self.t1 + 1.0
        while time.time() < deadline and not any(t > self.t1 for t, _ in self.lines):
            time.sleep(0.005)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.t.join(timeout=5)
        t_mark = getattr(self, "t_mark", self.t1)
        strict = sum(1 for t, _ in self.lines if self.t0 <= t <= t_mark)
        inside = [ln for t, ln in self.lines if self.t0 <= t <= self.t1]
        where = "during"
        if not inside:
            inside = [ln for t, ln in self.lines if t > self.t1][:1]
            where = "after"
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in inside:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "sampled": where,
                "samples_in_timed_steps": strict, "window_ms": round((self.t1 - self.t0) * 1000.0, 1),
                "period_ms": self.PERIOD_MS}


def extend_clock_window(clk: Clocks, fn, torch):
    """After the timed steps: mark their end, then keep running the same step
    (untimed) until the sampler's window reaches Clocks.MIN_WINDOW_S, so that a
    short timed region still yields several clock samples of this workload."""
    clk.mark()
    while time.time() - clk.t0 < Clocks.MIN_WINDOW_S:
        for _ in range(8):
            fn()
        torch.cuda.synchronize()


def step_stats(per_step_ms) -> dict:
    """Mean and median of the per-step device times (ms)."""
    a = np.asarray(per_step_ms, np.float64)
    return {"mean_ms": float(a.mean()), "median_ms": float(np.median(a)), "min_ms": float(a.min()),
            "max_ms": float(a.max()), "steps": int(a.size)}


# ---------------------------------------------------------------- oracle legs (CPU)
def _oracle_worker(args):
    """Generate the workload once, then time `count` full oracle evaluations."""
    workload, count = args
    from oracle import Oracle
    p = make_workload(workload)
    o = Oracle(p)
    times = []
    for _ in range(count):
        t0 = time.perf_counter()
        if p.get("mode", 0) == 1:
            o.eval2d(p["x"], p["y"], p["z"], density_mode=0)
        else:
            o.eval(p["x"], p["y"], p["z"], density_mode=0, fd_mode=1)
        times.append(time.perf_counter() - t0)
    return times


def oracle_throughput(workload: str, evals: int, workers: int) -> dict:
    """`evals` full oracle evaluations split over `workers` spawned processes
    (each evaluation single-threaded).  evals/s = evals / the largest
    per-worker evaluation time (problem generation is not timed)."""
    import oracle
    oracle.build()
    workers = max(1, min(workers, evals))
    chunks = [evals // workers + (1 if k < evals % workers else 0) for k in range(workers)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        per = pool.map(_oracle_worker, [(workload, c) for c in chunks])
    busiest = max(sum(t) for t in per)
    flat = [t for ts in per for t in ts]
    return {"value": evals / busiest, "busiest_s": busiest, "per_eval_s": float(np.median(flat)),
            "evals": evals, "workers": workers}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(a):
    """The oracle (FP64 CPU, as it stands) on the host cores, same workload,
    metric and unit.  Each step is one full evaluation; steps run
    concurrently on the host cores (one per worker process)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cores = host_cores()
    oracle_throughput(a.workload, min(cores, max(a.warmup, 1)), min(cores, max(a.warmup, 1)))  # warm-up
    r = oracle_throughput(a.workload, a.steps, cores)
    ms = 1000.0 / r["value"]
    line = {
        "impl": "reference", "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": _workload_desc(a.workload), "impl": "FP64 CPU oracle"},
        "cpu_baseline": {"value": r["value"], "unit": UNIT, "cores": r["workers"], "kind": "oracle",
                         "sample": f"{a.steps} full evaluations of {a.workload} split over {r['workers']} "
                                   f"worker processes (single-threaded each); median "
                                   f"{r['per_eval_s']:.2f} s per evaluation"},
        "e2e": {"value": r["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


FILLER_U = 0.8  # maximum utilisation of each die for the "<base>_fillers" workloads


def make_workload(name: str) -> dict:
    """A named synthetic problem.  "<base>_fillers" appends the dummy fillers
    of eqs. filler-vol / free-filler-vol (u+ = u- = 0.8) to <base>, spread
    uniformly over the region (a mid-placement state).  "<base>_2d" is the
    multi-die 2D problem (eq. 2d-place) of <base>'s placement: partition from
    z, one HBT per crossing net at its optimal-region centre; "<base>_2d_fillers"
    adds the dies' fillers (die area minus instance area, spread uniformly)."""
    from paper_2403_09070_gb300 import fillers, place2d, synth
    if name.endswith("_2d_fillers"):
        p = synth.make_problem(name[:-len("_2d_fillers")])
        return place2d.from_3d(p, fillers=True, seed=11)
    if name.endswith("_2d"):
        return place2d.from_3d(synth.make_problem(name[:-len("_2d")]), fillers=False)
    if name.endswith("_fillers"):
        p = synth.make_problem(name[:-len("_fillers")])
        return fillers.insert(p, FILLER_U, FILLER_U, seed=11, positions="uniform")
    return synth.make_problem(name)


def _workload_desc(name, prob=None):
    from paper_2403_09070_gb300 import synth
    base = name
    for suf in ("_2d_fillers", "_2d", "_fillers"):
        if base.endswith(suf):
            base = base[:-len(suf)]
            break
    w = synth.WORKLOADS[base]
    d = (f"{name}: {w.n_std} std cells + {w.n_macro} macros, {w.n_net} nets (+{w.n_hifanout} high-fanout), "
         f"{w.die:g}x{w.die:g} dies, {w.nx}x{w.ny}x{w.nz} bins")
    if prob is not None and prob.get("mode", 0) == 1:
        d += (f"; multi-die 2D (eq. 2d-place): {int(prob['is_hbt'].sum())} HBTs at optimal-region centres, "
              f"{prob['nx']}x{prob['ny']} bins x 3 layers")
        if "fillers" in prob:
            f = prob["fillers"]
            d += f", {f['n_top']} top / {f['n_bot']} bottom die fillers"
    elif prob is not None and "fillers" in prob:
        f = prob["fillers"]
        d += (f" + {f['n_top']} top / {f['n_bot']} bottom z-fixed and {f['n_free']} free fillers "
              f"(u+ = u- = {FILLER_U})")
    return d


# ---------------------------------------------------------------- batch workload
def run_batch(a):
    """24 independent instances of uneven size (cell counts log-uniform in
    5k..300k, per-instance grids 64x64x2 .. 512x512x4) evaluated by one CUDA
    graph launch per step; grad evals/s counts instance evaluations."""
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2403_09070_gb300 import place3d as P
    from paper_2403_09070_gb300 import synth
    probs = synth.make_batch(24, seed=4)
    stream = torch.cuda.current_stream()
    hs, xyz, gs = [], [], []
    for p in probs:
        prec = "fp32_tc" if p["nx"] % 128 == 0 else "fp32"
        h = P.Place3D(p, precision=prec, device=local, stream=stream)
        v = [torch.tensor(p[k], device="cuda", dtype=torch.float32) for k in ("x", "y", "z")]
        h.set_positions(*v)
        h.autotune(2)
        hs.append(h)
        xyz.append(v)
        gs.append([torch.empty(p["n_inst"], device="cuda", dtype=torch.float32) for _ in range(3)])
    batch = P.Batch(hs)
    cols = [[v[k] for v in xyz] for k in range(3)] + [[g[k] for g in gs] for k in range(3)]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def one_graph():
        batch.eval(*cols, stream=stream)

    def sequential():
        for h, v, g in zip(hs, xyz, gs):
            h.eval_graph(*v, *g)

    def timed(fn, k):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for i in range(k):
            flush.zero_()
            ev[i][0].record(stream)
            fn()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        per = [e0.elapsed_time(e1) for e0, e1 in ev]
        timed.last = per
        return max_over_ranks(float(sum(per)), dist if world > 1 else None, "cuda")

    for _ in range(a.warmup):
        one_graph()
        sequential()
    torch.cuda.synchronize()
    clk = Clocks(local)
    clk.start()
    torch.cuda.nvtx.range_push("timed_batch")
    ms = timed(one_graph, a.steps)
    torch.cuda.nvtx.range_pop()
    per_step = timed.last
    extend_clock_window(clk, one_graph, torch)
    clocks = clk.stop()
    ms_seq = timed(sequential, a.steps)
    n_total = sum(p["n_inst"] for p in probs)
    # end to end: host positions in, host gradients out, through the C ABI
    hx = [[t.cpu().pin_memory() for t in v] for v in xyz]
    hg = [[torch.empty_like(t, device="cpu").pin_memory() for t in g] for g in gs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        for v, hv in zip(xyz, hx):
            for d_, s_ in zip(v, hv):
                d_.copy_(s_, non_blocking=True)
        one_graph()
        for g, hgg in zip(gs, hg):
            for s_, d_ in zip(g, hgg):
                d_.copy_(s_, non_blocking=True)
        torch.cuda.synchronize()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1000.0, dist if world > 1 else None, "cuda")
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    alg = sum(sum(algorithmic(p, "fp32")["bytes"].values()) for p in probs)
    ach = alg / (ms / a.steps * 1e6)
    hbm = peaks.get("hbm_gbs", 6800.0)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": job_throughput(world, a.steps * len(probs), ms), "unit": UNIT,
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps,
            "step_ms": step_stats(per_step),
            "median_evals_per_s": len(probs) * 1000.0 / step_stats(per_step)["median_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (transforms bf16x3 split on tensor cores where N_x, N_y are multiples of 128)",
            "data": "synthetic",
            "config": {"workload": f"batch24: 24 instances, {n_total} instances in total, cells log-uniform in "
                                   f"5k..300k, grids 64x64x2..512x512x4, one CUDA-graph launch per step",
                       "l2": "flushed between timed steps", "parallelism": f"replicas x{world}"},
            "sequential_graphs_evals_per_s": job_throughput(world, a.steps * len(probs), ms_seq),
            "shared_stages": ("wirelength stage (zeroing, packing, degree groups, norms, reductions): one launch "
                              "per stage for all 24 instances" if batch.shared_stages() else "none"),
            "e2e": {"value": job_throughput(world, a.steps * len(probs), e2e_ms), "unit": UNIT,
                    "h2d_bytes_per_step": 12 * n_total, "d2h_bytes_per_step": 12 * n_total},
            "gpu_launches": a.steps * sum(h.launches_per_eval() + 1 for h in hs),
            "roofline": {"bound": "hbm", "kernel": "whole batch step", "achieved": ach, "peak": hbm,
                         "unit": "GB/s", "frac": ach / hbm, "traffic": None},
            "clocks": clocks}), flush=True)
    batch.close()
    for h in hs:
        h.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- GPU arm
def main():
    a = _args()
    if a.impl == "reference":
        return run_reference(a)
    if a.workload == "batch24":
        return run_batch(a)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cores = host_cores()
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        # before the first GPU call (the pool is spawned, but keep it simple)
        cpu = oracle_throughput(a.workload, min(cores, 16), min(cores, 16))  # one evaluation per core
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2403_09070_gb300 import place3d as P
    from paper_2403_09070_gb300 import synth

    prob = make_workload(a.workload)
    n = prob["n_inst"]
    precision = a.precision
    if precision == "auto":
        precision = "fp32_tc"
        try:
            P.Place3D(synth.make_problem("cells_2k", n_std=64, n_net=16) | {"nx": 128, "ny": 128},
                      precision="fp32_tc", device=local).close()
        except P.Place3DError:
            precision = "fp32"
    stream = torch.cuda.current_stream()
    dt = torch.float64 if precision == "fp64" else torch.float32
    h = P.Place3D(prob, precision=precision, device=local, stream=stream)
    xyz = [torch.tensor(prob[k], device="cuda", dtype=dt) for k in ("x", "y", "z")]
    grads = [torch.empty(n, device="cuda", dtype=dt) for _ in range(3)]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def step_launches():
        h.set_positions(*xyz)
        h.eval(*grads, sync=False)

    def step_graph():
        h.eval_graph(*xyz, *grads)

    step = step_launches if a.no_graph else step_graph

    h.set_positions(*xyz)
    h.autotune(3)  # per-bucket reduction forms, timed on this workload

    def timed(fn, k, profile=False, tag="timed"):
        """k steps bracketed by barriers + syncs; per-step CUDA events on the
        launching stream, L2 flushed between steps outside the event pairs.
        The steps sit in an NVTX range named `tag` (a profiler filter)."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        if profile:
            h.stage_times(reset=True)
            h.set_profiling(True)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push(tag)
        for i in range(k):
            flush.zero_()
            ev[i][0].record(stream)
            fn()
            ev[i][1].record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        st = None
        if profile:
            h.set_profiling(False)
            st = h.stage_times(reset=True)
        per = [e0.elapsed_time(e1) for e0, e1 in ev]
        timed.last = per
        tot = max_over_ranks(float(sum(per)), dist if world > 1 else None, "cuda")
        return tot, st

    for _ in range(a.warmup):
        flush.zero_()
        step()
        flush.zero_()
        (step_launches if step is step_graph else step_graph)()
    torch.cuda.synchronize()
    # timed region A: the measured path (CUDA graph unless --no-graph), clocks sampled
    clk = Clocks(local)
    clk.start()
    total_ms, st_a = timed(step, a.steps, profile=step is step_launches, tag="timed_main")
    per_step = timed.last
    extend_clock_window(clk, step, torch)
    clocks = clk.stop()
    # timed region B: separate launches with per-stage CUDA events (stages and roofline)
    total_b_ms, st = timed(step_launches, a.steps, profile=True, tag="timed_launches")
    if st_a is not None:
        st = st_a
    alt_rate = job_throughput(world, a.steps, total_b_ms)
    res = h.get_result()
    h_forms = h.wl_forms()
    h_tiles = h.tc_tiles()
    launches = h.launches_per_eval() + 1  # + the position-packing kernel
    value = job_throughput(world, a.steps, total_ms)

    # timed region C: the same evaluation on a handle whose two paths share one
    # stream (PLACE3D_FLAG_SERIAL), per-stage CUDA events: each stage's kernels
    # run alone, so a stage's time is its kernels' own launch durations (the
    # roofline); region B's stage times are the concurrent ones.  The serial
    # handle takes the launch plan that is fastest alone (its own autotuning);
    # the concurrent graph may prefer finer wirelength launch groups, whose
    # kernels alone are timed after it for comparison.
    hs = P.Place3D(prob, precision=precision, device=local, stream=stream, flags=P.FLAG_SERIAL)
    hs.set_positions(*xyz)
    hs.autotune(3)
    hs_forms = hs.wl_forms()

    def serial_stages(k, tag):
        for _ in range(max(a.warmup, 1)):
            hs.eval(*grads, sync=False)
        torch.cuda.synchronize()
        hs.stage_times(reset=True)
        hs.set_profiling(True)
        torch.cuda.nvtx.range_push(tag)
        for _ in range(k):
            flush.zero_()
            hs.set_positions(*xyz)
            hs.eval(*grads, sync=False)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        hs.set_profiling(False)
        return hs.stage_times(reset=True)

    st_serial = serial_stages(a.steps, "timed_serial")
    st_serial_main = None
    if hs_forms != h_forms:
        hs.set_wl_plan(h_forms)
        st_serial_main = serial_stages(max(a.steps // 4, 3), "timed_serial_main_plan")
    hs.close()

    # roofline of the dominant stage (per-stage CUDA events on the launching stream)
    alg = algorithmic(prob, precision)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    bf16_peak = peaks.get("bf16_tflops_sustained", 1700.0)

    def stage_table(stt):
        evals = max(stt["evals"], 1)
        out = {}
        for name, (ms, nl) in stt["stages"].items():
            if nl == 0:
                continue
            t_eval = ms / evals
            b = alg["bytes"].get(name, 0)
            out[name] = {"ms_per_eval": t_eval, "launches_per_eval": nl / evals,
                         "alg_bytes": b, "gbs": b / (t_eval * 1e6) if t_eval > 0 and b else None}
            if name in alg["flops"]:
                out[name]["tflops"] = alg["flops"][name] / (t_eval * 1e9) if t_eval > 0 else None
        return out

    stages_conc = stage_table(st)
    stages = stage_table(st_serial)
    dom = max(stages, key=lambda k: stages[k]["ms_per_eval"])
    prof_traffic = _profiled_traffic(dom, a.workload, precision)
    if dom in ("transform_fwd", "transform_inv") and precision == "fp32_tc":
        ach = stages[dom]["tflops"]
        roof = {"bound": "tensor", "kernel": dom, "achieved": ach, "peak": bf16_peak, "unit": "TFLOP/s",
                "frac": ach / bf16_peak, "traffic": prof_traffic, "peak_source": "measured (bf16 sustained)"}
    else:
        ach = stages[dom]["gbs"]
        roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak if ach else None, "traffic": prof_traffic,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback"}
        if dom == "wirelength":
            roof["limiter"] = ("latency and issue, not DRAM: ncu shows the group kernels issuing on 56-58 % of "
                               "active cycles at 28 % occupancy (96 registers) with 14-19 % of DRAM peak, "
                               "16-30 warp instructions per pin (profiles/ncu_wirelength_cells_1m.md)")
    roof["timing"] = ("the stage's kernels timed alone (serial stream, CUDA events over K steps, L2 flushed "
                      "between steps) in the launch plan fastest alone; "
                      f"timed concurrently with the other path: {stages_conc.get(dom, {}).get('gbs')} GB/s")
    roof["plan"] = hs_forms
    if st_serial_main is not None:
        alone_main = stage_table(st_serial_main).get(dom, {})
        roof["headline_plan"] = {"plan": h_forms, "ms_per_eval": alone_main.get("ms_per_eval"),
                                 "gbs": alone_main.get("gbs"),
                                 "note": "the concurrent graph's launch plan, its kernels timed alone"}

    # end to end through the C ABI with pinned host buffers
    hx = [torch.tensor(prob[k], dtype=dt).pin_memory() for k in ("x", "y", "z")]
    hg = [torch.empty(n, dtype=dt).pin_memory() for _ in range(3)]
    for _ in range(2):
        h.set_positions(*hx)
        h.eval(*hg, sync=True)
    e2e_s = 0.0
    torch.cuda.nvtx.range_push("timed_e2e")
    for _ in range(a.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.set_positions(*hx)
        r2 = h.eval(*hg, sync=True)
        e2e_s += time.perf_counter() - t0
    torch.cuda.nvtx.range_pop()
    e2e_ms = max_over_ranks(e2e_s * 1000.0, dist if world > 1 else None, "cuda")
    h.close()

    fp64 = None
    if not a.no_fp64 and precision != "fp64" and rank == 0 and world == 1:
        fp64 = _fp64_plain(prob, torch, P)
    nest = None
    if rank == 0 and world == 1 and "_2d" not in a.workload:
        nest = _nesterov_rate(prob, precision, torch)

    if rank == 0:
        esz = 8 if precision == "fp64" else 4
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": total_ms / a.steps,
            "step_ms": step_stats(per_step),
            "median_evals_per_s": job_throughput(world, 1, step_stats(per_step)["median_ms"]),
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32_tc": "f32 (transforms bf16x3 split on tensor cores, f64 scalars)",
                      "fp32": "f32 (f64 scalars)", "fp64": "f64"}[precision],
            "data": "synthetic",
            "config": {"workload": _workload_desc(a.workload, prob), "precision": precision,
                       "n_inst": n, "n_pin": prob["n_pin"], "n_net": prob["n_net"],
                       "l2": "flushed between timed steps (256 MiB write, outside the step's event pair)",
                       "parallelism": f"replicas x{world}"},
            "e2e": {"value": job_throughput(world, a.steps, e2e_ms), "unit": UNIT,
                    "h2d_bytes_per_step": 3 * n * esz, "d2h_bytes_per_step": 3 * n * esz + 80,
                    "path": "place3d_set_positions + place3d_eval_objective_and_grad with page-locked host "
                            "arrays, host wall clock per step: the packing kernel reads the positions and the "
                            "final kernel writes the gradients over the CPU-GPU link; the scalars come back "
                            "by copy"},
            "gpu_launches": launches * a.steps,
            "roofline": roof,
            "stages": stages,
            "stages_concurrent": stages_conc,
            "clocks": clocks,
            "objective": res["obj"],
            "timed_path": "separate launches" if a.no_graph else "CUDA graph (pack + evaluation)",
            "separate_launches_evals_per_s": alt_rate,
            "stages_from": ("stages: a PLACE3D_FLAG_SERIAL handle with its own autotuned launch plan (the one "
                            "fastest alone), each stage's kernels alone, per-stage CUDA events over K steps (L2 "
                            "flushed between steps); stages_concurrent: the separate-launch timed region of the "
                            "main handle, both paths concurrent"),
            "wl_forms": h_forms,
            "tc_tile_columns": h_tiles,
        }
        if cpu is not None:
            line["cpu_baseline"] = {"value": cpu["value"], "unit": UNIT, "cores": cpu["workers"], "kind": "oracle",
                                    "sample": f"{cpu['evals']} full evaluations of {a.workload} on "
                                              f"{cpu['workers']} worker processes, one single-threaded "
                                              f"evaluation each; median {cpu['per_eval_s']:.2f} s per evaluation"}
        if fp64 is not None:
            line["fp64_plain"] = fp64
            line["speedup_vs_fp64_plain"] = value / fp64["value"]
        if nest is not None:
            line["nesterov"] = nest
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def _nesterov_rate(prob, precision, torch, iters=30, warmup=5, ref_iters=10):
    """Iterations per second of the Nesterov placement loop on the workload:
    the device-helper loop (NesterovPlacer.run) and the torch statement of it
    (run_reference), host wall clock with a synchronise on both sides, no
    logging inside the timed iterations."""
    from paper_2403_09070_gb300.nesterov import NesterovPlacer
    out = {}
    for name, k in (("run", iters), ("run_reference", ref_iters)):
        pl = NesterovPlacer(prob, precision=precision)
        f = getattr(pl, name)
        f(prob["x"], prob["y"], prob["z"], iters=warmup, log_every=0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f(prob["x"], prob["y"], prob["z"], iters=k, log_every=0)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1000.0 / k
        pl.obj.handle.close()
        out[name] = {"iters_per_s": 1000.0 / ms, "ms_per_iter": ms, "iters": k}
    return {"what": "preconditioned Nesterov iterations (eq. improved-precond, Lipschitz step, projection; "
                    "one evaluation each); `run` = the device helpers, `run_reference` = torch operations",
            **out}


def _fp64_plain(prob, torch, P, steps=20, warmup=3):
    """The plain FP64 GPU path on the same workload (context for the fast path)."""
    n = prob["n_inst"]
    h = P.Place3D(prob, precision="fp64", stream=torch.cuda.current_stream())
    xyz = [torch.tensor(prob[k], device="cuda", dtype=torch.float64) for k in ("x", "y", "z")]
    g = [torch.empty(n, device="cuda", dtype=torch.float64) for _ in range(3)]
    for _ in range(warmup):
        h.set_positions(*xyz)
        h.eval(*g, sync=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        h.set_positions(*xyz)
        h.eval(*g, sync=False)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    h.close()
    return {"value": 1000.0 / ms, "unit": UNIT, "ms_per_step": ms, "steps": steps}


def _profiled_traffic(stage, workload, precision):
    """DRAM bytes (read + write) per evaluation of a stage's kernels from the
    committed ncu launch list (profiles/traffic.json), or None when there is
    none or when any source file it lists has changed since the capture
    (its SHA-256 no longer matches)."""
    import hashlib
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        e = t[workload][precision][stage]
        for path, digest in e["sources"].items():
            with open(os.path.join(ROOT, path), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() != digest:
                    return None
        return e["bytes_per_eval"]
    except (OSError, ValueError, KeyError, TypeError):
        return None


if __name__ == "__main__":
    sys.exit(main())
