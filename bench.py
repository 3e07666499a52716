#!/usr/bin/env python3
"""Benchmark of the MPPI hot path on GB300: one JSON line on stdout.

A step is one ``mppi_step`` (noise + rollout + cost, weights, update) on the
quadrotor workload (13 states, 4 controls, RK4, 32 obstacles, K=8192,
T=150, lambda=0.5).  Metric: rollout-steps/s = K*T / step time.

  value      device time per step (CUDA events on the launch stream), inputs
             resident in HBM, L2 flushed (256 MiB write) before every step
  e2e        the same step through mppi_step_host(): pinned host inputs copied
             in and u_new + statistics copied out every step, wall-clock
  roofline   rollout kernel (the dominant one) against the FP32 pipe peak,
             measured by the library's FMA probe (the derived figure beside it)
  graph_replay  the same step captured in a CUDA graph: p50 / p99 of 1000
             replays after 50 warm-ups, L2 flushed before each
  cpu_baseline  the FP64 C oracle on this host's cores (all cores, and one
             thread on a bounded sample)
  oracle_err the oracle leg: every benchmarked form's GPU result (one untimed
             step on the bench inputs) against the FP64 oracle; per form in
             extensions.*.oracle_err, all forms in oracle_err_all
  extensions configuration 0 (cart-pole), the batched, differentiable,
             multi-iteration, CEM and BF16-MLP forms, the paper's diff-drive
             benchmark over its K sweep, a quadrotor K sweep

``--impl reference`` times the oracle alone as the reference arm.
Multi-GPU (torchrun): independent replicas, one per rank (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "rollout-steps/sec (K*T per mppi_step)"
UNIT = "rollout-steps/s"

# Algorithmic FP32 operations per rollout-step (FMA = 2), counted from the
# formulas; transcendentals and the integer Philox work are not counted.
#  quadrotor: RK4 (4 derivative evaluations of 60, stage combinations 169,
#    renormalisation 13) 422, quadratic cost 64, crash test over 32 spheres
#    32 x 10, noise scaling + importance term 31, compensated accumulation 4.
#  cart-pole: Euler step 30, quadratic cost 14, noise + importance term 7,
#    compensated accumulation 4.
#  diff drive (the paper's benchmark): dynamics 8, goal and angle terms 10,
#    costmap bilinear 15, noise + importance 14, compensated accumulation 4.
#  bicycle + MLP: MLP 2 (6*64 + 64*64 + 64*4) + 132 biases = 9604, kinematics
#    and Euler 20, costmap bilinear + speed cost 15, noise + importance 14,
#    compensated accumulation 4.
QUAD_FLOPS_PER_ROLLOUT_STEP = 422 + 64 + 320 + 31 + 4
FLOPS_PER_ROLLOUT_STEP = {
    "quadrotor": QUAD_FLOPS_PER_ROLLOUT_STEP,
    "cartpole": 30 + 14 + 7 + 4,
    "bicycle": 9604 + 20 + 15 + 14 + 4,
    "diffdrive": 8 + 10 + 15 + 14 + 4,
}
KERNEL_NAME = {
    "quadrotor": "quad_pair_kernel<true,false> (one sample per thread; dynamics, two noise and "
                 "a cost warp per 32 samples)",
    "cartpole": "pair_rollout_kernel<CartpoleDyn, QuadraticCost<4,1>> (dynamics, noise and "
                "cost warps per 32 samples)",
    "bicycle": "bicycle_mlp_f32_kernel (four lanes per sample, FP32 CUDA cores)",
    "diffdrive": "pair_rollout_kernel<DiffDriveDyn, GoalCostmapCost> (dynamics, noise and "
                 "cost warps per 32 samples)",
}
# FP32 pipe: 128 FP32 lanes per SM, 2 flops per FMA.
FP32_LANES_PER_SM = 128


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def max_over_ranks(x, device, world):
    """The maximum of x over all ranks (every rank gets it); x itself when
    world == 1.  The job is as slow as its slowest replica."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(rollout_steps_per_rank, world, ms_max):
    """Whole-job rollout-steps/s: every rank processes its own replica of the
    workload (weak scaling), and the job takes the slowest rank's time."""
    return world * rollout_steps_per_rank / (ms_max * 1e-3)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 20 ms in the
    background, each with nvidia-smi's own timestamp, so that only the samples
    taken inside the timed region are summarised."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    @staticmethod
    def _epoch(stamp):
        """nvidia-smi's local-time stamp ("2026/12/03 18:40:01.123") as epoch seconds."""
        try:
            day, frac = stamp.rsplit(".", 1)
            return time.mktime(time.strptime(day, "%Y/%m/%d %H:%M:%S")) + float("0." + frac)
        except (ValueError, OverflowError):
            return None

    def stop(self, region=None):
        """Summary of the samples inside region = (t0, t1) (epoch seconds,
        widened by one sampling period); of every sample if none fell inside."""
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        return self.summarise(self.lines, region)

    @classmethod
    def summarise(cls, lines, region=None):
        rows = []
        for ln in lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 10:
                continue
            try:
                rows.append((cls._epoch(parts[0]), float(parts[2]), float(parts[3]), parts[6:10]))
            except ValueError:
                continue
        if not rows:
            return None
        inside = rows
        if region is not None:
            t0, t1 = region[0] - 0.02, region[1] + 0.02
            sel = [r for r in rows if r[0] is not None and t0 <= r[0] <= t1]
            if sel:
                inside = sel
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in inside:
            for name, flag in zip(names, r[3]):
                if flag.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r[1] for r in inside),
                "sm_max_mhz": max(r[2] for r in inside), "reasons": sorted(reasons),
                "samples": len(inside), "in_timed_region": inside is not rows or region is None}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def cpu_baseline(p, budget_s=12.0, single_budget_s=6.0):
    """The FP64 oracle as it stands on this host: all cores (OpenMP over
    samples), full workload steps until the time budget is spent (at least one
    step); and one thread on a bounded sample of the same workload."""
    import oracle
    threads = os.cpu_count() or 1
    oracle.mppi_step(dict(p, K=min(p["K"], 64)), n_threads=threads)  # build + warm
    t0 = time.perf_counter()
    n = 0
    while True:
        oracle.mppi_step(p, step=n, n_threads=threads)
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s or n >= 1000:
            break
    out = {"value": p["K"] * p["T"] * n / el, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"{n} full oracle step(s) of {p['name']} (FP64, OpenMP over samples), "
                     f"{el:.1f} s"}
    ks = min(p["K"], 512)
    ps = dict(p, K=ks)
    t0 = time.perf_counter()
    n1 = 0
    while True:
        oracle.mppi_step(ps, step=n1, n_threads=1)
        n1 += 1
        el1 = time.perf_counter() - t0
        if el1 >= single_budget_s or n1 >= 1000:
            break
    out["single_thread"] = {"value": ks * p["T"] * n1 / el1, "unit": UNIT, "cores": 1,
                            "kind": "oracle",
                            "sample": f"{n1} oracle step(s) of {ks} of the {p['K']} samples of "
                                      f"{p['name']} on one thread, {el1:.1f} s"}
    return out


def _err_sigma(u_gpu, u_ref, sigma):
    sig = np.maximum(np.asarray(sigma, np.float64), 1e-30)
    d = np.abs(np.asarray(u_gpu, np.float64).reshape(-1, len(sig)) -
               np.asarray(u_ref, np.float64).reshape(-1, len(sig)))
    return float(np.max(d / sig[None, :]))


def _crash_jump(p):
    """The cost one crash decision adds (quadrotor with spheres), else None."""
    if p["cost_kind"] != W.COST_QUAD_OBSTACLES:
        return None
    base = 2 * p["nx"] + p["nu"] + 1
    return float(p["cost_params"][base + 1]) if p["cost_params"][base] > 0 else None


def _cost_rel(S_gpu, S_ref, p=None):
    """max |dS| / max(1, |S|) over the samples, with whole crash-cost jumps (a
    step decided the other way within FP32 rounding of a sphere's surface)
    taken out and counted; returns (max relative error, samples with a jump)."""
    a, b = np.asarray(S_gpu, np.float64), np.asarray(S_ref, np.float64)
    fin = np.isfinite(a) & np.isfinite(b)
    if not fin.any():
        return 0.0, 0
    d = a[fin] - b[fin]
    jump = _crash_jump(p) if p is not None else None
    flips = 0
    if jump:
        n = np.rint(d / jump)
        flips = int(np.count_nonzero(n))
        d = d - n * jump
    return float(np.max(np.abs(d) / np.maximum(1.0, np.abs(b[fin])))), flips


def oracle_errors(probes):
    """The oracle leg: each benchmarked form's GPU result (one step on the
    bench inputs, run outside every timed region) against the FP64 oracle on
    the same seeded inputs.  u_new errors are max |du| / sigma over (t, j);
    cost errors max |dS| / max(1, |S|) over the samples; the gradient error is
    max |dg| / max |g|.  'cost_propagated' is |u(S_gpu) - u(S_oracle)| / sigma
    with the oracle's own FP64 weighting and update: the part of the u_new
    difference that FP32 cost resolution accounts for.  Crash decisions taken
    the other way (a step within FP32 rounding of a sphere's surface) are
    counted and their whole cost jumps left out of cost_max_rel."""
    import oracle
    nt = os.cpu_count() or 1
    out = {}
    for name, pr in probes.items():
        kind = pr["kind"]
        if kind == "step":
            p = pr["problem"]
            o = oracle.mppi_step(p, step=pr["step"], n_threads=nt, want_eps=True)
            wg, _, cg = oracle.weights(pr["costs"], p["lam"])
            prop = 0.0
            if cg == 0 and o["status"] == 0:
                prop = _err_sigma(np.einsum("k,ktj->tj", wg - o["w"], o["eps"]),
                                  np.zeros((p["T"], p["nu"])), p["sigma"])
            crel, flips = _cost_rel(pr["costs"], o["S"], p)
            out[name] = {"u_new_err_over_sigma": _err_sigma(pr["u_new"], o["u_new"], p["sigma"]),
                         "cost_max_rel": crel, "crash_decisions_flipped": flips,
                         "cost_propagated_over_sigma": prop,
                         "ess": float(o["stats"][3])}
        elif kind == "batched":
            errs, props, crel, flips = [], [], 0.0, 0
            for p, (u_g, S_g) in zip(pr["problems"], pr["outputs"]):
                o = oracle.mppi_step(p, n_threads=nt, want_eps=True)
                wg, _, _ = oracle.weights(S_g, p["lam"])
                errs.append(_err_sigma(u_g, o["u_new"], p["sigma"]))
                props.append(_err_sigma(np.einsum("k,ktj->tj", wg - o["w"], o["eps"]),
                                        np.zeros((p["T"], p["nu"])), p["sigma"]))
                c, f = _cost_rel(S_g, o["S"], p)
                crel, flips = max(crel, c), flips + f
            errs, props = np.array(errs), np.array(props)
            over = errs > 1e-4
            out[name] = {"u_new_err_over_sigma_max": float(errs.max()),
                         "u_new_err_over_sigma_median": float(np.median(errs)),
                         "instances": int(len(errs)),
                         "instances_above_1e-4_sigma": int(over.sum()),
                         "above_explained_by_cost_propagation": bool(
                             np.all(np.abs(errs[over] - props[over]) <= 1e-5)),
                         "cost_max_rel": crel, "crash_decisions_flipped": flips}
        elif kind == "iterate":
            p = pr["problem"]
            o = oracle.mppi_iterate(p, pr["rounds"], pr["gamma"], n_threads=nt)
            out[name] = {"u_new_err_over_sigma": _err_sigma(pr["u_new"], o["u_new"], p["sigma"])}
        elif kind == "cem":
            p = pr["problem"]
            o = oracle.cem_step(p, pr["fraction"], n_threads=nt)
            out[name] = {"u_new_err_over_sigma": _err_sigma(pr["u_new"], o["u_new"], p["sigma"]),
                         "elite_set_equal": bool(np.array_equal(np.flatnonzero(pr["weights"]),
                                                                np.flatnonzero(o["w"])))}
        elif kind == "grad":
            p = pr["problem"]
            g_o, st = oracle.mppi_grad_cartpole(p, pr["G"], n_threads=nt)
            o = oracle.mppi_step(p, n_threads=nt)
            g_g = np.asarray(pr["grad"], np.float64)
            out[name] = {"grad_rel_err": float(np.max(np.abs(g_g - g_o)) / np.max(np.abs(g_o))),
                         "u_new_err_over_sigma": _err_sigma(pr["u_new"], o["u_new"], p["sigma"])}
    return out


def reference_arm(args, p):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    threads = os.cpu_count() or 1
    # size each step so the whole run stays within about two minutes
    t0 = time.perf_counter()
    oracle.mppi_step(p, n_threads=threads)
    t_full = time.perf_counter() - t0
    total = args.steps + args.warmup
    k_sample = p["K"]
    if t_full * total > 120.0:
        k_sample = max(32, int(p["K"] * 120.0 / (t_full * total)))
    ps = dict(p, K=k_sample)
    for i in range(args.warmup):
        oracle.mppi_step(ps, step=i, n_threads=threads)
    t0 = time.perf_counter()
    for i in range(args.steps):
        oracle.mppi_step(ps, step=args.warmup + i, n_threads=threads)
    el = time.perf_counter() - t0
    ms = el * 1e3 / args.steps
    value = k_sample * p["T"] / (ms * 1e-3)
    sample = (f"{k_sample} of {p['K']} samples of {p['name']} per step, FP64 oracle, "
              f"OpenMP over samples")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(p),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def make_workload(name, K=None):
    """The benchmark workloads; the quadrotor is the headline one."""
    kw = {"K": K} if K else {}
    if name == "quadrotor":
        return W.quadrotor(**kw)
    if name == "cartpole":
        return W.cartpole(**kw)
    if name == "bicycle":
        return W.bicycle_mlp(**kw)
    if name == "diffdrive":
        return W.diff_drive(**kw)
    raise ValueError(name)


def kernel_source_hash():
    """Hash of the CUDA sources; a stored ncu traffic figure is only used while
    the kernels are unchanged since it was taken."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2409_07563_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        if fn.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(csrc, fn), "rb") as f:
                h.update(fn.encode() + f.read())
    return h.hexdigest()[:16]


def time_steps_flushed(fn, steps, flush, warmup=3):
    """Mean milliseconds of fn() with the L2 flushed before each call (CUDA
    events around each call on the current stream)."""
    import torch
    for _ in range(warmup):
        fn()
    stream = torch.cuda.current_stream()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    torch.cuda.synchronize()
    for i in range(steps):
        flush.fill_(float(i))
        starts[i].record(stream)
        fn()
        ends[i].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in zip(starts, ends)) / steps


def step_times_flushed(fn, steps, flush, warmup=3):
    """Per-call milliseconds of fn() with the L2 flushed before each call."""
    import torch
    for _ in range(warmup):
        fn()
    stream = torch.cuda.current_stream()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    torch.cuda.synchronize()
    for i in range(steps):
        flush.fill_(float(i))
        starts[i].record(stream)
        fn()
        ends[i].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in zip(starts, ends)]


def graph_replay_latency(ctl, x0, u_nom, u_new, stats, flush, steps=1000, warmup=50):
    """mppi_step captured once in a CUDA graph, then replayed: CUDA events
    around each of `steps` replays after `warmup` untimed ones, L2 flushed
    before each.  Returns p50 / p99 / mean in ms."""
    import torch
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        ctl.step_into(x0, u_nom, u_new, stats=stats)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ctl.step_into(x0, u_nom, u_new, stats=stats)
    torch.cuda.synchronize()
    t = step_times_flushed(g.replay, steps, flush, warmup=warmup)
    del g
    return {"steps": steps, "warmup": warmup, "p50_ms": float(np.percentile(t, 50)),
            "p99_ms": float(np.percentile(t, 99)), "mean_ms": float(np.mean(t)),
            "l2": "flushed before every replay"}


def extensions(m, dev, peak_tflops, bf16_peak):
    """The batched, differentiable, multi-iteration, CEM and BF16-MLP forms, and
    the paper's own diff-drive benchmark over its K sweep, on the
    same GPU, and the quadrotor on a K sweep (where the FP32 roofline fraction
    is the meaningful figure)."""
    import torch
    out = {}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    # configuration 0: cart-pole K=1024, T=100 (latency-bound: 100 dependent steps)
    p = W.cartpole()
    ctl = m.MPPI.from_problem(p)
    x0 = torch.tensor(p["x0"], dtype=torch.float32, device=dev)
    u = torch.tensor(p["u_nom"].reshape(-1), dtype=torch.float32, device=dev)
    un = torch.empty_like(u)
    st = torch.empty(4, dtype=torch.float32, device=dev)
    t = step_times_flushed(lambda: ctl.step_into(x0, u, un, stats=st), 200, flush)
    ms0 = float(np.mean(t))
    ctl.profile(True)
    for i in range(50):
        flush.fill_(float(i))
        ctl.step_into(x0, u, un, stats=st)
    torch.cuda.synchronize()
    prof = ctl.profile_read()
    ctl.profile(False)
    roll_ms = prof["rollout"][0] / max(prof["rollout"][1], 1)
    tf0 = FLOPS_PER_ROLLOUT_STEP["cartpole"] * p["K"] * p["T"] / (roll_ms * 1e-3) / 1e12
    x0_h = torch.tensor(p["x0"], dtype=torch.float32).pin_memory()
    u_h = torch.tensor(p["u_nom"].reshape(-1), dtype=torch.float32).pin_memory()
    un_h = torch.empty_like(u_h).pin_memory()
    st_h = torch.empty(4, dtype=torch.float32).pin_memory()
    for _ in range(3):
        ctl.step_host_ptr(x0_h.data_ptr(), u_h.data_ptr(), un_h.data_ptr(), st_h.data_ptr())
    t0 = time.perf_counter()
    for _ in range(200):
        ctl.step_host_ptr(x0_h.data_ptr(), u_h.data_ptr(), un_h.data_ptr(), st_h.data_ptr())
    e2e0 = (time.perf_counter() - t0) * 1e3 / 200
    out["cartpole"] = {"workload": "cart-pole K=1024 T=100 (configuration 0)",
                       "ms_per_step": ms0, "rollout_steps_per_s": p["K"] * p["T"] / (ms0 * 1e-3),
                       "latency_ms": {"p50": float(np.percentile(t, 50)),
                                      "p99": float(np.percentile(t, 99))},
                       "e2e_ms_per_step": e2e0, "rollout_kernel_ms": roll_ms,
                       "achieved_tflops": tf0, "fp32_roofline_frac": tf0 / peak_tflops,
                       "graph_replay": graph_replay_latency(ctl, x0, u, un, st, flush)}
    ctl.close()
    # batched: 256 instances, cart-pole and quadrotor, uneven K and T
    probs = W.batched()
    b = m.MPPIBatch(probs)
    ms = time_steps_flushed(b.step, 20, flush)
    lat = b.latency_ms()
    rs = sum(p["K"] * p["T"] for p in probs)
    flops = sum(p["K"] * p["T"] * FLOPS_PER_ROLLOUT_STEP[
        "quadrotor" if p["dyn_kind"] == W.DYN_QUADROTOR else "cartpole"] for p in probs)
    tflops = flops / (ms * 1e-3) / 1e12
    out["batched"] = {"workload": "256 instances (128 cart-pole, 128 quadrotor), K in "
                                  "{256..8192}, T in {50..200}, one graph launch per step",
                      "rollout_steps_per_s": rs / (ms * 1e-3), "ms_per_step": ms,
                      "instance_latency_ms": {"p50": float(np.percentile(lat, 50)),
                                              "p99": float(np.percentile(lat, 99))},
                      "block_threads": b.info()["block_threads"],
                      "achieved_tflops": tflops, "fp32_roofline_frac": tflops / peak_tflops}
    b.close()
    # quadrotor K sweep (configuration 1 with more samples)
    sweep = []
    for K in (32768, 131072, 524288):
        p = W.quadrotor(K=K)
        c = m.MPPI.from_problem(p)
        x0 = torch.tensor(p["x0"], dtype=torch.float32, device=dev)
        u = torch.tensor(p["u_nom"].reshape(-1), dtype=torch.float32, device=dev)
        un = torch.empty_like(u)
        ms_k = time_steps_flushed(lambda: c.step_into(x0, u, un), 10, flush)
        c.close()
        tf = QUAD_FLOPS_PER_ROLLOUT_STEP * K * p["T"] / (ms_k * 1e-3) / 1e12
        sweep.append({"K": K, "ms_per_step": ms_k, "rollout_steps_per_s": K * p["T"] / (ms_k * 1e-3),
                      "achieved_tflops": tf, "fp32_roofline_frac": tf / peak_tflops})
    out["quadrotor_k_sweep"] = sweep
    # differentiable: cart-pole K=4096, T=100, forward + adjoint backward
    p = W.differentiable()
    ctl = m.MPPI.from_problem(p)
    x0 = torch.tensor(p["x0"], dtype=torch.float32, device=dev)
    u = torch.tensor(p["u_nom"].reshape(-1), dtype=torch.float32, device=dev)
    tgt = torch.tensor(p["u_target"].reshape(-1), dtype=torch.float32, device=dev)
    un = torch.empty_like(u)
    gbuf = torch.empty_like(u)

    def fwd_bwd():
        ctl.step_into(x0, u, un)
        torch.mul(torch.sub(un, tgt), 2.0, out=gbuf)
        ctl.backward(gbuf)
    ms_f = time_steps_flushed(lambda: ctl.step_into(x0, u, un), 20, flush)
    ms_fb = time_steps_flushed(fwd_bwd, 20, flush)
    out["differentiable"] = {"workload": "cart-pole K=4096 T=100, loss ||u_new - u_target||^2, "
                                         "grads w.r.t. Q(4), R, l, m_c",
                             "forward_ms": ms_f, "forward_backward_ms": ms_fb,
                             "rollout_steps_per_s": p["K"] * p["T"] / (ms_fb * 1e-3)}
    ctl.close()
    # multi-iteration MPPI with the DMD-MPC step size (Algorithm 1's outer
    # loop, Sec. V-B), the output trajectory and the MPC shift (Sec. IV-A)
    p = W.quadrotor()
    ctl = m.MPPI.from_problem(p)
    x0 = torch.tensor(p["x0"], dtype=torch.float32, device=dev)
    u = torch.tensor(p["u_nom"].reshape(-1), dtype=torch.float32, device=dev)
    un = torch.empty_like(u)
    rounds, gamma = 3, 0.5
    ctl.set_iterations(rounds, gamma)
    ms_it = time_steps_flushed(lambda: ctl.step_into(x0, u, un), 20, flush)
    ms_traj = time_steps_flushed(lambda: ctl.nominal_trajectory(x0, un), 20, flush)
    ms_shift = time_steps_flushed(lambda: ctl.shift(un, 1), 20, flush)
    out["multi_iteration"] = {"workload": f"quadrotor K={p['K']} T={p['T']}, {rounds} rounds, "
                                          f"step size {gamma}",
                              "ms_per_step": ms_it, "ms_per_round": ms_it / rounds,
                              "rollout_steps_per_s": rounds * p["K"] * p["T"] / (ms_it * 1e-3),
                              "nominal_trajectory_ms": ms_traj, "shift_ms": ms_shift}
    ctl.close()
    # CEM elite-set weights (Sec. IV-C) on the same workload, one round
    ctl = m.MPPI.from_problem(p)
    ctl.set_cem(0.1)
    ms_cem = time_steps_flushed(lambda: ctl.step_into(x0, u, un), 20, flush)
    ctl.profile(True)
    for _ in range(10):
        ctl.step_into(x0, u, un)
    prof = ctl.profile_read()
    ctl.profile(False)
    out["cem"] = {"workload": f"quadrotor K={p['K']} T={p['T']}, elite fraction 0.1",
                  "ms_per_step": ms_cem,
                  "rollout_steps_per_s": p["K"] * p["T"] / (ms_cem * 1e-3),
                  "elite_select_ms": prof["other"][0] / max(1, prof["other"][1])}
    ctl.close()
    # the paper's own benchmark: differential drive, goal + angle + costmap
    # cost, T = 100, over its K sweep; device-resident and end to end from
    # host buffers (the paper's times include the host round trips).  The
    # paper's RTX 4090 + i9-13900K times are context, not a target.
    paper_4090_ms = {128: 0.1227, 256: 0.1219, 512: 0.1236, 1024: 0.1307, 2048: 0.1462,
                     4096: 0.1700, 6144: 0.2006, 8192: 0.2316, 16384: 0.3886}
    sweep = []
    for K in W.DD_K_SWEEP:
        p = W.diff_drive(K=K)
        ctl = m.MPPI.from_problem(p)
        x0 = torch.tensor(p["x0"], dtype=torch.float32, device=dev)
        u = torch.tensor(p["u_nom"].reshape(-1), dtype=torch.float32, device=dev)
        un = torch.empty_like(u)
        ms_dev = time_steps_flushed(lambda: ctl.step_into(x0, u, un), 20, flush)
        x0_h = torch.tensor(p["x0"], dtype=torch.float32).pin_memory()
        u_h = torch.tensor(p["u_nom"].reshape(-1), dtype=torch.float32).pin_memory()
        un_h = torch.empty_like(u_h).pin_memory()
        st_h = torch.empty(4, dtype=torch.float32).pin_memory()
        for _ in range(3):
            ctl.step_host_ptr(x0_h.data_ptr(), u_h.data_ptr(), un_h.data_ptr(), st_h.data_ptr())
        t0 = time.perf_counter()
        for _ in range(50):
            ctl.step_host_ptr(x0_h.data_ptr(), u_h.data_ptr(), un_h.data_ptr(), st_h.data_ptr())
        ms_e2e = (time.perf_counter() - t0) * 1e3 / 50
        sweep.append({"K": K, "ms_per_step": ms_dev, "e2e_ms_per_step": ms_e2e,
                      "rollout_steps_per_s": K * p["T"] / (ms_dev * 1e-3),
                      "paper_rtx4090_ms": paper_4090_ms[K]})
        ctl.close()
    out["diffdrive_sweep"] = {"workload": "differential drive, goal + angle + costmap "
                                          "(110 x 110), T=100, lambda=1, sigma=0.2",
                              "points": sweep}
    # precision: bicycle + MLP, BF16 tensor cores vs FP32 CUDA cores
    p = W.bicycle_mlp()
    x0 = torch.tensor(p["x0"], dtype=torch.float32, device=dev)
    u = torch.tensor(p["u_nom"].reshape(-1), dtype=torch.float32, device=dev)
    un = torch.empty_like(u)
    res = {}
    for name, prec, var in (("bf16", m.MPPI_PREC_BF16_MLP, 0), ("fp32", m.MPPI_PREC_FP32, 0),
                            ("bf16_tcgen05", m.MPPI_PREC_BF16_MLP, 2)):
        c = m.MPPI.from_problem(p, precision=prec, rollout_variant=var)
        res[name] = time_steps_flushed(lambda: c.step_into(x0, u, un), 20, flush)
        if name in ("bf16", "bf16_tcgen05"):
            c.profile(True)
            for i in range(20):
                flush.fill_(float(i))
                c.step_into(x0, u, un)
            torch.cuda.synchronize()
            prof = c.profile_read()
            c.profile(False)
            res[name + "_rollout_kernel"] = prof["rollout"][0] / max(prof["rollout"][1], 1)
        c.close()
    mlp_tflops = 2 * (6 * 64 + 64 * 64 + 64 * 4) * p["K"] * p["T"] / (res["bf16"] * 1e-3) / 1e12
    # the 128 hidden-layer tanh per rollout-step run on the XU (MUFU) pipe:
    # 16 per clock per SM
    props = torch.cuda.get_device_properties(dev)
    xu_peak = props.multi_processor_count * 16 * measured_peaks().get("sm_max_mhz", 2070.0) * 1e6
    tanh_rate = 128 * p["K"] * p["T"] / (res["bf16"] * 1e-3)
    mlp_flops = 2 * (6 * 64 + 64 * 64 + 64 * 4) * p["K"] * p["T"]
    kmlp = mlp_flops / (res["bf16_rollout_kernel"] * 1e-3) / 1e12
    kmlp_tc = mlp_flops / (res["bf16_tcgen05_rollout_kernel"] * 1e-3) / 1e12
    out["bf16_mlp"] = {"workload": "bicycle + MLP 6-64-64-4, K=16384 T=100, costmap 512x512",
                       "kernel": "bicycle_mlp_bf16_kernel (warp-level mma.sync, weights in "
                                 "registers; the faster of the two tensor-core kernels here)",
                       "ms_per_step": res["bf16"], "fp32_ms_per_step": res["fp32"],
                       "rollout_kernel_ms": res["bf16_rollout_kernel"],
                       "kernel_mlp_tflops": kmlp,
                       "kernel_bf16_tensor_frac": kmlp / bf16_peak if bf16_peak else None,
                       "tcgen05": {"kernel": "bicycle_mlp_tc_kernel (tcgen05.mma, FP32 "
                                             "accumulators in tensor memory, two 64-sample "
                                             "tiles per CTA)",
                                   "ms_per_step": res["bf16_tcgen05"],
                                   "rollout_kernel_ms": res["bf16_tcgen05_rollout_kernel"],
                                   "kernel_mlp_tflops": kmlp_tc,
                                   "kernel_bf16_tensor_frac":
                                       kmlp_tc / bf16_peak if bf16_peak else None},
                       "rollout_steps_per_s": p["K"] * p["T"] / (res["bf16"] * 1e-3),
                       "mlp_tflops": mlp_tflops,
                       "bf16_tensor_frac": mlp_tflops / bf16_peak if bf16_peak else None,
                       "tanh_per_s": tanh_rate, "xu_tanh_frac": tanh_rate / xu_peak}
    return out


def _f32_inputs(p):
    """The problem with its inputs rounded to FP32, as the GPU receives them,
    so that the oracle starts from the same values."""
    q = dict(p)
    for key in ("dyn_params", "cost_params", "sigma", "x0", "u_nom", "map", "u_target"):
        if q.get(key) is not None:
            q[key] = np.asarray(q[key], dtype=np.float32).astype(np.float64)
    q["dt"] = float(np.float32(p["dt"]))
    q["lam"] = float(np.float32(p["lam"]))
    return q


def parity_probes(m, dev):
    """One untimed step of every benchmarked form on its bench inputs, with the
    step counter at 0, read back to the host for the oracle leg."""
    import torch

    def one_step(p, **kw):
        ctl = m.MPPI.from_problem(p, **kw)
        x0 = torch.tensor(p["x0"], dtype=torch.float32, device=dev)
        u = torch.tensor(p["u_nom"].reshape(-1), dtype=torch.float32, device=dev)
        return ctl, x0, u

    probes = {}
    for name, p, kw in (("quadrotor", W.quadrotor(), {}), ("cartpole", W.cartpole(), {}),
                        ("bicycle_fp32", W.bicycle_mlp(), {}),
                        ("bicycle_bf16", W.bicycle_mlp(), {"precision": m.MPPI_PREC_BF16_MLP}),
                        ("diffdrive", W.diff_drive(), {})):
        p = _f32_inputs(p)
        ctl, x0, u = one_step(p, **kw)
        r = ctl.step(x0, u, want_weights=True, want_costs=True)
        torch.cuda.synchronize()
        probes[name] = {"kind": "step", "problem": p, "step": 0,
                        "u_new": r["u_new"].cpu().numpy(), "costs": r["costs"].cpu().numpy()}
        ctl.close()
    # batched: every instance
    probs = [_f32_inputs(p) for p in W.batched()]
    b = m.MPPIBatch(probs)
    b.step()
    torch.cuda.synchronize()
    probes["batched"] = {"kind": "batched", "problems": probs,
                         "outputs": [(b.u_new_of(i).cpu().numpy(),
                                      b.samples_of(i)[0].cpu().numpy()) for i in range(len(probs))]}
    b.close()
    # rounds with the DMD-MPC step size, and CEM, on the headline workload
    p = _f32_inputs(W.quadrotor())
    ctl, x0, u = one_step(p)
    ctl.set_iterations(3, 0.5)
    r = ctl.step(x0, u)
    torch.cuda.synchronize()
    probes["multi_iteration"] = {"kind": "iterate", "problem": p, "rounds": 3, "gamma": 0.5,
                                 "u_new": r["u_new"].cpu().numpy()}
    ctl.close()
    ctl, x0, u = one_step(p)
    ctl.set_cem(0.1)
    r = ctl.step(x0, u, want_weights=True)
    torch.cuda.synchronize()
    probes["cem"] = {"kind": "cem", "problem": p, "fraction": float(np.float32(0.1)),
                     "u_new": r["u_new"].cpu().numpy(), "weights": r["weights"].cpu().numpy()}
    ctl.close()
    # differentiable: the adjoint gradient of sum(G u_new), G = dL/du_new
    p = _f32_inputs(W.differentiable())
    ctl, x0, u = one_step(p)
    r = ctl.step(x0, u)
    G = 2.0 * (r["u_new"].reshape(-1) - torch.tensor(p["u_target"].reshape(-1),
                                                     dtype=torch.float32, device=dev))
    grad = ctl.backward(G)
    torch.cuda.synchronize()
    probes["differentiable"] = {"kind": "grad", "problem": p,
                                "G": G.cpu().numpy().astype(np.float64).reshape(p["T"], 1),
                                "grad": grad.cpu().numpy(), "u_new": r["u_new"].cpu().numpy()}
    ctl.close()
    return probes


def fp32_peak(m):
    """The FP32 pipe peak: measured by the library's FMA probe (scalar and
    paired FMA, the faster of the two) and derived from the SM count and the
    maximum SM clock."""
    import torch
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sm_max = measured_peaks().get("sm_max_mhz", 2070.0)
    derived = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    meas = {}
    for name, pair in (("scalar_fma", False), ("f32x2_fma", True)):
        m.fp32_fma_probe(pair, 20000)                    # settle the clock
        tf, ms = m.fp32_fma_probe(pair, 400000)
        meas[name] = {"tflops": tf, "ms": ms}
    best = max(v["tflops"] for v in meas.values())
    return {"measured_tflops": best, "derived_tflops": derived, "probe": meas,
            "sms": props.multi_processor_count, "sm_max_mhz": sm_max}


def workload_config(p):
    return {"workload": f"{p['name']} (lambda={p['lam']}, seeded inputs)",
            "K": p["K"], "T": p["T"], "nx": p["nx"], "nu": p["nu"],
            "l2": "flushed by a 256 MiB write before every timed step"}


def profile_form(args):
    """Steps of the batched (configuration 3) or differentiable (configuration
    4, forward + adjoint backward) form only, for an ncu capture of their
    kernels; prints one line, measures nothing."""
    import torch
    import paper_2409_07563_gb300 as m
    m.build()
    dev = torch.device("cuda", 0)
    n = args.warmup + args.steps
    if args.profile_form == "batched":
        b = m.MPPIBatch(W.batched())
        for _ in range(n):
            b.step()
        torch.cuda.synchronize()
        b.close()
    else:
        p = W.differentiable()
        ctl = m.MPPI.from_problem(p)
        x0 = torch.tensor(p["x0"], dtype=torch.float32, device=dev)
        u = torch.tensor(p["u_nom"].reshape(-1), dtype=torch.float32, device=dev)
        tgt = torch.tensor(p["u_target"].reshape(-1), dtype=torch.float32, device=dev)
        un, g = torch.empty_like(u), torch.empty_like(u)
        for _ in range(n):
            ctl.step_into(x0, u, un)
            torch.mul(torch.sub(un, tgt), 2.0, out=g)
            ctl.backward(g)
        torch.cuda.synchronize()
        ctl.close()
    print(json.dumps({"profile_form": args.profile_form, "steps": n}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extensions", action="store_true",
                    help="skip the batched / differentiable / BF16 measurements")
    ap.add_argument("--K", type=int, default=None, help="override the sample count")
    ap.add_argument("--workload", default="quadrotor", choices=sorted(FLOPS_PER_ROLLOUT_STEP),
                    help="quadrotor (configuration 1, the headline) or a diagnostic run")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16"],
                    help="bf16: the bicycle workload's MLP on the tensor cores (diagnostic)")
    ap.add_argument("--rollout-variant", type=int, default=0,
                    help="the context's rollout_variant option (diagnostic)")
    ap.add_argument("--profile-form", default=None, choices=["batched", "differentiable"],
                    help="run only --warmup + --steps steps of one extension form and exit "
                         "(a short program for an ncu capture of its kernels; no timing)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.profile_form:
        return profile_form(args)

    p = make_workload(args.workload, args.K)
    if args.precision == "bf16" and args.workload != "bicycle":
        ap.error("--precision bf16 applies to the bicycle workload")
    if args.impl == "reference":
        return reference_arm(args, p)

    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    import paper_2409_07563_gb300 as m
    m.build()
    ctl = m.MPPI.from_problem(
        p, precision=m.MPPI_PREC_BF16_MLP if args.precision == "bf16" else m.MPPI_PREC_FP32,
        rollout_variant=args.rollout_variant)
    x0 = torch.tensor(p["x0"], dtype=torch.float32, device=dev)
    u_nom = torch.tensor(p["u_nom"].reshape(-1), dtype=torch.float32, device=dev)
    u_new = torch.empty_like(u_nom)
    stats = torch.empty(4, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        ctl.step_into(x0, u_nom, u_new, stats=stats)
    torch.cuda.synchronize()

    # ---- device-timed region ------------------------------------------------
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_region = time.perf_counter()
    wall0 = time.time()
    for i in range(args.steps):
        flush.fill_(float(i))
        starts[i].record(stream)
        ctl.step_into(x0, u_nom, u_new, stats=stats)
        ends[i].record(stream)
    torch.cuda.synchronize()
    region_s = time.perf_counter() - t_region
    wall1 = time.time()
    if world > 1:
        torch.distributed.barrier()
    # Per-kernel durations: a second pass of the same timed loop with the
    # library's event pairs around each launch (kept out of the pass above
    # because an event between the rollout and the update launch cancels
    # their programmatic-dependent-launch overlap).
    ctl.profile(True)
    for i in range(args.steps):
        flush.fill_(float(i))
        ctl.step_into(x0, u_nom, u_new, stats=stats)
    torch.cuda.synchronize()
    ctl.profile(False)
    prof = ctl.profile_read()
    clk = clocks.stop((wall0, wall1))
    per_step = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = max_over_ranks(sum(per_step) / len(per_step), dev, world)
    rollout_steps = p["K"] * p["T"]
    value = job_throughput(rollout_steps, world, ms)

    # ---- end to end through the host-buffer entry point -----------------------
    x0_h = torch.tensor(p["x0"], dtype=torch.float32).pin_memory()
    u_h = torch.tensor(p["u_nom"].reshape(-1), dtype=torch.float32).pin_memory()
    un_h = torch.empty_like(u_h).pin_memory()
    st_h = torch.empty(4, dtype=torch.float32).pin_memory()
    for _ in range(3):
        ctl.step_host_ptr(x0_h.data_ptr(), u_h.data_ptr(), un_h.data_ptr(), st_h.data_ptr())
    e2e_steps = max(20, min(args.steps, 500))
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctl.step_host_ptr(x0_h.data_ptr(), u_h.data_ptr(), un_h.data_ptr(), st_h.data_ptr())
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / e2e_steps, dev, world)
    h2d = (p["nx"] + p["T"] * p["nu"]) * 4
    d2h = (p["T"] * p["nu"] + 4) * 4

    # ---- graph-replayed latency of the same step -------------------------------
    graph = graph_replay_latency(ctl, x0, u_nom, u_new, stats, flush)

    # ---- roofline of the rollout kernel ---------------------------------------
    props = torch.cuda.get_device_properties(dev)
    peak = fp32_peak(m)
    peak_tflops = peak["measured_tflops"]
    roll_ms, roll_n = prof["rollout"]
    upd_ms, upd_n = prof["update"]
    roll_avg_ms = roll_ms / max(roll_n, 1)
    achieved = FLOPS_PER_ROLLOUT_STEP[args.workload] * rollout_steps / (roll_avg_ms * 1e-3) / 1e12
    kernel_name = KERNEL_NAME[args.workload]
    if args.precision == "bf16":
        # the MLP flops on the BF16 tensor pipe against its measured peak
        mlp = 2 * (6 * 64 + 64 * 64 + 64 * 4) * rollout_steps / (roll_avg_ms * 1e-3) / 1e12
        bf16_peak = measured_peaks().get("bf16_tflops", 1979.2)
        achieved, peak_tflops = mlp, bf16_peak
        kernel_name = ("bicycle_mlp_tc_kernel (MLP on tcgen05.mma BF16, FP32 accumulators in "
                       "tensor memory)" if args.rollout_variant == 2 else
                       "bicycle_mlp_bf16_kernel (MLP on mma.sync BF16, FP32 accumulate)")
    roofline = {"bound": "tensor" if args.precision == "bf16" else "alu",
                "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": None,
                "kernel": kernel_name,
                "kernel_ms": roll_avg_ms, "update_kernel_ms": upd_ms / max(upd_n, 1),
                "peak_note": ("measured BF16 GEMM burst (MEASURED_PEAKS.json), MLP flops only"
                              if args.precision == "bf16" else
                              "of measured: FP32 FMA rate from the library's probe "
                              "(mppi_fp32_fma_probe, the faster of scalar and f32x2 FMA chains "
                              f"on all SMs); derived {peak['derived_tflops']:.1f} TFLOP/s = "
                              f"{peak['sms']} SMs x 128 lanes x 2 x {peak['sm_max_mhz']:.0f} MHz"),
                "fp32_peak": peak}
    traffic_file = os.path.join(ROOT, "profiles", f"rollout_{args.workload}_traffic.json")
    if args.precision == "bf16":
        traffic_file = os.path.join(ROOT, "profiles", "rollout_bicycle_bf16_traffic.json")
    if os.path.exists(traffic_file):
        try:
            with open(traffic_file) as f:
                tr = json.load(f)
            if tr.get("kernel_source_hash") == kernel_source_hash() and tr.get("K") == p["K"]:
                roofline["traffic"] = tr.get("bytes_per_launch")
        except (OSError, ValueError):
            pass

    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded, workloads.py)",
        "config": workload_config(p),
        "latency_ms": {"p50": float(np.percentile(per_step, 50)),
                       "p99": float(np.percentile(per_step, 99)),
                       "region_s": region_s},
        "e2e": {"value": job_throughput(rollout_steps, world, e2e_ms), "unit": UNIT,
                "ms_per_step": e2e_ms, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": roll_n + upd_n,
        "roofline": roofline,
        "clocks": clk,
        "graph_replay": graph,
    }
    if world == 1 and not args.no_extensions and args.workload == "quadrotor":
        line["extensions"] = extensions(m, dev, peak["measured_tflops"],
                                        measured_peaks().get("bf16_tflops"))
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p)
        if args.workload == "quadrotor" and args.K is None:
            # the oracle leg: every form's GPU result against the FP64 oracle
            errs = oracle_errors(parity_probes(m, dev))
            line["oracle_err"] = errs["quadrotor"]
            for name, key in (("cartpole", "cartpole"), ("batched", "batched"),
                              ("differentiable", "differentiable"),
                              ("multi_iteration", "multi_iteration"), ("cem", "cem")):
                if "extensions" in line and key in line["extensions"]:
                    line["extensions"][key]["oracle_err"] = errs[name]
            if "extensions" in line:
                line["extensions"]["bf16_mlp"]["oracle_err"] = {
                    "bf16": errs["bicycle_bf16"], "fp32": errs["bicycle_fp32"]}
                line["extensions"]["diffdrive_sweep"]["oracle_err_K16384"] = errs["diffdrive"]
            line["oracle_err_all"] = errs
    print(json.dumps(line), flush=True)
    ctl.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
