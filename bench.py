#!/usr/bin/env python
"""Benchmark of the GB300 Hermite-spline MPPI path.

Metric: MPPI rollout steps/s (step-samples per second) and solves/s of one full MPPI
update (Alg. 1: knot noise, rollouts, weights, knot average; 3 iterations) on the
single-instance scale workload: the 18-DoF quadruped, K = 8192 samples, 6 Hermite knots
over 1.0 s, dt = 0.005 (200 semi-implicit Euler steps), lambda = 0.1, random initial base
velocity. Synthetic, seeded inputs; inputs resident in HBM when the timed region starts;
L2 flushed (256 MiB write) between timed solves.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 (torchrun): every rank solves its own instance (replicas, no data-path collective);
value = all ranks' step-samples / max-over-ranks time ("scaling": "weak").
--impl reference times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MPPI rollout steps/s & solves/s on 1 GB300; p50/p99 solve latency vs plain launch"
UNIT = "rollout steps/s"
WORKLOAD = ("single-instance scale: quadruped (floating base + 12 revolute joints), K=8192 samples, "
            "6 Hermite knots over 1.0 s, H=200 steps (dt 0.005), 3 MPPI iterations per solve")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--samples", type=int, default=8192)
    ap.add_argument("--mapping", type=int, default=-1, help="-1 autotuned, 0 warp, 1 half-warp, 2 lanes-per-chain")
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-samples", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched uneven-instance workload")
    ap.add_argument("--no-receding", action="store_true", help="skip the receding-horizon cycle timing")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving workload")
    ap.add_argument("--no-configs", action="store_true", help="skip the other single-instance configurations")
    ap.add_argument("--only-config", default=None, choices=sorted(CONFIGS),
                    help="time one single-instance configuration alone and print its result (for profiling)")
    return ap.parse_args()


# ------------------------------------------------------------------------------------
# multi-rank control plane (gloo; timing only, no data-path collective)
# ------------------------------------------------------------------------------------
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world):
    if world <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group("gloo")
    return dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def reduce_max_sum(dist, t_local: float, units_local: float):
    """(max over ranks of the timed seconds, sum over ranks of the units)."""
    if dist is None:
        return t_local, units_local
    import torch
    t = torch.tensor([t_local], dtype=torch.float64)
    u = torch.tensor([units_local], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# ------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ------------------------------------------------------------------------------------
# FP32 peak of the device the bench runs on
# ------------------------------------------------------------------------------------
def device_fp32_peak(torch, index: int, flops):
    """(peak TFLOP/s, basis) from the device's SM count and maximum SM clock (nvidia-smi);
    the maximum clock falls back to 2070 MHz (GB300) when nvidia-smi cannot be asked."""
    sms = torch.cuda.get_device_properties(index).multi_processor_count
    mhz, src = 2070.0, "assumed (nvidia-smi unavailable)"
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(index), "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20).stdout
        mhz, src = float(out.strip().splitlines()[0]), "nvidia-smi clocks.max.sm"
    except Exception:
        pass
    return flops.fp32_peak_tflops(sms, mhz), (f"{sms} SMs (device query) x 128 FP32 lanes x 2 flops x {mhz:.0f} MHz "
                                             f"({src})")


# ------------------------------------------------------------------------------------
# DRAM traffic of the dominant kernel, from a committed ncu summary
# ------------------------------------------------------------------------------------
TRAFFIC_SOURCES = ["rollout_lanes.cuh", "chain_kernel.cuh", "chain_f32.cuh", "scalar_macros.h", "common.cuh",
                   "rollout_warp.cuh", "internal.h"]


def sources_sha256(names=TRAFFIC_SOURCES) -> str:
    import hashlib
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2511_19204_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def profiled_values(name: str):
    """The `- key: value` lines of profiles/<name>.md, or None when the kernel's sources
    changed since the capture (the summary records their SHA-256)."""
    path = os.path.join(ROOT, "profiles", name + ".md")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and line.startswith("- "):
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    return vals if vals.get("source-sha256") == sources_sha256() else None


def profiled_traffic(name: str, samples: int):
    """dram__bytes_read.sum + dram__bytes_write.sum per launch from profiles/<name>.md,
    scaled to `samples` if the capture used another count; None when the kernel's
    sources changed since the capture."""
    vals = profiled_values(name)
    try:
        return float(vals["dram-bytes-per-launch"]) * samples / float(vals["samples"])
    except (TypeError, KeyError, ValueError):
        return None


def profiled_fma_pipe(name: str):
    """ncu's FP32 (FMA) pipe utilisation of the captured launch, as a fraction, or None."""
    vals = profiled_values(name)
    try:
        return float(vals["fma-pipe-pct"]) / 100.0
    except (TypeError, KeyError, ValueError):
        return None


# ------------------------------------------------------------------------------------
# CPU baseline: the FP64 oracle as it stands, on the host cores
# ------------------------------------------------------------------------------------
def _timed_solves(oracle, p, nthreads, min_s=2.0):
    """Solves of p (successive noise counters) until min_s seconds of wall time have
    passed: (solves, seconds)."""
    n, t0 = 0, time.perf_counter()
    while True:
        oracle.solve_problem(p, nthreads=nthreads, iter_base=p.iters * n)
        n += 1
        dt = time.perf_counter() - t0
        if dt >= min_s:
            return n, dt


def cpu_baseline(n_samples: int):
    import oracle
    from paper_2511_19204_gb300 import synth
    oracle.build()
    p = synth.scale_quadruped(n=n_samples)
    cores = os.cpu_count() or 1
    oracle.solve_problem(p, nthreads=cores)      # warm (page faults, thread start-up)
    n, dt = _timed_solves(oracle, p, cores)
    units = p.n * p.horizon * p.iters
    # the same oracle on one thread, on an eighth of the sample
    p1 = synth.scale_quadruped(n=max(n_samples // 8, 1))
    n1, dt1 = _timed_solves(oracle, p1, 1)
    return {"value": units * n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{p.n} of 8192 samples, all {p.iters} iterations x {p.horizon} steps, {n} solves "
                      f"({dt:.2f} s wall, FP64 C oracle, {cores} threads)",
            "single_thread_value": p1.n * p1.horizon * p1.iters * n1 / dt1,
            "single_thread_sample": f"{p1.n} samples, {n1} solves, one thread ({dt1:.2f} s wall)"}


def oracle_parity(mppi, synth, mapping, block):
    """Error of one full-size solve of the headline workload against the FP64 oracle on
    the same inputs (fresh controller, the problem's nominal as warm start, counter 0):
    the largest relative error over the updated control points, the best cost's relative
    error and whether the best sample agrees. Not timed."""
    import numpy as np
    import oracle
    oracle.build()
    p = synth.scale_quadruped()
    c = mppi.Controller.from_problem(mppi.Model(p.model), p, mapping=mapping, block=block)
    nom32 = p.nominal.astype(np.float32)
    mean, best, info = c.solve(p.state, warm=nom32)
    t0 = time.perf_counter()
    ref = oracle.solve(p.model, p.n, p.nk, p.horizon, p.iters, p.dt, p.lam, p.sigma, p.state,
                       nom32.astype(np.float64), seed=p.seed)
    dt = time.perf_counter() - t0
    err = float(np.max(np.abs(mean - ref["mean"]) / np.maximum(1.0, np.abs(ref["mean"]))))
    return {"workload": "the headline workload, one solve at full size", "oracle_s": dt,
            "mean_knots_max_rel_err": err,
            "best_cost_rel_err": abs(info["best_cost"] - ref["best_cost"]) / abs(ref["best_cost"]),
            "best_index_equal": bool(info["best_index"] == ref["best_index"]
                                     and info["best_iter"] == ref["best_iter"]),
            "tolerance": 1e-3}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    from paper_2511_19204_gb300 import synth
    oracle.build()
    n = max(64, args.cpu_samples // 2)
    p = synth.scale_quadruped(n=n)
    cores = os.cpu_count() or 1
    for _ in range(max(args.warmup, 0)):
        oracle.solve_problem(p, nthreads=cores)
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        oracle.solve_problem(p, nthreads=cores, iter_base=3 * k)
        times.append(time.perf_counter() - t0)
    units = p.n * p.horizon * p.iters
    value = units * len(times) / sum(times)
    ms = 1e3 * sum(times) / len(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": f"{n} of 8192 samples per step (bounded CPU sample)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n} of 8192 samples, 3 iterations x 200 steps per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------
def single_instance(mppi, synth, torch, flops, p, reps=20, warmup=5, mapping=-1, spline=0, block=0, method=None,
                    peak=None):
    """One instance's solve timed on its stream (CUDA events, L2 flushed between solves),
    plus its rollout kernel's in-graph duration."""
    stream = torch.cuda.Stream()
    ctrl = mppi.Controller.from_problem(mppi.Model(p.model), p, stream=stream.cuda_stream, mapping=mapping,
                                        spline=spline, block=block)
    x = torch.tensor(p.state, dtype=torch.float64, device="cuda")
    out = torch.zeros(ctrl.E, dtype=torch.float32, device="cuda")
    w = torch.tensor(p.nominal.reshape(-1), dtype=torch.float32, device="cuda")
    if mapping == -1:
        # tune on the workload's own state: one solve uploads it first
        ctrl.solve_device(x.data_ptr(), out.data_ptr(), d_warm=w.data_ptr())
        ctrl.sync()
        ctrl.autotune()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        ctrl.solve_device(x.data_ptr(), out.data_ptr(), d_warm=w.data_ptr())
    torch.cuda.synchronize()
    ms, roll = [], []
    for _ in range(reps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctrl.solve_device(x.data_ptr(), out.data_ptr(), d_warm=w.data_ptr())
            e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    # the rollout launches' durations from a profiled copy of the graph (events inside it)
    ctrl.profile(True)
    for _ in range(3):
        ctrl.solve_device(x.data_ptr(), out.data_ptr(), d_warm=w.data_ptr())
    torch.cuda.synchronize()
    for _ in range(reps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
            ctrl.solve_device(x.data_ptr(), out.data_ptr(), d_warm=w.data_ptr())
        torch.cuda.synchronize()
        roll.extend(float(v) for v in ctrl.rollout_ms())
    ctrl.profile(False)
    host = []
    for _ in range(reps):
        t0 = time.perf_counter()
        ctrl.solve(p.state, warm=p.nominal)
        host.append(1e3 * (time.perf_counter() - t0))
    ms.sort()
    host.sort()
    units = p.n * p.horizon * p.iters
    info = ctrl.info()
    fl_kernel = flops.flops_per_step(p.model, mapping_chain=info["mapping"] == mppi.MPPI_MAP_CHAIN)
    counted = flops.method_flops_per_step(method) if method else None
    fl_step = counted[1] if counted else fl_kernel
    achieved = fl_step * p.n * p.horizon / (statistics.mean(roll) * 1e-3) / 1e12
    peak = peak or flops.fp32_peak_tflops()
    return {"samples": p.n, "horizon": p.horizon, "knots": p.nk, "iters": p.iters, "dt": p.dt,
            "mapping": mppi.MAPPING_NAMES.get(info["mapping"]), "block": info["block"],
            "rollout_steps_per_s": units / (statistics.mean(ms) * 1e-3),
            "solves_per_s": 1e3 / statistics.mean(ms),
            "device_latency_ms": {"p50": ms[len(ms) // 2], "p99": ms[min(len(ms) - 1, int(0.99 * len(ms)))]},
            "host_latency_ms": {"p50": host[len(host) // 2], "p99": host[min(len(host) - 1, int(0.99 * len(host)))]},
            "rollout_launch_ms": statistics.mean(roll),
            "rollout_tflops": achieved, "rollout_frac_fp32_peak": achieved / peak,
            "flops_per_step_sample": fl_step,
            "flops_basis": ("the FP64 oracle's non-trivial operations per step-sample" if counted
                            else "the kernel's own formulation"),
            "kernel_flops_per_step_sample": fl_kernel}


# the other single-instance configurations: name -> (problem, spline variant, workload key
# of the method's counted flops (flops.METHOD_FLOPS) or None for the kernel's own count)
CONFIGS = {
    "plain_quadruped_K32": (lambda S: S.plain_quadruped(), 0, "plain_quadruped"),
    "scale_quadruped_K1024": (lambda S: S.scale_quadruped(n=1024), 0, "scale_quadruped"),
    "scale_quadruped_K4096": (lambda S: S.scale_quadruped(n=4096), 0, "scale_quadruped"),
    "humanoid_K2048": (lambda S: S.humanoid_problem(), 0, "humanoid"),
    "paper_cost_walking_K8192": (lambda S: S.paper_walking(), 0, None),
    "scale_quadruped_K8192_natural_cubic_spline": (lambda S: S.scale_quadruped(), 1, None),
}


def other_configs(mppi, synth, torch, flops, peak):
    return {name: single_instance(mppi, synth, torch, flops, make(synth), spline=spline, method=key, peak=peak)
            for name, (make, spline, key) in CONFIGS.items()}


def run_one_config(args):
    import torch

    from paper_2511_19204_gb300 import build as B
    from paper_2511_19204_gb300 import flops, mppi, synth
    B.build()
    mppi.load()
    make, spline, key = CONFIGS[args.only_config]
    peak, _ = device_fp32_peak(torch, 0, flops)
    r = single_instance(mppi, synth, torch, flops, make(synth), reps=args.steps, warmup=args.warmup,
                        mapping=args.mapping, spline=spline, block=args.block, method=key, peak=peak)
    print(json.dumps({"config": args.only_config, **r}))
    return 0


def receding_extra(mppi, synth, torch, p, reps=20, warmup=3, delays=(1, 5, 20)):
    """The receding-horizon cycle of Sec. III-E on device buffers: predict the state after
    the compute delay from the resident warm start, shift the warm start by the delay,
    solve from the prediction. Timed on the controller's stream (CUDA events, L2 flushed
    before each timed cycle)."""
    stream = torch.cuda.Stream()
    ctrl = mppi.Controller.from_problem(mppi.Model(p.model), p, stream=stream.cuda_stream)
    ctrl.autotune()
    x = torch.tensor(p.state, dtype=torch.float64, device="cuda")
    xp = torch.zeros_like(x)
    out = torch.zeros(ctrl.E, dtype=torch.float32, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()

    def timed(fn):
        ms = []
        for i in range(warmup + reps):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
            e1.synchronize()
            if i >= warmup:
                ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    solve_ms = timed(lambda: ctrl.solve_device(x.data_ptr(), out.data_ptr()))
    res = {"workload": f"{p.n} samples, H {p.horizon}, {p.nk} knots, {p.iters} iterations, dt {p.dt}",
           "solve_ms": solve_ms, "delay_steps_at_solve_latency": int(solve_ms * 1e-3 / p.dt), "delays": {}}
    for d in delays:
        def cycle():
            ctrl.predict_state_device(x.data_ptr(), d, xp.data_ptr())
            ctrl.shift_warm_start(d)
            ctrl.solve_device(xp.data_ptr(), out.data_ptr())
        res["delays"][str(d)] = {
            "cycle_ms": timed(cycle),
            "predict_ms": timed(lambda: ctrl.predict_state_device(x.data_ptr(), d, xp.data_ptr())),
            "shift_ms": timed(lambda: ctrl.shift_warm_start(d))}
    ctrl.sync()
    res["kernels_per_cycle"] = 2 + ctrl.kernels_per_solve
    return res


def batched_extra(mppi, synth, torch, count=256, reps=5):
    """Batched uneven instances: one persistent graph-captured launch per solve of all
    instances vs the same instances as sequential plain launches (one CUDA graph each,
    all on one stream). Each instance: one MPPI iteration, its own model/K/H/knots/lambda."""
    probs = synth.batched_problems(count)
    models = {}
    stream = torch.cuda.Stream()
    ctrls = []
    for p in probs:
        if p.model.name not in models:
            models[p.model.name] = mppi.Model(p.model)
        ctrls.append(mppi.Controller.from_problem(models[p.model.name], p, stream=stream.cuda_stream))
    units = sum(p.n * p.horizon * p.iters for p in probs)
    states = [p.state for p in probs]
    warms = [p.nominal for p in probs]
    # batched (host buffers in and out, packed into one H2D and one D2H inside the graph)
    for _ in range(2):
        mppi.solve_batch(ctrls, states, warms)
    tb = []
    for _ in range(reps):
        t0 = time.perf_counter()
        mppi.solve_batch(ctrls, states, warms)
        tb.append(time.perf_counter() - t0)
    # sequential plain launches, device-resident inputs, completion time of each instance
    xs = [torch.tensor(p.state, dtype=torch.float64, device="cuda") for p in probs]
    ws = [torch.tensor(p.nominal.reshape(-1), dtype=torch.float32, device="cuda") for p in probs]
    outs = [torch.zeros(c.E, dtype=torch.float32, device="cuda") for c in ctrls]
    for _ in range(2):
        for c, x, w, o in zip(ctrls, xs, ws, outs):
            c.solve_device(x.data_ptr(), o.data_ptr(), d_warm=w.data_ptr())
    torch.cuda.synchronize()
    tp, done_ms = [], []
    for _ in range(reps):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(count + 1)]
        with torch.cuda.stream(stream):
            evs[0].record(stream)
            for i, (c, x, w, o) in enumerate(zip(ctrls, xs, ws, outs)):
                c.solve_device(x.data_ptr(), o.data_ptr(), d_warm=w.data_ptr())
                evs[i + 1].record(stream)
        evs[-1].synchronize()
        tp.append(evs[0].elapsed_time(evs[-1]) / 1e3)
        done_ms = [evs[0].elapsed_time(e) for e in evs[1:]]
    tb_s, tp_s = statistics.median(tb), statistics.median(tp)
    done_ms.sort()
    q = lambda v, f: v[min(len(v) - 1, int(f * len(v)))]
    return {"workload": f"{count} uneven instances (70% quadruped / 30% humanoid, K log-uniform 64-2048, "
                        f"H 50-200, 4-8 knots, lambda U(0.05,0.5), 1 iteration), seeds 1000+i",
            "step_samples_per_batch": units,
            "batched": {"launch": "one persistent kernel walking a device work queue, graph-captured "
                                  "with packed H2D/D2H (host buffers, wall clock)",
                        "ms": 1e3 * tb_s, "solves_per_s": count / tb_s, "rollout_steps_per_s": units / tb_s,
                        "latency_ms_p50": 1e3 * tb_s, "latency_ms_p99": 1e3 * max(tb)},
            "plain_sequential": {"launch": f"{count} mppi_solve_device graphs back to back on one stream "
                                           "(device-resident inputs, CUDA events)",
                                 "ms": 1e3 * tp_s, "solves_per_s": count / tp_s, "rollout_steps_per_s": units / tp_s,
                                 "instance_done_ms_p50": q(done_ms, 0.5), "instance_done_ms_p99": q(done_ms, 0.99)},
            "speedup": tp_s / tb_s}


def _serving_controllers(mppi, synth, n_ctrl, seed=7):
    """The serving workload's controllers: 70 % quadruped / 30 % humanoid, K log-uniform
    256..2048, H 100..200, 4..8 knots, lambda U(0.05, 0.5), 1 iteration, dt 0.005."""
    import math

    import numpy as np
    rng = np.random.default_rng(seed)
    quad, hum = synth.quadruped(), synth.humanoid()
    mods = {"quadruped": mppi.Model(quad), "humanoid": mppi.Model(hum)}
    ctrls, states, work = [], [], []
    for i in range(n_ctrl):
        rob = quad if rng.random() < 0.7 else hum
        n = int(math.floor(math.exp(rng.uniform(math.log(256), math.log(2048)))))
        h = int(rng.integers(100, 201))
        nk = int(rng.integers(4, 9))
        c = mppi.Controller(mods[rob.name], n, h, nk, float(rng.uniform(0.05, 0.5)), synth.linear_sigma(nk),
                            dt=0.005, seed=7000 + i, instance=i)
        ctrls.append(c)
        states.append(synth.standing_state(rob, jitter=0.02, seed=7000 + i))
        work.append(n * h)
    return ctrls, states, work, rng


def _quantiles(lat, prefix="latency_ms"):
    lat = sorted(lat)
    q = lambda f: lat[min(len(lat) - 1, int(f * len(lat)))] if lat else None
    return {f"{prefix}_p50": q(0.5), f"{prefix}_p99": q(0.99), f"{prefix}_p999": q(0.999)}


def _plain_under_load(ctrls, states, work, rate_per_ctrl, seconds, warm_s, rng):
    """The plain single-instance path under the same Poisson arrivals: one host thread
    solves the requests first come, first served, each by a synchronous mppi_solve on its
    controller; a controller's newer state replaces its request still waiting in the queue
    (superseded). Latency = completion - arrival of the requests arriving in the window."""
    import heapq
    n_ctrl = len(ctrls)
    now0 = time.monotonic_ns()
    heap = [(now0 + int(rng.exponential(1e9 / rate_per_ctrl)), i) for i in range(n_ctrl)]
    heapq.heapify(heap)
    t_meas, t_end = now0 + int(warm_s * 1e9), now0 + int((warm_s + seconds) * 1e9)
    lat, done, units, superseded = [], 0, 0, 0
    queue = []                  # (arrival, controller), first come first served
    queued = {}                 # controller -> its queued arrival (at most one: the latest state)
    while True:
        now = time.monotonic_ns()
        while heap and heap[0][0] <= now and now < t_end:
            t_arr, i = heapq.heappop(heap)
            heapq.heappush(heap, (t_arr + int(rng.exponential(1e9 / rate_per_ctrl)), i))
            if i in queued:     # the newer state replaces the queued one
                superseded += t_meas <= t_arr
                queue.remove((queued[i], i))
            queued[i] = t_arr
            queue.append((t_arr, i))
        if now >= t_end:
            break
        if not queue:
            continue
        t_arr, i = queue.pop(0)
        del queued[i]
        ctrls[i].solve(states[i])
        t_done = time.monotonic_ns()
        if t_meas <= t_arr:
            lat.append((t_done - t_arr) / 1e6)
        if t_meas <= t_done < t_end:
            done += 1
            units += work[i]
    out = {"completed_req_per_s": done / seconds, "superseded_req_per_s": superseded / seconds,
           "rollout_steps_per_s": units / seconds, **_quantiles(lat)}
    out["saturated"] = done / seconds < 0.95 * rate_per_ctrl * n_ctrl
    return out


def serving_extra(mppi, synth, loads=(5000, 15000, 25000), seconds=30.0, warm_s=5.0, n_ctrl=512,
                  deadline_ms=20.0, plain_seconds=10.0, plain_warm_s=2.0):
    """Continuous-batching server under Poisson load: 512 closed-loop controllers (70 %
    quadruped, K log-uniform 256-2048, H 100-200, 4-8 knots), each request = current
    state + resident warm start; a controller's next request waits for its previous
    result, and a newer state replaces one still waiting (superseded: a controller acts on
    its latest state). Requests still waiting for admission after the deadline (one 50 Hz
    control period) are shed. Latency = server completion time - arrival time (CLOCK_MONOTONIC)
    of the served requests arriving in the measurement window (it includes a request's wait
    behind its controller's previous one and any lateness of this Python generator);
    submit_to_result = server completion - host submit of the same requests; throughput =
    completions inside the window. Beside it, the plain single-instance path (synchronous mppi_solve, first
    come first served) under the same arrivals."""
    import heapq

    import numpy as np
    ctrls, states, work, rng = _serving_controllers(mppi, synth, n_ctrl)
    # plain single-instance launches back to back: capacity of the unbatched path
    t0 = time.perf_counter()
    done = 0
    for i in range(0, n_ctrl, 4):
        ctrls[i].solve(states[i])
        done += 1
    plain_solves_per_s = done / (time.perf_counter() - t0)
    srv = mppi.Server(mem_budget_bytes=8 << 30, max_inflight=4)
    srv.set_deadline(int(deadline_ms * 1000))
    out = {"workload": f"{n_ctrl} controllers, Poisson arrivals, 70% quadruped / 30% humanoid, K 256-2048, "
                       f"H 100-200, 4-8 knots, 1 iteration; {seconds:.0f} s per load after {warm_s:.0f} s warm-up",
           "memory_budget_bytes": 8 << 30, "max_inflight_launches": 4, "deadline_ms": deadline_ms,
           "plain_single_instance_solves_per_s": plain_solves_per_s, "loads": []}
    import gc
    for load in loads:
        rate = load / n_ctrl
        # the load generator is Python: its garbage collector is paused during each load,
        # so that a collection pause (tens of ms) is not charged to the server's latency
        gc.collect()
        gc.disable()
        now0 = time.monotonic_ns()
        heap = [(now0 + int(rng.exponential(1e9 / rate)), i) for i in range(n_ctrl)]
        heapq.heapify(heap)
        busy = [None] * n_ctrl          # outstanding ticket
        backlog = [None] * n_ctrl       # the latest arrival waiting for the controller's running request
        owner, arrival = {}, {}
        lat, lat_sub, units, done_in_window, shed_in_window, arrived, superseded = [], [], 0, 0, 0, 0, 0
        t_end = now0 + int((seconds + warm_s) * 1e9)
        t_meas = now0 + int(warm_s * 1e9)
        s0 = srv.stats()

        def submit(i, t_arr):
            x = states[i].copy()
            x[7:7 + ctrls[i].nj] += rng.normal(scale=0.002, size=ctrls[i].nj)
            t = srv.submit(ctrls[i], x)
            busy[i] = t
            owner[t] = i
            arrival[t] = t_arr

        window_open = False
        while True:
            now = time.monotonic_ns()
            if now >= t_end and not owner:
                break
            if not window_open and now >= t_meas:
                srv.reset_timing()       # the worker maxima below are the window's
                window_open = True
            while heap and heap[0][0] <= now and now < t_end:
                t_arr, i = heapq.heappop(heap)
                heapq.heappush(heap, (t_arr + int(rng.exponential(1e9 / rate)), i))
                if t_arr >= t_meas:
                    arrived += 1
                if busy[i] is None:
                    submit(i, t_arr)
                else:
                    if backlog[i] is not None and backlog[i] >= t_meas:
                        superseded += 1          # the newer state replaces the waiting one
                    backlog[i] = t_arr
            nc = srv.next_completed(timeout_us=200)
            while nc is not None:
                t, t_sub, t_done = nc
                i = owner.pop(t)
                t_arr = arrival.pop(t)
                st = srv.poll(t, ctrls[i], timeout_us=0)[0]
                busy[i] = None
                if st == mppi.MPPI_OK:
                    if t_arr >= t_meas and t_arr < t_end:
                        lat.append((t_done - t_arr) / 1e6)
                        lat_sub.append((t_done - t_sub) / 1e6)
                    if t_meas <= t_done < t_end:
                        done_in_window += 1
                        units += work[i]
                elif t_meas <= t_done < t_end:
                    shed_in_window += 1
                if backlog[i] is not None and time.monotonic_ns() < t_end:
                    submit(i, backlog[i])
                backlog[i] = None
                nc = srv.next_completed(timeout_us=0)
        gc.enable()
        s1 = srv.stats()
        launches = s1["launches"] - s0["launches"]
        completed = s1["completed"] - s0["completed"] - (s1["shed"] - s0["shed"])
        entry = {"offered_req_per_s": load, "arrived_req_per_s": arrived / seconds,
                 "completed_req_per_s": done_in_window / seconds, "shed_req_per_s": shed_in_window / seconds,
                 "superseded_req_per_s": superseded / seconds,
                 "saturated": done_in_window / seconds < 0.95 * load,
                 "rollout_steps_per_s": units / seconds, **_quantiles(lat),
                 **_quantiles(lat_sub, "submit_to_result_ms"),
                 "mean_requests_per_launch": completed / max(launches, 1),
                 # the server thread's longest host-side pauses inside the measurement window
                 "server_max_worker_pass_ms": s1["max_worker_pass_ns"] / 1e6,
                 "server_max_launch_call_ms": s1["max_launch_ns"] / 1e6,
                 "server_max_unpack_ms": s1["max_unpack_ns"] / 1e6}
        gc.collect()
        entry["plain_launch"] = _plain_under_load(ctrls, states, work, rate, plain_seconds, plain_warm_s, rng)
        entry["plain_launch"]["window_s"] = plain_seconds
        out["loads"].append(entry)
    srv.close()
    out["capacity_req_per_s"] = max(e["completed_req_per_s"] for e in out["loads"])
    return out


def run_ours(args, rank, world, local):
    import numpy as np
    import torch

    from paper_2511_19204_gb300 import build as B
    from paper_2511_19204_gb300 import flops, mppi, synth

    torch.cuda.set_device(local)
    dist = dist_init(world)
    B.build()
    mppi.load()
    p = synth.scale_quadruped(n=args.samples, seed_state=20 + rank)
    p.instance = rank
    stream = torch.cuda.Stream()
    model = mppi.Model(p.model)
    ctrl = mppi.Controller.from_problem(model, p, mapping=args.mapping, block=args.block,
                                        stream=stream.cuda_stream)
    tuned = None
    if args.mapping == -1:
        try:
            # tune on the workload's own state: one solve uploads it first
            ctrl.solve(p.state)
            m, b, ms = ctrl.autotune()
            tuned = {"mapping": mppi.MAPPING_NAMES.get(m, m), "block": b,
                     "ms_per_rollout": {mppi.MAPPING_NAMES[k]: [round(float(v), 4) if v > 0 else None for v in ms[k]]
                                        for k in range(4)}}
        except mppi.MppiError:
            tuned = None
    info = ctrl.info()
    nx, E = p.model.nx, ctrl.E
    x = torch.tensor(p.state, dtype=torch.float64, device="cuda")
    mean = torch.zeros(E, dtype=torch.float32, device="cuda")
    best = torch.zeros(E, dtype=torch.float32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    # clocks sampled from the warm-up on (the timed region alone can be shorter than the
    # sampling period); the samples are those of the loaded device
    clocks = Clocks(local)
    clocks.start()
    for _ in range(max(args.warmup, 3)):
        ctrl.solve_device(x.data_ptr(), mean.data_ptr(), best.data_ptr())
    torch.cuda.synchronize()
    per_solve_ms, rollout_ms = [], []
    barrier(dist)
    torch.cuda.synchronize()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)                                   # L2 flush (not timed)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            ctrl.solve_device(x.data_ptr(), mean.data_ptr(), best.data_ptr())
            ev1.record(stream)
        ev1.synchronize()
        per_solve_ms.append(ev0.elapsed_time(ev1))
    torch.cuda.synchronize()
    barrier(dist)
    t_local = sum(per_solve_ms) / 1e3
    # the rollout launches' own durations: the same solves with CUDA events around each
    # kernel inside the graph (a separate graph, so the timed solves above carry no events)
    ctrl.profile(True)
    for _ in range(3):
        ctrl.solve_device(x.data_ptr(), mean.data_ptr(), best.data_ptr())
    torch.cuda.synchronize()
    for _ in range(max(3, min(args.steps, 20))):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
            ctrl.solve_device(x.data_ptr(), mean.data_ptr(), best.data_ptr())
        torch.cuda.synchronize()
        rollout_ms.extend(float(v) for v in ctrl.rollout_ms())
    ctrl.profile(False)
    units = p.n * p.horizon * p.iters
    t_max, units_all = reduce_max_sum(dist, t_local, units * args.steps)
    value = units_all / t_max
    # end to end through the C ABI with host buffers (H2D state, graph, D2H results, sync)
    xs = p.state.copy()
    e2e_t = []
    for k in range(args.e2e_steps + 2):
        t0 = time.perf_counter()
        ctrl.solve(xs)
        if k >= 2:
            e2e_t.append(time.perf_counter() - t0)
    e2e_local = sum(e2e_t)
    clk = clocks.stop()
    if clk:
        clk["window"] = "warm-up, timed and end-to-end solves (the timed region alone is shorter than the sampling period)"
    e2e_max, e2e_units = reduce_max_sum(dist, e2e_local, units * len(e2e_t))
    if rank != 0:
        return 0
    # roofline of the dominant kernel (the rollout): FP32 ALU bound. The numerator is the
    # method's work per step-sample (the oracle's non-trivial operations, counted); the
    # kernel's own formulation does slightly less and is reported beside it
    fl_kernel = flops.flops_per_step(p.model, mapping_chain=info["mapping"] == mppi.MPPI_MAP_CHAIN)
    fl_step = flops.method_flops_per_step("scale_quadruped")[1]
    roll_ms = statistics.mean(rollout_ms)
    achieved = fl_step * p.n * p.horizon / (roll_ms * 1e-3) / 1e12
    peak, peak_basis = device_fp32_peak(torch, local, flops)
    lat = sorted(per_solve_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "samples": p.n, "knots": p.nk, "horizon": p.horizon,
                   "iters": p.iters, "dt": p.dt, "lambda": p.lam,
                   "mapping": mppi.MAPPING_NAMES.get(info["mapping"], info["mapping"]), "block": info["block"],
                   "autotune": tuned, "l2": "flushed between timed solves (256 MiB write, untimed)",
                   "parallelism": f"replicas x{world}"},
        "solves_per_s": args.steps * world / t_max,
        "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                       "mean": statistics.mean(lat)},
        "e2e": ({"value": e2e_units / e2e_max, "unit": UNIT,
                 "h2d_bytes_per_step": ctrl.io_bytes()[0], "d2h_bytes_per_step": ctrl.io_bytes()[1],
                 "ms_per_step": 1e3 * e2e_local / len(e2e_t)} if e2e_t else None),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "traffic": (profiled_traffic("rollout_lanes_quadruped", p.n)
                                 if info["mapping"] == mppi.MPPI_MAP_CHAIN else None),
                     "fp32_pipe_util_ncu": (profiled_fma_pipe("rollout_lanes_quadruped")
                                            if info["mapping"] == mppi.MPPI_MAP_CHAIN else None),
                     "kernel": "rollout", "launch_ms": roll_ms,
                     "flops_per_step_sample": fl_step,
                     "flops_basis": ("the FP64 oracle's non-trivial operations per step-sample on this workload "
                                     "(counted by its operation-counting build; dense count "
                                     f"{flops.method_flops_per_step('scale_quadruped')[0]:.0f})"),
                     "kernel_flops_per_step_sample": fl_kernel,
                     "frac_at_kernel_count": fl_kernel * p.n * p.horizon / (roll_ms * 1e-3) / 1e12 / peak,
                     "peak_basis": peak_basis},
        "gpu_launches": args.steps * ctrl.kernels_per_solve,
        "clocks": clk,
    }
    if not args.no_configs:
        try:
            line["other_configs"] = other_configs(mppi, synth, torch, flops, peak)
        except Exception as exc:  # reported, never silently dropped
            line["other_configs"] = {"error": repr(exc)}
    if not args.no_receding:
        try:
            line["receding_horizon"] = receding_extra(mppi, synth, torch, p)
        except Exception as exc:  # reported, never silently dropped
            line["receding_horizon"] = {"error": repr(exc)}
    if not args.no_batched:
        try:
            line["batched_uneven"] = batched_extra(mppi, synth, torch)
        except Exception as exc:  # reported, never silently dropped
            line["batched_uneven"] = {"error": repr(exc)}
    if not args.no_serving:
        try:
            line["serving"] = serving_extra(mppi, synth)
        except Exception as exc:  # reported, never silently dropped
            line["serving"] = {"error": repr(exc)}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_samples)
        try:
            line["oracle_parity"] = oracle_parity(mppi, synth, info["mapping"], info["block"])
        except Exception as exc:  # reported, never silently dropped
            line["oracle_parity"] = {"error": repr(exc)}
    print(json.dumps(line), flush=True)
    del np
    return 0


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.only_config:
        return run_one_config(args)
    return run_ours(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
