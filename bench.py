"""Benchmark: batched evaluation of the 20,000-op random straight-line program.

Workload (one step = one evaluation of the whole batch): the seeded random
program (64 inputs, 32 outputs, 20,000 generated ops with the stated op mix,
program seed 0) on N = 65,536 instances with N(0, 1) inputs (seed 1 + rank).
The FP64 kernel is the headline; the FP32 kernel is reported beside it with
its error against the FP64 kernel on the same FP32-rounded inputs.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun each rank evaluates its own
65,536 instances (weak scaling, no collective on the data path).
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
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("instance-evals/s & Gop/s vs FP32/FP64 peak at N=65536; adjoint/forward time ratio")
N_INST = 65536
N_OPS_GEN = 20000
PROGRAM_SEED, INPUT_SEED = 0, 1
L2_FLUSH_BYTES = 256 << 20
# ALU peaks derived from unit counts and clocks (GB300: 152 SMs, 2070 MHz max SM
# clock): FP64 1.25 TFLOP/s = 0.625 TFMA/s (about 2 FMA per clock per SM); FP32
# 128 FMA per clock per SM = 40.3 TFMA/s.  The measured FMA-chain rates of
# peaks.py are reported beside them.
NOMINAL_FMA_PER_S = {"f64": 1.25e12 / 2, "f32": 152 * 128 * 2.07e9}
# DRAM bytes (read + write) per launch that an ncu capture measured for the
# generated kernel with this source hash; a kernel whose source changed since
# the capture gets no traffic figure (null) rather than a stale one
NCU_TRAFFIC = {"7f243409b56b79cf": 26300672 + 10496}   # 4 warps per 32 instances, 2 groups per CTA


def workload_config(info=None):
    c = {"workload": "random straight-line program: 20000 generated ops, 64 inputs, 32 outputs, "
                     "op mix 30% add/sub, 30% mul, 5% div, 10% sin/cos, 10% exp(-x^2), "
                     "5% sqrt(1+x^2), 10% fma-const; N=65536 instances",
         "N": N_INST, "ops_generated": N_OPS_GEN, "program_seed": PROGRAM_SEED,
         "input_seed": INPUT_SEED, "inputs": "N(0,1), synthetic",
         "l2": "flushed between timed steps (256 MB write, outside the events)"}
    if info is not None:
        c["ops_ir"] = int(info.n_ops_ir)
        c["ops_live"] = int(info.n_ops)
    return c


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.f is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.f.seek(0)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
def cpu_oracle_baseline(ir: bytes, x: np.ndarray, sample: int):
    from oracle import Oracle
    orc = Oracle(ir)
    xs = np.ascontiguousarray(x[:, :sample])
    cores = os.cpu_count() or 1
    orc.eval(xs[:, :256], threads=cores)   # warm-up
    t = time.perf_counter()
    y = orc.eval(xs, threads=cores)
    dt = time.perf_counter() - t
    s1 = min(sample, 4096)                  # one core, on a smaller sample
    t = time.perf_counter()
    orc.eval(xs[:, :s1], threads=1)
    dt1 = time.perf_counter() - t
    return {"value": sample / dt, "unit": "instance-evals/s", "cores": cores, "kind": "oracle",
            "sample": f"{sample} of the {N_INST} instances, FP64 interpreter, {cores} threads, "
                      f"{dt:.2f} s wall",
            "single_core": {"value": s1 / dt1, "unit": "instance-evals/s",
                            "sample": f"{s1} instances, 1 thread, {dt1:.2f} s wall"}}, y


def _events_ms(fn, reps, flush):
    """Median device time of fn() over reps calls (CUDA events on the current stream)."""
    import torch
    ts = []
    for _ in range(reps):
        flush.zero_()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        fn()
        e.record()
        e.synchronize()
        ts.append(s.elapsed_time(e))
    return statistics.median(ts)


def batch_oracle_check(irs, sizes, xs, outs, sample=64):
    """CPU-baseline leg of the uneven batch: the FP64 oracle on `sample` sampled
    instances (plus the last one) of every program, all host cores; its outputs
    double as the per-output error record of the FP32 batch."""
    from oracle import Oracle, tolerance
    cores = os.cpu_count() or 1
    per, op_inst, t_cpu = [], 0, 0.0
    for j, (n, N) in enumerate(sizes):
        idx = np.unique(np.r_[np.random.default_rng(j).choice(N, sample, replace=False), N - 1])
        x = xs[j][:, idx].double().cpu().numpy()
        got = outs[j][:, idx].double().cpu().numpy()
        orc = Oracle(irs[j])
        t0 = time.perf_counter()
        ref = orc.eval(x, threads=cores)
        t_cpu += time.perf_counter() - t0
        op_inst += n * len(idx)
        s = np.max(np.abs(ref), axis=1, keepdims=True)
        rel = np.abs(got - ref) / s
        tol = tolerance(orc, x, ref, 2e-4, kind=1, mca_runs=8)
        per.append({"ops_generated": n, "instances_checked": int(len(idx)),
                    "max_rel_scaled": float(rel.max()), "median_rel_scaled": float(np.median(rel)),
                    "frac_within_2e-4": float(np.mean(rel <= 2e-4)),
                    "frac_within_rule": float(np.mean(np.abs(got - ref) <= tol))})
    return {"rule": "per output row k: |y32 - y64_oracle| <= max(2e-4 s_k, 2 B32, 4 S_k); B32 the "
                    "first-order rounding bound, S_k the largest deviation of 8 Monte Carlo "
                    "arithmetic runs at FP32 sizes; rel = |y32 - y64| / s_k",
            "programs": per}, {
        "value": op_inst / t_cpu, "unit": "generated op-instances/s", "cores": cores,
        "kind": "oracle",
        "sample": f"{sample} instances (+ the last) of each program, FP64 interpreter, {cores} threads"}


def other_configs(dev, pk64, pk32, flush, reps, oracle_check=True):
    """Live measurements of the other workloads (cart-pole, MPC, rollout, batch)."""
    import torch
    from concurrent.futures import ThreadPoolExecutor

    from paper_2408_09662_gb300 import inputs, peaks, programs
    from paper_2408_09662_gb300.api import Batch, Function
    from paper_2408_09662_gb300.rollout import GraphRollout, StepProgram, rollout

    out = {"fractions": "of the measured FMA-chain rates (peaks.py); the derived nominal peaks "
                        "are 0.625 (FP64) and 40.3 (FP32) TFMA/s"}

    def frac(fn, N, ms, dt):
        return peaks.roofline_seconds(fn, pk64, pk32) * N / (ms * 1e-3)

    # every program is compiled up front, concurrently (ctypes drops the GIL)
    t_all = time.perf_counter()
    sizes = [(1000, 65536), (5000, 32768), (10000, 32768), (20000, 16384), (50000, 8192),
             (100000, 4096), (150000, 2048), (200000, 512)]

    def make_batch():
        t0 = time.perf_counter()
        irs = [programs.random_program(n, seed=100 + j).to_bytes() for j, (n, _) in enumerate(sizes)]
        # ways=4: programs with few instances and many ops (here the 50k-200k-op
        # ones) run as satellite kernels, 4 warps per group of 32 instances,
        # beside the persistent kernel of the others (4 measured faster than 8
        # and 16 for this batch and for each of those programs alone)
        return Batch(irs, [N for _, N in sizes], dtype="f32", ways=4), time.perf_counter() - t0, irs
    ir3 = programs.quadrotor_mpc().to_bytes()
    ir1 = programs.quadrotor_lqr_step().to_bytes()
    srb = programs.srb_step().to_bytes()
    pool = ThreadPoolExecutor(8)
    ir_c1 = programs.cartpole_rk4().to_bytes()
    fut = {"c1": pool.submit(Function, ir_c1, dtype="f64"),
           "c1w4": pool.submit(Function, ir_c1, dtype="f64", ways=4),
           "lqr8": pool.submit(Function, ir1, dtype="f64", ways=8),
           "batch": pool.submit(make_batch),
           "lqr0": pool.submit(Function, ir1, dtype="f64"),
           "c3f64": pool.submit(Function, ir3, dtype="f64"),
           "c3mixed": pool.submit(Function, ir3, dtype="mixed"),
           "srbf64": pool.submit(Function, srb, dtype="f64", adjoint=1),
           "srbf64w8": pool.submit(Function, srb, dtype="f64", adjoint=1, ways=8),
           "srbf32": pool.submit(Function, srb, dtype="f32", adjoint=1)}
    pool.shutdown(wait=True)   # nothing is timed while host threads compile
    fut = {k: f.result() for k, f in fut.items()}
    out["compile_wall_seconds"] = time.perf_counter() - t_all

    # --- C1 cart-pole RK4 + Jacobian, FP64 ---
    c1 = fut["c1"]
    rec = {"ops_live": int(c1.info.n_ops)}
    for N in (4096, 65536):
        x = torch.tensor(inputs.cartpole(N, seed=0), device=dev)
        y = c1(x)
        ms = _events_ms(lambda: c1(x, out=y), reps, flush)
        rec[f"N{N}"] = {"ms": ms, "instance_evals_per_s": N / (ms * 1e-3),
                        "frac_of_measured_fma_f64": frac(c1, N, ms, "f64")}
    # N = 4096 leaves most SMs with one warp: 4 warps per 32 instances (cooperative)
    c1w = fut["c1w4"]
    x = torch.tensor(inputs.cartpole(4096, seed=0), device=dev)
    y = c1w(x)
    ms = _events_ms(lambda: c1w(x, out=y), reps, flush)
    rec["N4096_ways4"] = {"ms": ms, "instance_evals_per_s": 4096 / (ms * 1e-3),
                          "frac_of_measured_fma_f64": frac(c1w, 4096, ms, "f64")}
    # the autotuner's launch at both batch sizes (a short program: its candidates compile in
    # well under a second each)
    from paper_2408_09662_gb300.tune import autotune
    for N in (4096, 65536):
        x = torch.tensor(inputs.cartpole(N, seed=0), device=dev)
        fa = autotune(ir_c1, x, "f64", use_cache=False)
        y = fa(x)
        ms = _events_ms(lambda: fa(x, out=y), reps, flush)
        rec[f"N{N}_tuned"] = {"launch": fa.tune_record["options"], "ms": ms,
                              "instance_evals_per_s": N / (ms * 1e-3),
                              "frac_of_measured_fma_f64": frac(fa, N, ms, "f64")}
    out["cartpole_rk4_jacobian_f64"] = rec

    # --- C3 closed-form MPC, N = 16384, all-FP64 vs mixed (FP32 bulk, FP64 pivots) ---
    f3 = {"f64": fut["c3f64"], "mixed": fut["c3mixed"]}
    N = 16384
    rng = np.random.default_rng(0)
    X = np.vstack([rng.uniform(-0.5, 0.5, (6, N)), rng.uniform(-1, 1, (2, N))])
    rec = {"ops_live": int(f3["f64"].info.n_ops), "N": N, "kernels": int(f3["f64"].info.n_segments)}
    ys = {}
    for dt, fn in f3.items():
        Xd = X if dt == "f64" else X.astype(np.float32).astype(np.float64)
        x = torch.tensor(Xd, dtype=fn.torch_dtype, device=dev)
        y = fn(x)
        ms = _events_ms(lambda: fn(x, out=y), reps, flush)
        ys[dt] = (y.double().cpu().numpy(), Xd)
        rec[dt] = {"ms": ms, "instance_evals_per_s": N / (ms * 1e-3),
                   "frac_of_measured_fma": frac(fn, N, ms, dt)}
    # the mixed kernel's inputs are rounded to FP32; compare with the FP64 kernel on those inputs
    y64r = f3["f64"](torch.tensor(ys["mixed"][1], device=dev)).cpu().numpy()
    rec["mixed"]["max_rel_diff_vs_fp64_kernel"] = float(
        np.max(np.abs(ys["mixed"][0] - y64r) / np.max(np.abs(y64r), axis=1, keepdims=True)))
    rec["mixed_speedup_vs_f64"] = rec["f64"]["ms"] / rec["mixed"]["ms"]
    out["quadrotor_mpc"] = rec

    # --- C4 differentiable rollout: 50 RK4 steps, N = 4096, forward and reverse ---
    rec = {"N": 4096, "steps": 50, "checkpoint_every": 10}
    rng = np.random.default_rng(0)
    x0n, Kn = rng.uniform(-0.1, 0.1, (12, 4096)), rng.normal(0, 0.1, (12, 12))
    for dt in ("f64", "f32"):
        prog = StepProgram(fut["srb" + dt], 144, 12)
        tdt = prog.fn.torch_dtype
        x0 = torch.tensor(x0n, dtype=tdt, device=dev, requires_grad=True)
        K = torch.tensor(Kn.reshape(144), dtype=tdt, device=dev, requires_grad=True)
        L, _ = rollout(prog, x0, K, 50)
        L.backward()
        torch.cuda.synchronize()
        fwd = _events_ms(lambda: rollout(prog, x0.detach(), K.detach(), 50), reps, flush)

        def fb():
            L, _ = rollout(prog, x0, K, 50)
            L.backward()
        both = _events_ms(fb, reps, flush)
        # the same two passes replayed from CUDA graphs (one host launch per pass)
        gr = GraphRollout(prog, 4096, 50, 10, device=dev)
        gfwd = _events_ms(lambda: gr.forward(x0.detach(), K.detach()), reps, flush)

        def gfb():
            gr.forward(x0.detach(), K.detach())
            gr.backward()
        gboth = _events_ms(gfb, reps, flush)
        rec[dt] = {"forward_ms": fwd, "backward_ms": both - fwd,
                   "adjoint_forward_ratio": (both - fwd) / fwd,
                   "graph_forward_ms": gfwd, "graph_backward_ms": gboth - gfwd,
                   "graph_adjoint_forward_ratio": (gboth - gfwd) / gfwd,
                   "step_ops": int(prog.fn.info.n_ops),
                   "adjoint_ops": int(sum(prog.fn.op_counts(adjoint=True)))}
        # the step's forward and adjoint kernels alone at N = 65,536 (roofline points)
        fn, Nk = prog.fn, 65536
        rk = np.random.default_rng(1)
        Xk = np.vstack([np.tile(Kn.reshape(144, 1), (1, Nk)), rk.uniform(-0.1, 0.1, (12, Nk)),
                        np.zeros((1, Nk))])
        xk = torch.tensor(Xk, dtype=tdt, device=dev)
        yk = fn(xk)
        ybar = torch.ones_like(yk)
        xbar = fn.adjoint(xk, ybar, reduce_broadcast=True)
        ms_f = _events_ms(lambda: fn(xk, out=yk), reps, flush)
        ms_a = _events_ms(lambda: fn.adjoint(xk, ybar, out=xbar, reduce_broadcast=True), reps, flush)
        rec[dt]["kernels_N65536"] = {
            "forward_ms": ms_f, "adjoint_ms": ms_a, "adjoint_forward_ratio": ms_a / ms_f,
            "forward_frac_of_measured_fma": peaks.roofline_seconds(fn, pk64, pk32) * Nk / (ms_f * 1e-3),
            "adjoint_frac_of_measured_fma": peaks.roofline_seconds(fn, pk64, pk32, adjoint=True) * Nk / (ms_a * 1e-3)}
    # FP64 with 8 warps per 32 instances (cooperative forward and adjoint kernels)
    prog = StepProgram(fut["srbf64w8"], 144, 12)
    x0 = torch.tensor(x0n, device=dev, requires_grad=True)
    K = torch.tensor(Kn.reshape(144), device=dev, requires_grad=True)
    fwd = _events_ms(lambda: rollout(prog, x0.detach(), K.detach(), 50), reps, flush)

    def fbc():
        L, _ = rollout(prog, x0, K, 50)
        L.backward()
    both = _events_ms(fbc, reps, flush)
    rec["f64_ways8"] = {"forward_ms": fwd, "backward_ms": both - fwd,
                        "adjoint_forward_ratio": (both - fwd) / fwd}
    out["srb_rollout"] = rec

    # --- f1 LQR closed-loop step (SDA Riccati solve inside), N = 10,000, FP64 ---
    # one thread per instance leaves most SMs with two warps; W = 8 warps per
    # 32 instances (cooperative kernel) split each instance's program
    fl = {0: fut["lqr0"], 8: fut["lqr8"]}
    N = 10000
    rng = np.random.default_rng(0)
    X = np.vstack([rng.uniform(-0.5, 0.5, (6, N)), rng.uniform(10, 20, (1, N)),
                   rng.uniform(0.8, 1.2, (1, N)), rng.uniform(0.008, 0.012, (1, N)),
                   rng.uniform(0.5, 10, (6, N)), rng.uniform(0.05, 0.5, (1, N))])
    rec = {"ops_live": int(fl[0].info.n_ops), "N": N}
    ys = {}
    for w, fn in fl.items():
        x = torch.tensor(X, device=dev)
        y = fn(x)
        ms = _events_ms(lambda: fn(x, out=y), reps, flush)
        ys[w] = y.cpu().numpy()
        rec[f"ways{w}"] = {"ms": ms, "instance_evals_per_s": N / (ms * 1e-3),
                           "frac_of_measured_fma_f64": frac(fn, N, ms, "f64")}
    rec["coop_speedup"] = rec["ways0"]["ms"] / rec["ways8"]["ms"]
    rec["coop_max_rel_diff"] = float(np.max(np.abs(ys[8] - ys[0]) /
                                            np.max(np.abs(ys[0]), axis=1, keepdims=True)))
    out["quadrotor_lqr_step_f64"] = rec

    # --- C5 uneven batch: 8 random programs, one persistent graph launch vs 8 launches ---
    b, t_compile, batch_irs = fut["batch"]
    xs = [torch.tensor(inputs.normal(64, N, seed=200 + j), dtype=torch.float32, device=dev)
          for j, (_, N) in enumerate(sizes)]
    outs = [torch.empty((32, N), dtype=torch.float32, device=dev) for _, N in sizes]
    by_block = {}
    for blk in (32, 64, 128):
        b.set_block(blk)
        b(xs, outs, mode="persistent")
        by_block[blk] = _events_ms(lambda: b(xs, outs, mode="persistent"), reps, flush)
    block = min(by_block, key=by_block.get)
    b.set_block(block)
    ms_p = _events_ms(lambda: b(xs, outs, mode="persistent"), reps, flush)
    ms_s = _events_ms(lambda: b(xs, outs, mode="plain"), reps, flush)
    gen_ops = sum(n * N for n, N in sizes)
    fma_eq = sum(peaks.weighted_ops(b.op_counts(j), pk32["weights"]) * N for j, (_, N) in enumerate(sizes))
    ach = fma_eq / (ms_p * 1e-3)
    out["uneven_batch_f32"] = {
        "roofline": {"bound": "alu", "achieved": ach * 1e-12, "peak": NOMINAL_FMA_PER_S["f32"] * 1e-12,
                     "unit": "TFMA/s (FMA-equivalent ops of all 8 programs, FP32)",
                     "frac": ach / NOMINAL_FMA_PER_S["f32"],
                     "frac_of_measured": ach / pk32["fma_per_s"],
                     "work_fma_eq": fma_eq},
        "programs": [{"ops_generated": n, "N": N} for n, N in sizes],
        "op_instances_generated": gen_ops, "persistent_ms": ms_p, "plain_8_launches_ms": ms_s,
        "speedup_persistent_vs_plain": ms_s / ms_p, "tile_block": block,
        "persistent_ms_by_tile_block": {str(k): v for k, v in by_block.items()},
        "satellites": "ways=4: programs with N <= 8192 and >= 20,000 ops after the passes (here the "
                      "50k-, 100k-, 150k- and 200k-op ones) run as cooperative kernels of their own, "
                      "4 warps per group of 32 instances, on parallel graph branches beside the "
                      "persistent kernel of the other four; their plain launch runs the same kernels",
        **b.info(),
        "gop_per_s_generated": gen_ops / (ms_p * 1e-3) * 1e-9, "setup_seconds": t_compile}
    if oracle_check:
        b(xs, outs, mode="persistent")
        torch.cuda.synchronize()
        err, cpu = batch_oracle_check(batch_irs, sizes, xs, outs)
        out["uneven_batch_f32"]["err_vs_fp64_oracle"] = err
        out["uneven_batch_f32"]["cpu_baseline"] = cpu
    return out


def run_reference(args, rank, world):
    """The oracle as the reference arm, on this host's cores."""
    from oracle import Oracle
    from paper_2408_09662_gb300 import inputs, programs
    if rank != 0:
        return
    ir = programs.random_program(N_OPS_GEN, seed=PROGRAM_SEED).to_bytes()
    orc = Oracle(ir)
    sample = 8192
    x = inputs.normal(64, sample, seed=INPUT_SEED)
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        orc.eval(x[:, :512], threads=cores)
    t = time.perf_counter()
    for _ in range(args.steps):
        orc.eval(x, threads=cores)
    dt = time.perf_counter() - t
    value = sample * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "instance-evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(),
            "cpu_baseline": {"value": value, "unit": "instance-evals/s", "cores": cores,
                             "kind": "oracle",
                             "sample": f"each step evaluates {sample} of the {N_INST} instances"},
            "e2e": {"value": value, "unit": "instance-evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_experiment(name):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2408_09662_gb300 import experiments
    if name == "coop":
        experiments.coop_sweep()
    elif name == "mpc":
        experiments.mpc_pareto()
    elif name == "roa":
        experiments.lqr_roa()
    elif name == "batch":
        experiments.batch_sweep()
    elif name == "interp":
        experiments.interp_sweep()
    elif name == "spill":
        experiments.spill_sweep()
    elif name == "tune":
        experiments.tune_sweep()
    else:
        from oracle import Oracle
        cores = os.cpu_count() or 1
        cache = {}

        def cpu_ms(irb, X, n_ops):
            """The oracle on all host cores, timed on a bounded sample and scaled to N."""
            orc = cache.setdefault(irb, Oracle(irb))
            N = X.shape[1]
            sample = min(N, max(64, int(2e8 // max(n_ops, 1))))
            t0 = time.perf_counter()
            orc.eval(X[:, :sample], threads=cores)
            return (time.perf_counter() - t0) * 1e3 * N / sample, f"CPU oracle ms ({cores} cores)"
        experiments.ldlt_sweep(cpu_ms=cpu_ms)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-peaks", action="store_true",
                    help="reuse peaks measured earlier on this machine (_build/peaks.json)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the cart-pole / MPC / rollout / batch measurements")
    ap.add_argument("--only", choices=["both", "f64", "f32"], default="both",
                    help="time one kernel only (for profiling); prints no JSON line")
    ap.add_argument("--ways64", default="auto",
                    help="warps per 32 instances of the FP64 kernel: auto (faster of 0, 4), or a number")
    ap.add_argument("--ways32", default="auto",
                    help="warps per 32 instances of the FP32 kernel: auto (fastest of 0, 4, 8), or a number")
    ap.add_argument("--launch64", default=None,
                    help='fixed launch options of the FP64 kernel as JSON (e.g. \'{"ways": 4, '
                         '"coop_groups": 2}\'): no tuning')
    ap.add_argument("--launch32", default=None,
                    help="fixed launch options of the FP32 kernel as JSON: no tuning")
    ap.add_argument("--experiment", choices=["ldlt", "coop", "mpc", "roa", "batch", "interp", "spill", "tune"],
                    help="run one of the paper's experiments instead (markdown table, no JSON line); "
                         "ldlt adds the CPU oracle as its CPU baseline column")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    t_main = time.perf_counter()
    if args.experiment:
        run_experiment(args.experiment)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    from paper_2408_09662_gb300 import inputs, peaks, programs
    from paper_2408_09662_gb300.api import Function
    from paper_2408_09662_gb300.tune import autotune

    ir = programs.random_program(N_OPS_GEN, seed=PROGRAM_SEED).to_bytes()
    x_np = inputs.normal(64, N_INST, seed=INPUT_SEED + rank)
    x64 = torch.tensor(x_np, dtype=torch.float64, device=dev)
    x32 = x64.float()
    # launch configuration: the autotuner times one thread per instance (ways 0)
    # against W warps sharing each group of 32 instances, then refines the
    # faster shape (instances per thread, register caps, groups per CTA); every
    # candidate runs this batch.  FP64 with 2 warps per group measured 10.36 ms
    # on one box and 11.0-11.1 ms on others, so only the steady shapes compete.
    cand = {"f64": (0, 4) if args.ways64 == "auto" else (int(args.ways64),),
            "f32": (0, 4, 8) if args.ways32 == "auto" else (int(args.ways32),)}
    def launch(dt, fixed, x):
        if fixed is not None:
            opts = json.loads(fixed)
            fn = Function(ir, dtype=dt, **opts)
            fn.tune_record = {"options": opts, "candidates": [], "fixed": True}
            return fn
        return autotune(ir, x, dt, ways=cand[dt], use_cache=False)
    t_tune = time.perf_counter()
    fn64 = launch("f64", args.launch64, x64)      # one after the other:
    fn32 = launch("f32", args.launch32, x32)      # nothing else on the GPU
    t_tune = time.perf_counter() - t_tune
    tuning = {dt: {"chosen": fn.tune_record["options"],
                   "candidates_ms": [[json.dumps(o, sort_keys=True), ms] for o, ms in fn.tune_record["candidates"]]}
              for dt, fn in (("f64", fn64), ("f32", fn32))}

    y64 = torch.empty((fn64.nnz_out, N_INST), dtype=torch.float64, device=dev)
    y32 = torch.empty((fn32.nnz_out, N_INST), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, x, y, steps):
        times = []
        for _ in range(steps):
            flush.zero_()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            fn(x, out=y)
            e.record(stream)
            times.append((s, e))
        return times

    for _ in range(args.warmup):
        fn64(x64, out=y64)
        fn32(x32, out=y32)
    torch.cuda.synchronize()
    if args.only != "both":
        fn, x, y = (fn64, x64, y64) if args.only == "f64" else (fn32, x32, y32)
        ev = timed(fn, x, y, args.steps)
        torch.cuda.synchronize()
        ms = sum(s.elapsed_time(e) for s, e in ev) / args.steps
        print(f"{args.only}: {ms:.4f} ms/step over {args.steps} steps", flush=True)
        return

    # ---- timed region: K FP64 steps ------------------------------------------
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        ev = timed(fn64, x64, y64, args.steps)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    step_ms = [s.elapsed_time(e) for s, e in ev]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    clocks = clk.summary()

    # ---- FP32 kernel, same protocol ----------------------------------------------
    with ClockSampler(torch.cuda.current_device()) as clk32:
        ev32 = timed(fn32, x32, y32, args.steps)
        torch.cuda.synchronize()
    ms32 = sum(s.elapsed_time(e) for s, e in ev32) / args.steps

    # ---- end to end through the C ABI's host-buffer call (cusadi_eval_host): ------
    # pinned host inputs copied in and outputs copied out inside the timed region,
    # in chunks whose copies overlap the neighbouring chunks' kernels
    xh = x64.cpu().pin_memory()
    yh = torch.empty((fn64.nnz_out, N_INST), dtype=torch.float64).pin_memory()
    for _ in range(2):
        fn64.eval_host(xh, out=yh, sync=False)
    torch.cuda.synchronize()
    e2e_ev = []
    for _ in range(args.steps):
        flush.zero_()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        fn64.eval_host(xh, out=yh, sync=False)
        e.record(stream)
        e2e_ev.append((s, e))
    torch.cuda.synchronize()
    e2e_ms = sum(s.elapsed_time(e) for s, e in e2e_ev) / args.steps
    e2e_ok = bool(torch.equal(yh, y64.cpu()))

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    # ---- FP32 kernel against the FP64 kernel on the same (FP32-rounded) inputs ----
    ref = fn64(x32.double()).cpu().numpy()
    rel32 = np.abs(y32.double().cpu().numpy() - ref) / np.max(np.abs(ref), axis=1, keepdims=True)

    # ---- roofline: measured FMA rate and per-op weights -------------------------
    pk64, pk32 = peaks.cached_or_measure(torch.cuda.get_device_name(dev), reuse=args.no_peaks)
    # the FP32 FMA chains once more, back to back for 1.5 s with the clocks sampled:
    # the rate (and SM clock) a full FP32 FMA load sustains under the power cap
    with ClockSampler(torch.cuda.current_device()) as clk_fma:
        fma32_sustained = peaks.sustained_fma("f32", 1.5)
    w64 = peaks.weighted_ops(fn64.op_counts(), pk64["weights"])
    w32 = peaks.weighted_ops(fn32.op_counts(), pk32["weights"])
    t64, t32 = ms_per_step * 1e-3, ms32 * 1e-3
    ach64 = w64 * N_INST / t64
    ach32 = w32 * N_INST / t32
    ops_live = fn64.info.n_ops
    value = world * N_INST / t64

    cpu, f64_err = None, None
    if not args.no_cpu_baseline:
        # the CPU baseline's own outputs double as a full-batch check of the FP64 kernel
        cpu, ycpu = cpu_oracle_baseline(ir, x_np, N_INST)
        rel64 = np.abs(y64.cpu().numpy() - ycpu) / np.max(np.abs(ycpu), axis=1, keepdims=True)
        f64_err = {"max_rel_scaled": float(rel64.max()),
                   "frac_within_1e-12": float(np.mean(rel64 <= 1e-12))}
    extra = None
    if not args.no_configs:
        extra = other_configs(dev, pk64, pk32, flush, reps=max(args.steps // 2, 5),
                              oracle_check=not args.no_cpu_baseline)

    line = {
        "metric": METRIC, "value": value, "unit": "instance-evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": dict(workload_config(fn64.info), launch_f64=tuning["f64"]["chosen"],
                       launch_f32=tuning["f32"]["chosen"],
                       launch="ways = W: W warps share each group of 32 instances (cooperative "
                              "kernel), coop_groups such groups per CTA; ways = 0: one thread "
                              "per instance, inst_per_thread instances each, maxrregcount a "
                              "register cap"),
        "launch_tuning_ms": tuning, "launch_tuning_seconds": t_tune,
        "gop_per_s": ops_live * N_INST / t64 * 1e-9,
        "roofline": {"bound": "alu", "achieved": ach64 * 1e-12,
                     "peak": NOMINAL_FMA_PER_S["f64"] * 1e-12,
                     "unit": "TFMA/s (FMA-equivalent ops, FP64)",
                     "frac": ach64 / NOMINAL_FMA_PER_S["f64"],
                     "traffic": NCU_TRAFFIC.get(hashlib.sha256(fn64.source().encode()).hexdigest()[:16]),
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of this "
                                       "kernel's source hash; null: no capture of the current source",
                     "kernel_source_hash": hashlib.sha256(fn64.source().encode()).hexdigest()[:16],
                     "algorithmic_bytes": int((fn64.nnz_in + fn64.nnz_out) * 8 * N_INST),
                     "peak_source": "derived: FP64 1.25 TFLOP/s = 0.625 TFMA/s (2 FMA/clk/SM x 152 SMs "
                                    "x 2.07 GHz)",
                     "peak_measured": pk64["fma_per_s"] * 1e-12,
                     "frac_of_measured": ach64 / pk64["fma_per_s"],
                     "peak_measured_source": "FP64 FMA-chain microbenchmark on this GPU (peaks.py)",
                     "work_per_instance_fma_eq": w64},
        "fp32": {"value": world * N_INST / t32, "unit": "instance-evals/s", "ms_per_step": ms32,
                 "gop_per_s": fn32.info.n_ops * N_INST / t32 * 1e-9,
                 "roofline": {"bound": "alu", "achieved": ach32 * 1e-12,
                              "peak": NOMINAL_FMA_PER_S["f32"] * 1e-12,
                              "unit": "TFMA/s (FMA-equivalent ops, FP32)",
                              "frac": ach32 / NOMINAL_FMA_PER_S["f32"],
                              "peak_source": "derived: 128 FMA/clk/SM x 152 SMs x 2.07 GHz",
                              "peak_measured": pk32["fma_per_s"] * 1e-12,
                              "frac_of_measured": ach32 / pk32["fma_per_s"],
                              "peak_sustained_fma_chains": fma32_sustained * 1e-12,
                              "clocks_under_fma_chains": clk_fma.summary(),
                              "work_per_instance_fma_eq": w32},
                 "err_vs_fp64_kernel": {"max_rel_scaled": float(rel32.max()),
                                        "median_rel_scaled": float(np.median(rel32)),
                                        "frac_within_2e-4": float(np.mean(rel32 <= 2e-4))},
                 "speedup_vs_fp64": t64 / t32, "clocks": clk32.summary()},
        "f64_err_vs_oracle": f64_err,
        "op_weights_f64": pk64["weights"], "op_weights_f32": pk32["weights"],
        "compile_seconds": {"f64": fn64.info.compile_seconds, "f32": fn32.info.compile_seconds},
        "e2e": {"value": world * N_INST / (e2e_ms * 1e-3), "unit": "instance-evals/s",
                "h2d_bytes_per_step": int(x64.numel() * 8), "d2h_bytes_per_step": int(y64.numel() * 8),
                "ms_per_step": e2e_ms, "call": "cusadi_eval_host (pinned host buffers, chunked)",
                "matches_device_result": e2e_ok},
        "gpu_launches": args.steps * fn64.info.n_segments,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "gpu": torch.cuda.get_device_name(dev),
        "other_configs": extra,
    }
    if extra is not None:
        line["adjoint_forward_ratio"] = extra["srb_rollout"]["f64"]["adjoint_forward_ratio"]
    line["bench_wall_seconds"] = time.perf_counter() - t_main
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
