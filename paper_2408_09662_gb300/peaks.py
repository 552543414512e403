"""Measured arithmetic peaks and per-op costs for the ALU roofline.

A straight-line program is bound by the FP32 or FP64 pipes, not by memory, so
its roofline is an op rate.  Each op is timed here as long independent chains
(8 per thread, enough threads to fill every SM) through the engine's own
compiled kernels, against the same chains of fused multiply-adds:

    peak     = FMA chains' rate (FMA/s)              - the denominator
    w(op)    = time per op / time per FMA            - FMA-equivalent cost

so ``sum_op w(op) * count(op) * N / time`` over ``peak`` is the fraction of
the measured FMA rate a kernel reaches.  Chains that need a helper op to stay
bounded (exp, log) have the helper's cost subtracted.
"""
from __future__ import annotations

import numpy as np
import torch

from . import tracer as T
from .api import Function
from .ir import Op

CHAINS = 8
LENGTH = {"fma": 1024, "add": 1024, "mul": 1024, "div": 128, "sqrt": 128, "sin": 24, "cos": 24,
          "exp_mul": 24, "log_add": 24}


def _chain_program(kind: str):
    """CHAINS independent chains of LENGTH[kind] steps, interleaved step by step."""
    g = T.Graph()
    v = g.symbols(CHAINS)
    w = g.symbols(CHAINS)
    xs = list(v)
    for _ in range(LENGTH[kind]):
        for c in range(CHAINS):
            x, y = xs[c], w[c]
            if kind == "fma":
                x = T.fma_const(0.999, x, y)
            elif kind == "add":
                x = x + y
            elif kind == "mul":
                x = x * 0.9999
            elif kind == "div":
                x = y / x
            elif kind == "sqrt":
                x = T.sqrt(x)
            elif kind == "sin":
                x = T.sin(x)
            elif kind == "cos":
                x = T.cos(x)
            elif kind == "exp_mul":
                x = T.exp(x) * 0.1
            elif kind == "log_add":
                x = T.log(x) + y
            xs[c] = x
    return T.Function([("v", v), ("w", w)], [("y", xs)]).to_ir()


# op -> (chain kind, helper op whose cost is subtracted)
OP_CHAINS = {Op.FMA_CONST: ("fma", None), Op.ADD: ("add", None), Op.SUB: ("add", None),
             Op.MUL: ("mul", None), Op.SQ: ("mul", None), Op.DIV: ("div", None),
             Op.SQRT: ("sqrt", None), Op.SIN: ("sin", None), Op.COS: ("cos", None),
             Op.EXP: ("exp_mul", Op.MUL), Op.LOG: ("log_add", Op.ADD)}


def _time(fn: Function, x: torch.Tensor, reps: int = 5) -> float:
    y = fn(x)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        fn(x, out=y)
        e.record()
        e.synchronize()
        best = min(best, s.elapsed_time(e) * 1e-3)
    return best


def measure(dtype: str, n_instances: int | None = None) -> dict:
    """{"fma_per_s": peak, "weights": {op name: w}} for "f64" or "f32"."""
    props = torch.cuda.get_device_properties(0)
    N = n_instances or props.multi_processor_count * 2048 * 4
    tdt = torch.float64 if dtype == "f64" else torch.float32
    rng = np.random.default_rng(0)
    x = torch.tensor(np.vstack([rng.uniform(0.5, 1.5, (CHAINS, N)),
                                rng.uniform(1.0, 2.0, (CHAINS, N))]), dtype=tdt, device="cuda")
    from concurrent.futures import ThreadPoolExecutor
    kinds = sorted({k for k, _ in OP_CHAINS.values()})
    # math is inlined here: the weights describe the ops, not the call overhead
    with ThreadPoolExecutor(len(kinds)) as ex:
        fns = dict(zip(kinds, ex.map(lambda k: Function(_chain_program(k), dtype=dtype, schedule=0,
                                                         inline_math=1), kinds)))
    times = {k: _time(fns[k], x) / (fns[k].info.n_ops * N) for k in kinds}
    t_fma = times["fma"]
    per_op = {}
    for op, (kind, helper) in OP_CHAINS.items():
        t = times[kind]
        if helper is not None:
            # the chain alternates op and helper: per pair = 2 * t
            t = max(2 * t - times[OP_CHAINS[helper][0]], 0.0)
        per_op[op.name] = t / t_fma
    per_op["NEG"] = 0.0   # folded into the consumer as an operand modifier
    return {"fma_per_s": 1.0 / t_fma, "weights": per_op, "instances": N}


def weighted_ops(counts, weights: dict) -> float:
    """FMA-equivalent work per instance; ops without a measured weight count 1."""
    total = 0.0
    for op in Op:
        c = counts[int(op)] if int(op) < len(counts) else 0
        if c:
            total += c * weights.get(op.name, 1.0)
    return total


def cached_or_measure(gpu_name: str, reuse: bool, path: str | None = None):
    """(f64, f32) peak records; measured now unless reuse and a record for this GPU exists."""
    import json
    import os
    path = path or os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                "_build", "peaks.json")
    if reuse and os.path.exists(path):
        with open(path) as f:
            rec = json.load(f)
        if rec.get("gpu") == gpu_name:
            return rec["f64"], rec["f32"]
    f64, f32 = measure("f64"), measure("f32")
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump({"gpu": gpu_name, "f64": f64, "f32": f32}, f)
    return f64, f32


def roofline_seconds(fn, f64_peaks: dict, f32_peaks: dict, adjoint: bool = False) -> float:
    """Seconds per instance at the measured peaks: each op costs w(op)/peak of the
    precision it runs in (a MIXED function splits its ops between the FP64 and
    FP32 pipes by their tags)."""
    counts = fn.op_counts(adjoint)
    if fn.dtype == "f64":
        return weighted_ops(counts, f64_peaks["weights"]) / f64_peaks["fma_per_s"]
    if fn.dtype == "f32":
        return weighted_ops(counts, f32_peaks["weights"]) / f32_peaks["fma_per_s"]
    c64 = fn.op_counts(adjoint, f64_only=True)
    c32 = [a - b for a, b in zip(counts, c64)]
    return (weighted_ops(c64, f64_peaks["weights"]) / f64_peaks["fma_per_s"] +
            weighted_ops(c32, f32_peaks["weights"]) / f32_peaks["fma_per_s"])


def sustained_fma(dtype: str, seconds: float = 1.5) -> float:
    """FMA/s of the FMA-chain kernel launched back to back for about `seconds`
    (one CUDA-event interval around all launches): the rate under the power
    draw of a full FMA load, which a clock sampler can watch."""
    props = torch.cuda.get_device_properties(0)
    N = props.multi_processor_count * 2048 * 4
    tdt = torch.float64 if dtype == "f64" else torch.float32
    rng = np.random.default_rng(0)
    x = torch.tensor(np.vstack([rng.uniform(0.5, 1.5, (CHAINS, N)),
                                rng.uniform(1.0, 2.0, (CHAINS, N))]), dtype=tdt, device="cuda")
    fn = Function(_chain_program("fma"), dtype=dtype, schedule=0, inline_math=1)
    per_launch = _time(fn, x)
    reps = max(1, int(seconds / per_launch))
    y = fn(x)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        fn(x, out=y)
    e.record()
    e.synchronize()
    return fn.info.n_ops * N * reps / (s.elapsed_time(e) * 1e-3)
