"""Batch-size sweep of the §IV benchmark family (LDL^T solves of SPD systems,
each about ten times the operations of the previous one), timed three ways on
the same inputs: the engine (compiled, or the interpreter beyond the compile
limit), one launch per atomic op (Fig. 2 right, PyTorch eager) and the CPU
oracle on all host cores.  Prints a markdown table.

    python -m paper_2408_09662_gb300.experiments ldlt
"""
from __future__ import annotations

import os
import statistics
import sys
import time

import numpy as np
import torch

from . import programs
from .api import Function
from .vectorized import VectorizedProgram


def _spd(n, N, seed=0):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((N, n, n))
    A = M @ M.transpose(0, 2, 1) / n + np.eye(n)
    il = np.tril_indices(n)
    return np.vstack([A[:, il[0], il[1]].T, rng.standard_normal((n, N))])


def _gpu_ms(f, reps=5):
    f()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        f()
        e.record()
        e.synchronize()
        ts.append(s.elapsed_time(e))
    return statistics.median(ts)


def ldlt_sweep(Ns=(1024, 4096, 16384, 65536), vectorized_max_ops=50000):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from oracle import Oracle
    cores = os.cpu_count() or 1
    print("| n | ops | path | N | engine ms | one-launch-per-op ms | CPU oracle ms "
          f"({cores} cores) | engine vs per-op | engine vs CPU |")
    print("|---|---|---|---|---|---|---|---|---|")
    for n in programs.LDLT_SIZES:
        ir = programs.ldlt_spd_solve(n)
        irb = ir.to_bytes()
        fn = Function(irb, dtype="f64")
        vec = VectorizedProgram(ir) if ir.count_ops() <= vectorized_max_ops else None
        orc = Oracle(irb)
        for N in Ns:
            X = _spd(n, N, seed=n)
            x = torch.tensor(X, device="cuda")
            y = fn(x)
            t_eng = _gpu_ms(lambda: fn(x, out=y))
            t_vec = _gpu_ms(lambda: vec(x), reps=2) if vec is not None else float("nan")
            sample = min(N, max(64, int(2e8 // max(fn.info.n_ops, 1))))
            t0 = time.perf_counter()
            orc.eval(X[:, :sample], threads=cores)
            t_cpu = (time.perf_counter() - t0) * 1e3 * N / sample
            path = "compiled" if fn.compiled else "interp"
            print(f"| {n} | {fn.info.n_ops} | {path} | {N} | {t_eng:.4f} | {t_vec:.3f} | {t_cpu:.2f} | "
                  f"{t_vec / t_eng:.0f}x | {t_cpu / t_eng:.0f}x |", flush=True)


if __name__ == "__main__":
    if len(sys.argv) > 1 and sys.argv[1] == "ldlt":
        ldlt_sweep()
