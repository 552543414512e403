"""Autotuner of the compiled path's launch configuration.

CusADi fixes one kernel shape for every function (one instance per thread,
§III-A, Listing 2).  Which shape is fastest here depends on the program and
the batch: the register footprint decides how many warps an SM holds, a long
program with few instances wants several warps per instance group, a short
one wants more instances per thread, and a megabyte-sized kernel wants its
warps to stay in the same stretch of code.  The tuner compiles candidate
configurations (concurrently: the compiles release the GIL), times each on the
caller's own batch (CUDA events on the current stream, L2 flushed before every
launch, median of `reps`) and keeps the fastest.  The choice is cached on disk
keyed by the program's content hash, the GPU, the dtype, the batch size (to
the next power of two) and the caller's fixed options, so a later call loads
the chosen kernel directly.

Search, in three rounds:
1. shape: ways in `ways` (0 = one thread per instance, W = W warps per group
   of 32 instances);
2. around the best shape of each family (ways = 0 and ways > 0): for ways = 0,
   instances per thread (2, 4) and register caps (128, 96, 64: measured on
   GB300, a cap of 128 takes the random 20k-op FP32 kernel from 0.61 to 0.37 ms
   and 64 the cart-pole FP64 kernel from 0.142 to 0.115 ms); for ways > 0, 2 or
   4 groups of 32 instances per CTA;
3. a one-thread winner with paired out-of-line math calls (pair_calls).
(CTA barriers every few hundred ops, sync_every, and the engine's register
budget, spill_values, measured no faster on any program and are not searched.)
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics
import tempfile
from concurrent.futures import ThreadPoolExecutor

import torch

from .api import DEFAULT_CACHE, Function, _program_bytes


def _refinements(best: dict, dtype: str, n_ops: int, n_slots: int, adjoint: bool = False) -> list:
    """Candidate option sets one step away from `best`.  Instances per thread
    multiply the live values a thread holds, so a count needing more than
    twice the 255 registers a thread can have (two per FP64 value) is not
    tried: the spills would dominate.  n_slots is the forward program's live
    set; a reverse sweep holds at least those values and their adjoints, so for
    it the estimate is doubled."""
    out = []
    if best.get("ways", 0) == 0:
        regs_per_value = 2 if dtype == "f64" else 1
        live = n_slots * (2 if adjoint else 1)
        out += [dict(best, inst_per_thread=r) for r in (2, 4) if live * r * regs_per_value <= 512]
        # register caps: more resident warps at the price of some spills
        out += [dict(best, maxrregcount=r) for r in (128, 96, 64) if live * regs_per_value > r]
    else:
        out += [dict(best, coop_groups=2), dict(best, coop_groups=4)]
    return out


def _key(ir: bytes, dtype: str, N: int, fixed: dict, device, target: str = "eval") -> str:
    props = torch.cuda.get_device_properties(device)
    bucket = 1 << max(0, (int(N) - 1).bit_length())
    h = hashlib.sha256(ir).hexdigest()[:20]
    fx = ",".join(f"{k}={fixed[k]}" for k in sorted(fixed))
    key = f"{h}|{props.name}|sm_{props.major}{props.minor}|{dtype}|N<={bucket}|{fx}"
    return key if target == "eval" else key + "|" + target


def _load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_cache(path: str, key: str, rec: dict) -> None:
    d = _load_cache(path)
    d[key] = rec
    os.makedirs(os.path.dirname(path), exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(path), prefix=".tuning")
    with os.fdopen(fd, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time(run, flush: torch.Tensor, reps: int, device) -> float:
    for _ in range(2):
        run()
    ts = []
    stream = torch.cuda.current_stream(device)
    for _ in range(reps):
        flush.zero_()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        run()
        e.record(stream)
        e.synchronize()
        ts.append(s.elapsed_time(e))
    return statistics.median(ts)


def autotune(program, x: torch.Tensor, dtype: str = "f64", ways=(0, 2, 4, 8), refine: bool = True,
             reps: int = 5, flush_bytes: int = 256 << 20, cache_dir=DEFAULT_CACHE,
             use_cache: bool = True, compile_workers: int = 8, ybar: torch.Tensor | None = None,
             adjoint_kw: dict | None = None, **fixed) -> Function:
    """The program compiled in the fastest configuration found for the batch x
    ([nnz_in, N] CUDA tensor of the dtype's element type).  `fixed` options
    (e.g. fmad=0) apply to every candidate.  With `ybar` ([nnz_out, N]) the
    candidates are timed on the reverse sweep, `fn.adjoint(x, ybar, **adjoint_kw)`,
    instead of the forward evaluation (the launch options apply to both kernels
    of a Function; the cache keeps the two choices apart).  The returned Function
    carries `.tune_record`: the chosen options, their time and every candidate's
    time (ms), what was timed, and whether the record came from the cache."""
    ir = _program_bytes(program)
    N = int(x.shape[1])
    adjoint_kw = dict(adjoint_kw or {})
    target = "eval" if ybar is None else \
        "adjoint(" + ",".join(f"{k}={adjoint_kw[k]}" for k in sorted(adjoint_kw)) + ")"
    key = _key(ir, dtype, N, fixed, x.device, target)
    path = os.path.join(cache_dir, "tuning.json") if cache_dir else None
    if use_cache and path:
        rec = _load_cache(path).get(key)
        if rec is not None:
            fn = Function(ir, dtype=dtype, cache_dir=cache_dir, **fixed, **rec["options"])
            fn.tune_record = dict(rec, from_cache=True)
            return fn
    flush = torch.empty(flush_bytes, dtype=torch.uint8, device=x.device)
    tried = {}          # frozen options -> (ms, Function)

    def build(opts):
        return Function(ir, dtype=dtype, cache_dir=cache_dir, **fixed, **opts)

    def run_round(cands):
        cands = [c for c in cands if tuple(sorted(c.items())) not in tried]
        with ThreadPoolExecutor(max(1, min(compile_workers, len(cands)))) as ex:
            fns = list(ex.map(build, cands))
        for c, fn in zip(cands, fns):       # timed one after the other, nothing else on the GPU
            if ybar is None:
                y = torch.empty((fn.nnz_out, N), dtype=fn.torch_dtype, device=x.device)
                run = lambda: fn(x, out=y)
            else:
                y = torch.empty((fn.nnz_in, N), dtype=fn.torch_dtype, device=x.device)
                run = lambda: fn.adjoint(x, ybar, out=y, **adjoint_kw)
            tried[tuple(sorted(c.items()))] = (_time(run, flush, reps, x.device), fn)

    run_round([{"ways": int(w)} for w in ways])
    if refine:
        # refine the best of each family (one thread per instance; warps per
        # group): a register cap can take the first past the second, so the
        # family that loses the first round is not dropped
        cands = []
        for fam in (lambda k: dict(k).get("ways", 0) == 0, lambda k: dict(k).get("ways", 0) > 0):
            keys = [k for k in tried if fam(k)]
            if keys:
                best = min(keys, key=lambda k: tried[k][0])
                info = tried[best][1].info
                cands += _refinements(dict(best), dtype, info.n_ops, info.n_slots, adjoint=ybar is not None)
        run_round(cands)
        # a one-thread winner also tries paired math calls (sin/cos/exp issued two
        # at a time; measured 4 % on the random 20k-op FP32 kernel)
        best = min(tried, key=lambda k: tried[k][0])
        if dict(best).get("ways", 0) == 0 and dict(best).get("inst_per_thread", 1) == 1:
            run_round([dict(dict(best), pair_calls=256)])
    best = min(tried, key=lambda k: tried[k][0])
    ms, fn = tried[best]
    rec = {"options": dict(best), "ms": ms, "N": N, "target": target,
           "candidates": [[dict(k), v[0]] for k, v in sorted(tried.items(), key=lambda kv: kv[1][0])]}
    if path:
        _store_cache(path, key, rec)
    fn.tune_record = dict(rec, from_cache=False)
    return fn
