"""Experiments of the paper reproduced on synthetic inputs; each prints a
markdown table.

    python -m paper_2408_09662_gb300.experiments ldlt   # §IV benchmark family, batch-size sweep
    python -m paper_2408_09662_gb300.experiments coop   # within-instance parallelism (§VI)
    python -m paper_2408_09662_gb300.experiments roa    # LQR quadcopter region of attraction (§V-C)
    python -m paper_2408_09662_gb300.experiments mpc    # MPC cost/violation vs iterations (§V-A, Fig. 4)
    python -m paper_2408_09662_gb300.experiments batch  # uneven batch: satellite widths
    python -m paper_2408_09662_gb300.experiments interp # interpreter vs compiled (LDL^T family)
    python -m paper_2408_09662_gb300.experiments spill  # register budget on the MPC and LQR steps
    python -m paper_2408_09662_gb300.experiments one random20k f64 4096 8   # one kernel, for a profiler
    python -m paper_2408_09662_gb300.experiments one srb f64 65536 0 adjoint
    python -m paper_2408_09662_gb300.experiments one fmachain f32 1245184 0   # the FMA-chain peak kernel

ldlt: LDL^T solves of SPD systems, each about ten times the operations of the
previous one, timed on the same inputs by the engine (compiled, or the
interpreter beyond the compile limit), by one launch per atomic op (Fig. 2
right, PyTorch eager), and by a CPU evaluator the caller may pass in.
coop: the same programs with W warps per 32 instances (``ways``) against one
thread per instance, at batch sizes too small to fill the GPU.
mpc: closed-loop simulation of the planar quadrotor under the closed-form MPC
with M = 1, 2, ... solver iterations (barrier and penalty forms, cold and
warm-started), reporting time per MPC call, accumulated cost and thrust-bound
violation -- the axes of Fig. 4.
"""
from __future__ import annotations

import statistics
import sys
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import torch

from . import inputs, programs
from .api import Function
from .vectorized import VectorizedProgram


def _spd(n, N, seed=0):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((N, n, n))
    A = M @ M.transpose(0, 2, 1) / n + np.eye(n)
    il = np.tril_indices(n)
    return np.vstack([A[:, il[0], il[1]].T, rng.standard_normal((n, N))])


_FLUSH = []


def _gpu_ms(f, reps=5, flush=False):
    """Median CUDA-event time of f() in ms.  flush=True writes 256 MB (twice the
    L2) before every timed launch, so a multi-megabyte kernel's code and its
    inputs come from DRAM as they do between unrelated launches."""
    f()
    torch.cuda.synchronize()
    if flush and not _FLUSH:
        _FLUSH.append(torch.empty(256 << 20, dtype=torch.uint8, device="cuda"))
    ts = []
    for _ in range(reps):
        if flush:
            _FLUSH[0].zero_()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        f()
        e.record()
        e.synchronize()
        ts.append(s.elapsed_time(e))
    return statistics.median(ts)


def ldlt_sweep(Ns=(1024, 4096, 16384, 65536), vectorized_max_ops=50000, cpu_ms=None):
    """cpu_ms(ir_bytes, X, n_ops) -> (milliseconds for all N instances, label) or
    None: an optional CPU baseline supplied by the caller."""
    label = "CPU ms"
    rows = []
    for n in programs.LDLT_SIZES:
        ir = programs.ldlt_spd_solve(n)
        irb = ir.to_bytes()
        fn = Function(irb, dtype="f64")
        vec = VectorizedProgram(ir) if ir.count_ops() <= vectorized_max_ops else None
        for N in Ns:
            X = _spd(n, N, seed=n)
            x = torch.tensor(X, device="cuda")
            y = fn(x)
            t_eng = _gpu_ms(lambda: fn(x, out=y))
            t_vec = _gpu_ms(lambda: vec(x), reps=2) if vec is not None else float("nan")
            t_cpu = float("nan")
            if cpu_ms is not None:
                t_cpu, label = cpu_ms(irb, X, fn.info.n_ops)
            rows.append((n, fn.info.n_ops, "compiled" if fn.compiled else "interp", N,
                         t_eng, t_vec, t_cpu))
    print(f"| n | ops | path | N | engine ms | one-launch-per-op ms | {label} | "
          "engine vs per-op | engine vs CPU |")
    print("|---|---|---|---|---|---|---|---|---|")
    for n, ops, path, N, t_eng, t_vec, t_cpu in rows:
        print(f"| {n} | {ops} | {path} | {N} | {t_eng:.4f} | {t_vec:.3f} | {t_cpu:.2f} | "
              f"{t_vec / t_eng:.0f}x | {t_cpu / t_eng:.0f}x |", flush=True)
    return rows


def coop_sweep():
    """Cooperative kernels (W warps per 32 instances) against one thread per
    instance on batches that leave most of the GPU idle at one thread each."""
    rng = np.random.default_rng(0)
    srb_x = np.vstack([np.tile(rng.normal(0, 0.1, (144, 1)), (1, 4096)),
                       rng.uniform(-0.1, 0.1, (12, 4096)), np.zeros((1, 4096))])
    mpc_x = np.vstack([rng.uniform(-0.5, 0.5, (6, 4096)), rng.uniform(-1, 1, (2, 4096))])
    work = [  # (name, program, dtype, N, inputs, ways to try)
        ("cart-pole RK4 + Jacobian", programs.cartpole_rk4().to_bytes(), "f64", 4096,
         inputs.cartpole(4096), (0, 2, 4, 8)),
        ("SRB step", programs.srb_step().to_bytes(), "f64", 4096, srb_x, (0, 4, 8)),
        ("SRB step", programs.srb_step().to_bytes(), "f32", 4096, srb_x, (0, 4, 8)),
        ("quadrotor MPC", programs.quadrotor_mpc().to_bytes(), "f64", 4096, mpc_x, (0, 4, 8)),
        ("random 20k ops", programs.random_program(20000, seed=0).to_bytes(), "f64", 4096,
         inputs.normal(64, 4096, seed=1), (0, 4, 8)),
        ("random 200k ops", programs.random_program(200000, seed=107).to_bytes(), "f32", 512,
         inputs.normal(64, 512, seed=207), (0, 8)),
    ]
    cases = [(name, irb, dt, N, X, w) for name, irb, dt, N, X, ws in work for w in ws]

    def build(c):
        t = time.perf_counter()
        fn = Function(c[1], dtype=c[2], ways=c[5])
        return fn, time.perf_counter() - t
    with ThreadPoolExecutor(6) as ex:
        fns = list(ex.map(build, cases))
    print("| program | dtype | N | ways | kernels | ms | speedup vs ways 0 | compile s |")
    print("|---|---|---|---|---|---|---|---|")
    base = {}
    rows = []
    for (name, _, dt, N, X, w), (fn, ct) in zip(cases, fns):
        x = torch.tensor(X, dtype=fn.torch_dtype, device="cuda")
        y = fn(x)
        ms = _gpu_ms(lambda: fn(x, out=y), reps=9)
        if w == 0:
            base[(name, dt, N)] = ms
        sp = base[(name, dt, N)] / ms
        rows.append((name, dt, N, w, fn.info.n_segments, ms, sp, ct))
        print(f"| {name} | {dt} | {N} | {w} | {fn.info.n_segments} | {ms:.4f} | {sp:.2f}x | {ct:.1f} |",
              flush=True)
    return rows


def _shift_horizon(z, Tn):
    """Real-time-iteration guess: states and inputs moved one stage earlier,
    the last stage repeated (in place, rows of z = x_0..x_T, u_0..u_{T-1})."""
    nx = 6 * (Tn + 1)
    z[0:6 * Tn] = z[6:nx].clone()
    z[nx:nx + 2 * (Tn - 1)] = z[nx + 2:nx + 2 * Tn].clone()


def mpc_pareto(N=4096, steps=100, Ms=(1, 2, 3, 5, 8), warm_Ms=(1, 2), dtype="f64", seed=0,
               u_max=8.0, waypoint_range=3.0):
    """Closed-loop simulation under the closed-form MPC (§V-A): every step
    solves the MPC for all N quadrotors, applies u_0 and accumulates the stage
    cost and the thrust-bound violation (quadrotor_closed_loop_step).  Cold
    start: the program's own guess (hover thrusts, rolled out).  Warm start
    (real-time iteration, §V-A): the previous solution shifted by one stage.
    The thrust limit (8, hover is 4.9) and waypoints U(-3, 3)^2 make the bound
    active early in most runs, so the forms differ in violation."""
    prm = {"u_max": u_max}
    p = dict(programs.QUADROTOR, **prm)
    Tn = p["T"]
    nz = 6 * (Tn + 1) + 2 * Tn
    cases = ([(c, M, False) for c in ("barrier", "penalty") for M in Ms] +
             [(c, M, True) for c in ("barrier", "penalty") for M in warm_Ms])

    def build(c):
        form, M, warm = c
        return Function(programs.quadrotor_mpc(dict(prm, M=M), constraint=form,
                                               warm_start=warm).to_bytes(), dtype=dtype)
    with ThreadPoolExecutor(6) as ex:
        fns = list(ex.map(build, cases))
    cl = Function(programs.quadrotor_closed_loop_step(prm).to_bytes(), dtype=dtype)
    rng = np.random.default_rng(seed)
    X0 = np.vstack([rng.uniform(-0.5, 0.5, (6, N)),
                    rng.uniform(-waypoint_range, waypoint_range, (2, N))])
    dt = cl.torch_dtype
    print(f"| form | start | M | ops | kernels | ms per MPC call (N = {N}) | closed-loop cost "
          "(mean, finite runs) | thrust-bound violation (mean of per-run max) | worst run | diverged |")
    print("|---|---|---|---|---|---|---|---|---|---|")
    rows = []
    for (form, M, warm), fn in zip(cases, fns):
        buf = torch.zeros((8 + nz + 2, N), dtype=dt, device="cuda")   # x, wp, z, J, V
        buf[0:8] = torch.tensor(X0, dtype=dt, device="cuda")
        if warm:                                         # hover guess for the first call
            buf[8:8 + 6 * (Tn + 1)] = buf[0:6].repeat(Tn + 1, 1)
            buf[8 + 6 * (Tn + 1):8 + nz] = p["mass"] * p["g"] / 2.0
        z = torch.empty((nz, N), dtype=dt, device="cuda")
        nxt = torch.empty((8, N), dtype=dt, device="cuda")
        ts = []
        for _ in range(steps):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            fn(buf[0:8 + nz] if warm else buf[0:8], out=z)
            e.record()
            buf[8:8 + nz] = z
            cl(buf, out=nxt)
            buf[0:6] = nxt[0:6]
            buf[8 + nz:8 + nz + 2] = nxt[6:8]
            if warm:
                _shift_horizon(buf[8:8 + nz], Tn)
            ts.append((s, e))
        torch.cuda.synchronize()
        ms = statistics.median(a.elapsed_time(b) for a, b in ts)
        out = buf.double().cpu().numpy()
        J, V, xs = out[8 + nz], out[8 + nz + 1], out[0:6]
        ok = np.isfinite(J) & np.all(np.isfinite(xs), axis=0) & np.all(np.abs(xs) < 1e3, axis=0)
        cost = float(np.mean(J[ok])) if ok.any() else float("nan")
        Vf = np.where(np.isfinite(V), V, np.inf)
        viol, worst = float(np.mean(Vf)), float(np.max(Vf))
        rows.append((form, "warm" if warm else "cold", M, fn.info.n_ops, fn.info.n_segments, ms,
                     cost, viol, float(1 - ok.mean()), worst))
        print(f"| {form} | {rows[-1][1]} | {M} | {fn.info.n_ops} | {fn.info.n_segments} | {ms:.3f} | "
              f"{cost:.5g} | {viol:.3g} | {worst:.3g} | {1 - ok.mean():.3f} |", flush=True)
    return rows


def lqr_roa(N=10000, steps=250, u_maxes=(6.0, 8.0, 10.0, 15.0, 20.0), seed=3, dtype="f64"):
    """Region of attraction of the LQR-controlled planar quadcopter (§V-C):
    N closed loops from zero position and angle with initial velocities
    (v_x, v_z) ~ U(-3, 3)^2 and angular rate ~ U(-24, 24), for each thrust
    limit; each step evaluates quadrotor_lqr_step (SDA Riccati solve inside)
    for all instances.  A run is stable if |z| < 0.5 everywhere after `steps`
    steps.  Prints the stable fraction per thrust limit and initial-speed bin,
    and the time per closed-loop step."""
    fn = Function(programs.quadrotor_lqr_step().to_bytes(), dtype=dtype)
    rng = np.random.default_rng(seed)
    v0 = np.vstack([rng.uniform(-3, 3, (2, N)), rng.uniform(-24, 24, (1, N))])
    speed = np.sqrt(v0[0] ** 2 + v0[1] ** 2)
    bins = [0.0, 1.0, 2.0, 3.0, 5.0]
    print(f"| thrust limit | stable (all) | " + " | ".join(f"|v| in [{a:g}, {b:g})" for a, b in zip(bins, bins[1:]))
          + f" | ms per step (N = {N}) |")
    print("|---|---|" + "---|" * (len(bins) - 1) + "---|")
    rows = []
    for u_max in u_maxes:
        X = np.zeros((16, N))
        X[3:6] = v0
        X[6], X[7], X[8], X[9:15], X[15] = u_max, 1.0, 0.01, 5.0, 0.1
        buf = [torch.tensor(X, dtype=fn.torch_dtype, device="cuda") for _ in range(2)]
        fn(buf[0], out=buf[1][:6])
        torch.cuda.synchronize()
        buf[0].copy_(torch.tensor(X, dtype=fn.torch_dtype, device="cuda"))
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for t in range(steps):
            fn(buf[t % 2], out=buf[(t + 1) % 2][:6])
        e.record()
        e.synchronize()
        z = buf[steps % 2][:6].double().cpu().numpy()
        stable = np.all(np.abs(z) < 0.5, axis=0) & np.all(np.isfinite(z), axis=0)
        frac = [float(stable[(speed >= a) & (speed < b)].mean()) for a, b in zip(bins, bins[1:])]
        ms = s.elapsed_time(e) / steps
        rows.append((u_max, float(stable.mean()), frac, ms))
        print(f"| {u_max:g} | {stable.mean():.3f} | " + " | ".join(f"{f:.3f}" for f in frac) + f" | {ms:.3f} |",
              flush=True)
    return rows


UNEVEN_BATCH = [(1000, 65536), (5000, 32768), (10000, 32768), (20000, 16384), (50000, 8192),
                (100000, 4096), (150000, 2048), (200000, 512)]


def batch_sweep(ways_list=(4, 8, 16), reps=7):
    """The uneven batch (8 random programs of the 20k-op generator, seeds
    100..107, FP32) with its long few-instance programs as satellite kernels
    of W warps per group: persistent graph launch at each tile size, the 8
    plain launches, and each satellite-sized program alone at each W; L2
    flushed before every timed launch."""
    irs = [programs.random_program(n, seed=100 + j).to_bytes() for j, (n, _) in enumerate(UNEVEN_BATCH)]
    xs = [torch.tensor(inputs.normal(64, N, seed=200 + j), dtype=torch.float32, device="cuda")
          for j, (_, N) in enumerate(UNEVEN_BATCH)]
    outs = [torch.empty((32, N), dtype=torch.float32, device="cuda") for _, N in UNEVEN_BATCH]
    from .api import Batch
    print("| satellite ways | setup s | persistent ms (tile 32 / 64 / 128) | 8 plain launches ms |")
    print("|---|---|---|---|")
    rows = []
    for w in ways_list:
        t0 = time.perf_counter()
        b = Batch(irs, [N for _, N in UNEVEN_BATCH], dtype="f32", ways=w)
        setup = time.perf_counter() - t0
        per = []
        for blk in (32, 64, 128):
            b.set_block(blk)
            per.append(_gpu_ms(lambda: b(xs, outs), reps=reps, flush=True))
        plain = _gpu_ms(lambda: b(xs, outs, mode="plain"), reps=reps, flush=True)
        rows.append((w, setup, per, plain))
        print(f"| {w} | {setup:.0f} | {per[0]:.3f} / {per[1]:.3f} / {per[2]:.3f} | {plain:.3f} |", flush=True)
    print("\n| program | N | ways | ms alone |")
    print("|---|---|---|---|")
    for j in range(4, 8):
        n, N = UNEVEN_BATCH[j]
        for w in (0,) + tuple(ways_list):
            fn = Function(irs[j], dtype="f32", ways=w)
            y = torch.empty((32, N), dtype=torch.float32, device="cuda")
            ms = _gpu_ms(lambda: fn(xs[j], out=y), reps=reps, flush=True)
            rows.append((n, N, w, ms))
            print(f"| random {n // 1000}k ops | {N} | {w} | {ms:.3f} |", flush=True)
    # what sets the batch's length: subsets of the programs at 4 warps per group
    print("\n| what runs (ways 4, best tile of 32/64/128) | ms |")
    print("|---|---|")
    for name, sel in (("all 8", range(8)), ("without the 200k-op program", range(7)),
                      ("without the 200k- and 150k-op programs", range(6)),
                      ("the four satellites only", range(4, 8)), ("the four scheduler programs only", range(4)),
                      ("the 200k-op program alone", [7])):
        sel = list(sel)
        b = Batch([irs[j] for j in sel], [UNEVEN_BATCH[j][1] for j in sel], dtype="f32", ways=4)
        X, O = [xs[j] for j in sel], [outs[j] for j in sel]
        best = min(_gpu_ms(lambda: (b.set_block(blk), b(X, O))[1], reps=reps, flush=True) for blk in (32, 64, 128))
        rows.append((name, best))
        print(f"| {name} | {best:.3f} |", flush=True)
    return rows


def interp_sweep(sizes=(22, 47), N=65536, budgets_kb=(0, 16, 48, 96)):
    """The interpreter kernel against compiled code on the LDL^T family (FP64):
    time per op-instance at each shared-memory budget for the work slots,
    and the workspace the slots beyond it need."""
    from . import _lib as L
    print("| n | ops | path | shared KB | ms | ns per op-instance x 1e3 | vs compiled | workspace MB |")
    print("|---|---|---|---|---|---|---|---|")
    rows = []
    for n in sizes:
        irb = programs.ldlt_spd_solve(n).to_bytes()
        X = _spd(n, N, seed=n)
        fns = [("compiled", None, Function(irb, dtype="f64"))] + \
              [("interp", kb, Function(irb, dtype="f64", path="interp", interp_shared_kb=kb)) for kb in budgets_kb]
        base = None
        for path, kb, fn in fns:
            x = torch.tensor(X, device="cuda")
            y = torch.empty((fn.nnz_out, N), dtype=torch.float64, device="cuda")
            ms = _gpu_ms(lambda: fn(x, out=y))
            base = ms if base is None else base
            ws = L.cusadi_workspace_bytes(fn.handle, N, False) / 1e6
            rows.append((n, fn.info.n_ops, path, kb, ms, ws))
            print(f"| {n} | {fn.info.n_ops} | {path} | {'' if kb is None else kb} | {ms:.3f} | "
                  f"{ms * 1e9 / (fn.info.n_ops * N):.3f} | {ms / base:.1f}x | {ws:.0f} |", flush=True)
    return rows


def spill_sweep(reps=7):
    """The register budget (spill_values) on the programs with the most live
    values: the closed-form MPC (906 at once) at N = 16,384 and the LQR step
    (255) at N = 10,000, against the compiler's own register allocation."""
    rng = np.random.default_rng(2)
    mpc_x = np.vstack([rng.uniform(-0.5, 0.5, (6, 16384)), rng.uniform(-1, 1, (2, 16384))])
    r = np.random.default_rng(0)
    N = 10000
    lqr_x = np.vstack([r.uniform(-0.5, 0.5, (6, N)), r.uniform(10, 20, (1, N)), r.uniform(0.8, 1.2, (1, N)),
                       r.uniform(0.008, 0.012, (1, N)), r.uniform(0.5, 10, (6, N)), r.uniform(0.05, 0.5, (1, N))])
    work = [("quadrotor MPC", programs.quadrotor_mpc().to_bytes(), dt, mpc_x, sv)
            for dt in ("f64", "mixed") for sv in (0, 112, 96, 64)]
    work += [("LQR step", programs.quadrotor_lqr_step().to_bytes(), "f64", lqr_x, sv) for sv in (0, 112, 80)]
    with ThreadPoolExecutor(8) as ex:
        fns = list(ex.map(lambda w: Function(w[1], dtype=w[2], spill_values=w[4]), work))
    print("| program | dtype | N | register budget (values) | ms | max abs diff vs no budget |")
    print("|---|---|---|---|---|---|")
    ref, rows = {}, []
    for (name, _, dt, X, sv), fn in zip(work, fns):
        x = torch.tensor(X, dtype=fn.torch_dtype, device="cuda")
        y = torch.empty((fn.nnz_out, X.shape[1]), dtype=fn.torch_dtype, device="cuda")
        ms = _gpu_ms(lambda: fn(x, out=y), reps=reps)
        yn = y.double().cpu().numpy()
        d = float(np.max(np.abs(yn - ref.setdefault((name, dt), yn))))
        rows.append((name, dt, X.shape[1], sv, ms, d))
        print(f"| {name} | {dt} | {X.shape[1]} | {sv or 'none'} | {ms:.3f} | {d:.1e} |", flush=True)
    return rows


def tune_sweep(reps=5, ways=(0, 2, 4, 8)):
    """The autotuner (tune.autotune: L2 flushed before every timed launch,
    median of `reps`) on the kernels the default launch leaves furthest from
    their roofline: the SRB step's forward and reverse sweep at N = 65,536
    (gain rows broadcast, their adjoints reduced over instances) and the
    closed-form MPC at N = 16,384 in FP64 and mixed precision.  The default
    launch (one thread per instance) is the tuner's ways = 0 candidate."""
    from .tune import autotune
    rng = np.random.default_rng(0)
    Kn = rng.normal(0, 0.1, (144, 1))
    Nk, Nm = 65536, 16384
    rk = np.random.default_rng(1)
    Xs = np.vstack([np.tile(Kn, (1, Nk)), rk.uniform(-0.1, 0.1, (12, Nk)), np.zeros((1, Nk))])
    rm = np.random.default_rng(0)
    Xm = np.vstack([rm.uniform(-0.5, 0.5, (6, Nm)), rm.uniform(-1, 1, (2, Nm))])
    srb, mpc = programs.srb_step(), programs.quadrotor_mpc()
    cases = [("SRB step forward", srb, "f32", Xs, False), ("SRB step reverse sweep", srb, "f32", Xs, True),
             ("SRB step reverse sweep", srb, "f64", Xs, True),
             ("quadrotor MPC", mpc, "f64", Xm, False), ("quadrotor MPC", mpc, "mixed", Xm, False)]
    tdt = {"f64": torch.float64, "f32": torch.float32, "mixed": torch.float32}
    print("| kernel | dtype | N | default ms | tuned ms | speedup | chosen launch | candidates | tuning s |")
    print("|---|---|---|---|---|---|---|---|---|")
    rows = []
    for name, prog, dt, X, adj in cases:
        Xd = X if dt == "f64" else X.astype(np.float32).astype(np.float64)
        x = torch.tensor(Xd, dtype=tdt[dt], device="cuda")
        kw = {}
        if adj:
            kw = dict(ybar=torch.ones((prog.nnz_out, X.shape[1]), dtype=tdt[dt], device="cuda"),
                      adjoint_kw=dict(reduce_broadcast=True))
        t0 = time.perf_counter()
        fn = autotune(prog.to_bytes(), x, dt, ways=ways, reps=reps, use_cache=False, **kw)
        secs = time.perf_counter() - t0
        rec = fn.tune_record
        base = next(ms for o, ms in rec["candidates"] if o == {"ways": 0})
        opts = ", ".join(f"{k}={v}" for k, v in sorted(rec["options"].items()))
        rows.append((name, dt, X.shape[1], base, rec["ms"], rec["options"]))
        print(f"| {name} | {dt} | {X.shape[1]} | {base:.4f} | {rec['ms']:.4f} | {base / rec['ms']:.2f}x | "
              f"{opts} | {len(rec['candidates'])} | {secs:.0f} |", flush=True)
    return rows


def one_kernel(program="random20k", dtype="f64", N=4096, ways=0, reps=3, adjoint=False):
    """Compile one program and launch it `reps` times (a small case for a
    profiler); adjoint: its reverse sweep (broadcast rows reduced) instead."""
    from . import peaks
    irs = {"random20k": lambda: programs.random_program(20000, seed=0),
           "cartpole": programs.cartpole_rk4, "mpc": programs.quadrotor_mpc,
           "lqr": programs.quadrotor_lqr_step, "srb": programs.srb_step,
           "fmachain": lambda: peaks._chain_program("fma")}
    extra = dict(schedule=0, inline_math=1) if program == "fmachain" else {}   # as peaks.py builds it
    fn = Function(irs[program]().to_bytes(), dtype=dtype, ways=ways, adjoint=int(adjoint), **extra)
    x = torch.tensor(inputs.normal(fn.nnz_in, N, seed=1) * 0.1, dtype=fn.torch_dtype, device="cuda")
    y = fn(x)
    if adjoint:
        ybar = torch.ones_like(y)
        xbar = fn.adjoint(x, ybar, reduce_broadcast=True)
        run = lambda: fn.adjoint(x, ybar, out=xbar, reduce_broadcast=True)   # noqa: E731
    else:
        run = lambda: fn(x, out=y)                                           # noqa: E731
    for _ in range(reps):
        run()
    torch.cuda.synchronize()
    print(f"{program} {dtype} N={N} ways={ways}{' adjoint' if adjoint else ''}: "
          f"{fn.info.n_segments} forward kernel(s), {_gpu_ms(run):.4f} ms")


def main(argv):
    which = argv[1] if len(argv) > 1 else ""
    if which == "ldlt":
        ldlt_sweep()
    elif which == "coop":
        coop_sweep()
    elif which == "mpc":
        mpc_pareto()
    elif which == "roa":
        lqr_roa()
    elif which == "batch":
        batch_sweep()
    elif which == "interp":
        interp_sweep()
    elif which == "spill":
        spill_sweep()
    elif which == "tune":
        tune_sweep()
    elif which == "one":
        # one <program> <dtype> <N> <ways> [adjoint]
        prog, dt, N, w = (argv[2:] + ["random20k", "f64", "4096", "0"][len(argv) - 2:])[:4]
        one_kernel(prog, dt, int(N), int(w), adjoint="adjoint" in argv[6:])
    else:
        print(__doc__)
        return 2
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
