"""Host-side tests of libcusadi (no GPU): the library loads, exports every
entry point of include/cusadi.h, validates programs, runs its passes and
generates + compiles code with NVRTC."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2408_09662_gb300 import _lib as L
from paper_2408_09662_gb300 import programs
from paper_2408_09662_gb300.ir import Instr, Op, ProgramIR, Sparsity

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "cusadi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cusadi_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_entry_point():
    names = _declared_functions()
    assert "cusadi_load" in names and "cusadi_eval" in names and "cusadi_adjoint" in names
    lib = L.lib()
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(L.SIGNATURES)


def test_binding_constants_match_the_header():
    """The Python binding repeats a few #define values of include/cusadi.h; a
    change on one side only would make the binding's size checks use the
    wrong limits."""
    src = open(os.path.join(ROOT, "include", "cusadi.h")).read()
    m = re.search(r"#define CUSADI_NOALLOC_SCRATCH_BYTES \(\(size_t\)(\d+) << (\d+)\)", src)
    assert m and int(m.group(1)) << int(m.group(2)) == L.CUSADI_NOALLOC_SCRATCH_BYTES
    for name in ("CUSADI_ADJ_ACCUMULATE", "CUSADI_ADJ_REDUCE_BROADCAST",
                 "CUSADI_ADJ_ACCUMULATE_BROADCAST", "CUSADI_BATCH_PERSISTENT", "CUSADI_BATCH_PLAIN"):
        m = re.search(rf"#define {name} (\d+)u?\b", src)
        assert m and int(m.group(1)) == getattr(L, name), name


def test_default_options():
    """The defaults the header states, read through the binding's struct: a
    field out of step with include/cusadi.h would show up as a wrong value."""
    o = L.cusadi_default_options()
    assert (o.dtype, o.path, o.block, o.fmad, o.schedule) == (0, 0, 128, 1, 1)
    assert (o.compile_limit_ops, o.segment_ops, o.maxrregcount, o.inline_math) == (300000, 40000, 0, 0)
    assert (o.ways, o.own_math, o.debug_checks, o.adjoint) == (0, 0, 0, 0)
    assert (o.inst_per_thread, o.coop_groups, o.sync_every, o.interp_shared_kb) == (1, 1, 0, 48)
    assert (o.spill_values, o.spill_shared_kb, o.pair_calls) == (0, 96, 0)
    assert o.cache_dir is None
    src = open(os.path.join(ROOT, "include", "cusadi.h")).read()
    body = src[src.index("typedef struct {\n  int32_t dtype;"):src.index("} cusadi_options;")]
    fields = re.findall(r"^\s*(?:int32_t|int64_t|const char\*)\s+(\w+);", body, flags=re.M)
    assert fields == [f for f, _ in L.cusadi_options._fields_]


def test_debug_checks_instrument_the_stores():
    ir = programs.cartpole_rk4().to_bytes()
    plain = L.cusadi_load(ir, _opt())
    dbg = L.cusadi_load(ir, _opt(debug_checks=1))
    coop = L.cusadi_load(ir, _opt(debug_checks=1, ways=4))
    interp = L.cusadi_load(ir, _opt(debug_checks=1, path=L.CUSADI_PATH_INTERP))
    try:
        assert "cs_dbg" not in L.cusadi_source(plain)
        for fn in (dbg, coop):
            src = L.cusadi_source(fn)
            assert "__device__ unsigned int cs_dbg;" in src
            assert src.count("atomicAdd(&cs_dbg, 1u)") == 24          # one per output row
        with pytest.raises(L.CusadiError) as e:
            L.cusadi_debug_count(plain)                               # no checks compiled in
        assert e.value.status == L.CUSADI_E_INVALID_ARG
        with pytest.raises(L.CusadiError) as e:
            L.cusadi_debug_count(interp)
        assert e.value.status == L.CUSADI_E_UNSUPPORTED
    finally:
        for fn in (plain, dbg, coop, interp):
            L.cusadi_free(fn)


def _opt(**kw):
    o = L.cusadi_default_options()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def test_load_info_and_arg_patterns():
    fn = L.cusadi_load(programs.cartpole_rk4().to_bytes(), _opt())
    try:
        i = L.cusadi_info(fn)
        assert (i.n_in, i.n_out, i.nnz_in, i.nnz_out) == (2, 2, 5, 24)
        assert i.path == L.CUSADI_PATH_COMPILED and i.n_segments == 1
        assert 0 < i.n_ops <= i.n_ops_ir
        jac = L.cusadi_arg_info(fn, True, 1)
        assert (jac.nrow, jac.ncol, jac.nnz, jac.row_offset) == (4, 5, 20, 4)
        assert [jac.rowptr[k] for k in range(5)] == [0, 5, 10, 15, 20]
        assert [jac.col[k] for k in range(5)] == [0, 1, 2, 3, 4]
        assert jac.name == b"jac"
        counts = L.cusadi_op_counts(fn)
        assert sum(counts) == i.n_ops
        assert counts[Op.SIN] > 0 and counts[Op.COS] > 0
    finally:
        L.cusadi_free(fn)


def test_generated_source_follows_listing2():
    fn = L.cusadi_load(programs.listing2().to_bytes(), _opt())
    src = L.cusadi_source(fn)
    L.cusadi_free(fn)
    body = [l.strip() for l in src.splitlines() if l.strip().startswith(("const double v", "Y["))]
    assert body == ["const double v0 = (double)X[0ll * ldx];",
                    "const double v1 = cs_sin_d(v0);",
                    "const double v2 = v0 + v1;",
                    "const double v3 = v2 * v2;",
                    "Y[0ll * ldy] = (double)v3;"]


def test_fp32_source_uses_float_math_and_literals():
    fn = L.cusadi_load(programs.random_program(200, n_in=4, n_out=2, seed=3).to_bytes(),
                       _opt(dtype=L.CUSADI_F32))
    src = L.cusadi_source(fn)
    L.cusadi_free(fn)
    assert "double" not in src
    assert re.search(r"fmaf\(\(0x[0-9a-f.]+p[-+]\d+f\)", src)


@pytest.mark.parametrize("mutate,what", [
    (lambda b: b"XXXX" + b[4:], "magic"),
    (lambda b: b[:-3], "truncated"),
    (lambda b: b + b"\0", "trailing"),
])
def test_malformed_bytes_are_rejected(mutate, what):
    with pytest.raises(L.CusadiError) as e:
        L.cusadi_load(mutate(programs.listing2().to_bytes()))
    assert e.value.status == L.CUSADI_E_INVALID_IR


def _listing2_with(instrs, n_work=2):
    return ProgramIR(n_work, [Sparsity.dense(1, 1, "x")], [Sparsity.dense(1, 1, "y")], instrs, [])


@pytest.mark.parametrize("instrs,msg", [
    ([Instr(Op.INPUT, 0, 0), Instr(Op.SIN, 1, 5), Instr(Op.OUTPUT, 0, 1)], "undefined"),
    ([Instr(Op.INPUT, 0, 0), Instr(Op.SIN, 1, 1), Instr(Op.OUTPUT, 0, 1)], "undefined"),
    ([Instr(Op.INPUT, 0, 3), Instr(Op.OUTPUT, 0, 0)], "input row"),
    ([Instr(Op.INPUT, 0, 0)], "written 0 times"),
    ([Instr(Op.INPUT, 0, 0), Instr(Op.OUTPUT, 0, 0), Instr(Op.OUTPUT, 0, 0)], "written 2 times"),
    ([Instr(Op.INPUT, 0, 0), Instr(99, 1, 0), Instr(Op.OUTPUT, 0, 1)], "unknown op"),
    ([Instr(Op.INPUT, 0, 0), Instr(Op.CONST, 1, 4), Instr(Op.OUTPUT, 0, 1)], "constant"),
])
def test_inconsistent_programs_are_rejected(instrs, msg):
    with pytest.raises(L.CusadiError) as e:
        L.cusadi_load(_listing2_with(instrs).to_bytes())
    assert e.value.status == L.CUSADI_E_INVALID_IR
    assert msg in str(e.value)


def test_bad_sparsity_is_rejected():
    ir = programs.listing2()
    ir.outputs = [Sparsity(1, 1, [0, 2], [0, 0], "y")]
    with pytest.raises(L.CusadiError):
        L.cusadi_load(ir.to_bytes())


@pytest.mark.parametrize("field,value", [("dtype", 7), ("block", 100), ("block", 2048),
                                         ("maxrregcount", 300), ("path", 9)])
def test_bad_options_are_rejected(field, value):
    with pytest.raises(L.CusadiError) as e:
        L.cusadi_load(programs.listing2().to_bytes(), _opt(**{field: value}))
    assert e.value.status == L.CUSADI_E_INVALID_ARG


def test_eval_argument_errors_are_caught_on_the_host():
    fn = L.cusadi_load(programs.listing2().to_bytes(), _opt())
    try:
        L.cusadi_eval(fn, 0, 0, 0, 0, 0, 0, 0)        # N = 0 is a no-op
        with pytest.raises(L.CusadiError):
            L.cusadi_eval(fn, 0, 16, 0, 16, -1, 0, 0)  # N < 0
        with pytest.raises(L.CusadiError):
            L.cusadi_eval(fn, 0, 16, 8, 16, 16, 0, 0)  # NULL input
        with pytest.raises(L.CusadiError):
            L.cusadi_eval(fn, 8, 8, 8, 16, 16, 0, 0)   # ld_in < N
        with pytest.raises(L.CusadiError):
            L.cusadi_adjoint(fn, 8, 16, 8, 16, 8, 16, 16, 8, 0, 0)  # unknown flag
    finally:
        L.cusadi_free(fn)


def test_sum_and_shared_adjoint_argument_errors_are_caught_on_the_host():
    buf = ctypes.create_string_buffer(64)
    p = ctypes.addressof(buf)
    for args in [(7, p, 4, 1, 4, p), (L.CUSADI_F64, p, 2, 1, 4, p), (L.CUSADI_F64, p, 4, 1, 4, 0),
                 (L.CUSADI_F64, 0, 4, 1, 4, p), (L.CUSADI_F64, p, 4, -1, 4, p),
                 (L.CUSADI_F64, p, 4, 70000, 4, p)]:
        with pytest.raises(L.CusadiError) as e:
            L.cusadi_sum_instances(*args, False, 0)
        assert e.value.status == L.CUSADI_E_INVALID_ARG
    L.cusadi_sum_instances(L.CUSADI_F64, p, 4, 0, 4, p, False, 0)     # no rows: nothing to do
    fn = L.cusadi_load(programs.listing2().to_bytes(), None)
    try:
        with pytest.raises(L.CusadiError) as e:
            L.cusadi_adjoint_shared(fn, p, 4, p, 4, p, 4, 0, 4, 0, 0, 0)
        assert e.value.status == L.CUSADI_E_INVALID_ARG and "shared_bar" in str(e.value)
        with pytest.raises(L.CusadiError) as e:
            L.cusadi_adjoint_shared(fn, p, 4, p, 4, p, 4, p, 4, L.CUSADI_ADJ_REDUCE_BROADCAST, 0, 0)
        assert e.value.status == L.CUSADI_E_INVALID_ARG
    finally:
        L.cusadi_free(fn)


def test_eval_host_argument_errors_are_caught_on_the_host():
    fn = L.cusadi_load(programs.listing2().to_bytes(), _opt())
    try:
        L.cusadi_eval_host(fn, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0)             # N = 0 is a no-op
        L.cusadi_densify(fn, 0, 0, 0, 0, 0, 0, 0)                           # likewise
        bad = [(fn, 8, 16, 8, 16, -1, 8, 8, 0, 0, 0),                    # N < 0
               (fn, 0, 16, 8, 16, 16, 8, 8, 0, 0, 0),                    # NULL host input
               (fn, 8, 16, 8, 16, 16, 0, 8, 0, 0, 0),                    # NULL device input
               (fn, 8, 16, 0, 16, 16, 8, 8, 0, 0, 0),                    # NULL host output
               (fn, 8, 16, 8, 16, 16, 8, 0, 0, 0, 0),                    # NULL device output
               (fn, 8, 8, 8, 16, 16, 8, 8, 0, 0, 0),                     # ld_in < N
               (fn, 8, 16, 8, 8, 16, 8, 8, 0, 0, 0),                     # ld_out < N
               (fn, 8, 16, 8, 16, 16, 8, 8, 0, -1, 0)]                   # chunks < 0
        for args in bad:
            with pytest.raises(L.CusadiError) as e:
                L.cusadi_eval_host(*args)
            assert e.value.status == L.CUSADI_E_INVALID_ARG, args
    finally:
        L.cusadi_free(fn)


def test_interpreter_work_slots_split_between_shared_memory_and_workspace():
    """The interpreter keeps at most interp_shared_kb of work slots per
    128-thread CTA in shared memory and the rest in workspace rows
    ([rows x round_up(N, 128)]): no shared budget puts every slot in the
    workspace, a larger budget never needs more rows."""
    ir = programs.ldlt_spd_solve(22).to_bytes()
    rows = []
    for kb in (0, 16, 48, 200):
        fn = L.cusadi_load(ir, _opt(path=L.CUSADI_PATH_INTERP, interp_shared_kb=kb))
        try:
            n_slots = L.cusadi_info(fn).n_slots
            nb = L.cusadi_workspace_bytes(fn, 1000, False)
            assert nb % (8 * 1024) == 0
            rows.append(nb // (8 * 1024))
            if kb == 0:
                assert rows[-1] == n_slots
        finally:
            L.cusadi_free(fn)
    assert rows == sorted(rows, reverse=True) and rows[-1] < rows[0]
    assert rows[1] <= rows[0] - 16 * 1024 // (128 * 8)      # 16 KB = 16 shared slots of doubles
    with pytest.raises(L.CusadiError):
        L.cusadi_load(ir, _opt(path=L.CUSADI_PATH_INTERP, interp_shared_kb=201))


@pytest.mark.parametrize("prog,opts", [
    ("random3k", dict(dtype=L.CUSADI_F64, spill_values=24, spill_shared_kb=4, segment_ops=900)),
    ("random3k", dict(dtype=L.CUSADI_F32, spill_values=16, segment_ops=700)),
    ("mpc", dict(dtype=L.CUSADI_MIXED, spill_values=96))])
def test_register_budget_reads_follow_writes_in_every_kernel(prog, opts):
    """Under a register budget a value out of registers is stored once to its
    shared slot (cs_sp) or spill row (Wv) and re-read at each use.  Every read
    of a slot must come after a store to it in the same kernel, and every read
    of a row after a store in the same kernel or a carried row stored by an
    earlier kernel: the slots and spill rows of one kernel mean nothing in the
    next."""
    ir = {"random3k": lambda: programs.random_program(3000, seed=61),
          "mpc": lambda: programs.quadrotor_mpc()}[prog]().to_bytes()
    fn = L.cusadi_load(ir, _opt(**opts))
    try:
        carried, spilled_any = set(), False
        for seg in range(L.cusadi_info(fn).n_segments):
            src = L.cusadi_source(fn, False, seg)
            body = src[src.index("__global__"):]
            slots, rows = set(), set()
            for line in body.splitlines():
                st = line.strip()
                for m in re.finditer(r"cs_sp\[(\d+) \* blockDim\.x\]", line):
                    k = int(m.group(1))
                    if st.startswith(f"cs_sp[{k} "):
                        slots.add(k)
                    else:
                        assert k in slots, (seg, line)
                for m in re.finditer(r"Wv\[(\d+)ll \* ldw\]", line):
                    r = int(m.group(1))
                    if st.startswith(f"Wv[{r}ll"):
                        rows.add(r)
                    else:
                        assert r in rows or r in carried, (seg, line)
            spilled_any |= bool(slots or rows)
            carried |= {int(r) for r in re.findall(r"\bW\[(\d+)ll \* ldw\] =", body)}
        assert spilled_any
    finally:
        L.cusadi_free(fn)


def test_paired_calls_compile_and_cover_both_ops():
    """With pair_calls a sin/cos/exp call is issued with a later one of the same
    function whose argument already exists; the generated kernel compiles (so
    every argument is declared before its use) and each paired op's value is
    defined exactly once."""
    ir = programs.random_program(3000, seed=61).to_bytes()
    fn = L.cusadi_load(ir, _opt(dtype=L.CUSADI_F32, pair_calls=64, segment_ops=1200))
    try:
        n_pairs = 0
        for seg in range(L.cusadi_info(fn).n_segments):
            src = L.cusadi_source(fn, False, seg)
            pairs = re.findall(r"const float2 p(\d+) = cs_(sin|cos|exp)2_f\(", src)
            n_pairs += len(pairs)
            defs = re.findall(r"const float (v\d+) = ", src)
            assert len(defs) == len(set(defs))
        assert n_pairs > 0
    finally:
        L.cusadi_free(fn)
    with pytest.raises(L.CusadiError):
        L.cusadi_load(ir, _opt(pair_calls=-1))


def test_segmented_program_needs_a_workspace():
    ir = programs.random_program(3000, n_in=16, n_out=8, seed=5).to_bytes()
    fn = L.cusadi_load(ir, _opt(segment_ops=700, dtype=L.CUSADI_F32))
    try:
        i = L.cusadi_info(fn)
        assert i.n_segments >= 3
        nb = L.cusadi_workspace_bytes(fn, 1000, False)
        assert nb > 0 and nb % (4 * 1024) == 0        # rows x round_up(N, 32) floats
        with pytest.raises(L.CusadiError):
            L.cusadi_eval(fn, 8, 1000, 8, 1000, 1000, 0, 0)
    finally:
        L.cusadi_free(fn)


def test_interpreter_path_packs_without_compiling():
    ir = programs.random_program(5000, seed=7).to_bytes()
    fn = L.cusadi_load(ir, _opt(path=L.CUSADI_PATH_INTERP))
    try:
        i = L.cusadi_info(fn)
        assert i.path == L.CUSADI_PATH_INTERP and i.n_segments == 0
        assert i.compile_seconds < 5
        with pytest.raises(L.CusadiError) as e:
            L.cusadi_source(fn)
        assert e.value.status == L.CUSADI_E_UNSUPPORTED
    finally:
        L.cusadi_free(fn)


def test_auto_path_respects_compile_limit():
    ir = programs.random_program(800, seed=8).to_bytes()
    fn = L.cusadi_load(ir, _opt(compile_limit_ops=100))
    assert L.cusadi_info(fn).path == L.CUSADI_PATH_INTERP
    L.cusadi_free(fn)


def test_scheduling_lowers_live_values():
    ir = programs.random_program(5000, seed=9).to_bytes()
    a = L.cusadi_load(ir, _opt(path=L.CUSADI_PATH_INTERP, schedule=0))
    b = L.cusadi_load(ir, _opt(path=L.CUSADI_PATH_INTERP, schedule=1))
    sa, sb = L.cusadi_info(a).n_slots, L.cusadi_info(b).n_slots
    L.cusadi_free(a)
    L.cusadi_free(b)
    assert sb < sa


def test_adjoint_source_generates_reduction_for_broadcast_inputs():
    from paper_2408_09662_gb300 import tracer as T
    from paper_2408_09662_gb300.ir import ARG_BROADCAST
    g = T.Graph()
    x = g.symbols(2)
    k = g.symbols(2)
    y = [T.sin(x[0]) * k[0] + x[1] * k[1]]
    ir = T.Function([("x", x), ("k", k, ARG_BROADCAST)], [("y", y)]).to_ir()
    fn = L.cusadi_load(ir.to_bytes(), _opt())
    try:
        src = L.cusadi_source(fn, adjoint=True)
        # rows 2 and 3 are the reduced rows 0 and 1: per-instance terms, no atomics
        assert "atomicAdd" not in src and "__shfl" not in src
        assert "Wp[0ll * ldw]" in src and "Wp[1ll * ldw]" in src
        assert "cs_reduce_row[] = {2, 3}" in src and "cs_adj_f64_finish" in src
        assert L.cusadi_workspace_bytes(fn, 1000, True) == 2 * 1024 * 8   # 2 rows x round_up(N, 32)
        assert L.cusadi_workspace_bytes(fn, 1000, False) == 0
        assert L.cusadi_info(fn).n_bcast_in == 2
        counts = L.cusadi_op_counts(fn, adjoint=True)
        assert counts[Op.COS] == 1
    finally:
        L.cusadi_free(fn)


def test_batch_compiles_and_links_without_a_gpu():
    irs = [programs.random_program(n, seed=100 + j).to_bytes() for j, n in enumerate([400, 1500])]
    o = _opt(dtype=L.CUSADI_F32, segment_ops=600)
    b = L.cusadi_batch_create(irs, [1000, 65], o)
    try:
        n_tiles, block, grid, regs = L.cusadi_batch_info(b)
        assert n_tiles == 8 + 1 and block == 128 and grid == 0
        assert L.cusadi_batch_workspace_bytes(b) > 0
        L.cusadi_batch_set_block(b, 32)
        assert L.cusadi_batch_info(b)[:2] == (32 + 3, 32)
        with pytest.raises(L.CusadiError):
            L.cusadi_batch_set_block(b, 48)
    finally:
        L.cusadi_batch_free(b)
    with pytest.raises(L.CusadiError):
        L.cusadi_batch_create(irs, [1000, 0], o)


def _run_with_env(code, **env):
    import subprocess
    import sys
    e = dict(os.environ, **env)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=e, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    return r.stdout.strip()


def test_injected_compile_failure_falls_back_to_the_interpreter_under_auto():
    code = ("from paper_2408_09662_gb300 import _lib as L, programs as P\n"
            "ir = P.cartpole_rk4().to_bytes()\n"
            "o = L.cusadi_default_options()\n"
            "fn = L.cusadi_load(ir, o)\n"
            "print(L.cusadi_info(fn).path)\n"
            "o.path = L.CUSADI_PATH_COMPILED\n"
            "try:\n"
            "    L.cusadi_load(ir, o)\n"
            "    print('no error')\n"
            "except L.CusadiError as e:\n"
            "    print(e.status)\n")
    out = _run_with_env(code, CUSADI_INJECT="compile").split()
    assert out == [str(L.CUSADI_PATH_INTERP), str(L.CUSADI_E_COMPILE)]


@pytest.mark.parametrize("shared_kb", [None, "1"])
@pytest.mark.parametrize("ways", [2, 4, 8, 16])
def test_cooperative_kernels_reach_every_barrier(ways, shared_kb, monkeypatch):
    """Cooperative kernels are laid out phase by phase: each phase holds one
    `if (warp == w)` block per warp with work, and the phases are separated by
    __syncthreads() at function scope, so every thread of the CTA executes the
    same barrier instructions.  Simulating the phases, every value a warp reads
    from shared memory or the workspace was written by its owner in an earlier
    phase and not overwritten before the read.  With a 1 KB shared budget
    nearly every cross-warp value goes through workspace rows instead."""
    import re as _re
    if shared_kb is not None:
        monkeypatch.setenv("CUSADI_COOP_SHARED_KB", shared_kb)

    def sources(fn):
        for adjoint in (False, True):      # the adjoint kernels are cooperative too
            seg = 0
            while True:
                try:
                    yield L.cusadi_source(fn, adjoint, seg)
                except L.CusadiError:
                    break
                seg += 1
    for ir in (programs.cartpole_rk4(), programs.random_program(3000, seed=ways), programs.srb_step()):
        fn = L.cusadi_load(ir.to_bytes(), _opt(ways=ways, segment_ops=1200))
        try:
            for src in sources(fn):
                # the cooperative kernel (an adjoint's fixed-order finishing kernel follows it)
                body = src[src.index("if (warp =="):].split("static __device__ const long long cs_reduce_row")[0]
                assert "barrier.sync" not in src and "return" not in body
                for line in body.splitlines():
                    if "__syncthreads" in line:
                        assert line == "  __syncthreads();"
                phases = body.split("\n  __syncthreads();\n")
                writes, reads = {}, []
                for ph, text in enumerate(phases):
                    for w, block in _re.findall(r"if \(warp == (\d+)\) \{\n(.*?)\n  \}", text, flags=_re.S):
                        for m in _re.finditer(r"cs_x\[(\d+) \* 32 \+ lane\] = \(\w+\)v(\d+);", block):
                            writes.setdefault(("s", m.group(1)), []).append((ph, int(w), m.group(2)))
                        for m in _re.finditer(r"v(\d+)_\d+ = \(\w+\)cs_x\[(\d+) \* 32 \+ lane\];", block):
                            reads.append((ph, int(w), ("s", m.group(2)), m.group(1)))
                        for m in _re.finditer(r"if \(active\) W\[(\d+)ll \* ldw\] = \(\w+\)v(\d+);", block):
                            writes.setdefault(("g", m.group(1)), []).append((ph, int(w), m.group(2)))
                        for m in _re.finditer(r"v(\d+)_\d+ = \(\w+\)W\[(\d+)ll \* ldw\];", block):
                            reads.append((ph, int(w), ("g", m.group(2)), m.group(1)))
                for ph, w, loc, var in reads:
                    ws = writes.get(loc, [])
                    mine = [x for x in ws if x[2] == var]
                    if loc[0] == "g" and not mine:
                        continue          # a row carried from an earlier kernel of the program
                    assert mine and mine[0][0] < ph and mine[0][1] != w
                    assert not [x for x in ws if x[2] != var and mine[0][0] <= x[0] <= ph]
        finally:
            L.cusadi_free(fn)


def test_batch_ways_validated():
    for w in (1, 17, -1):
        with pytest.raises(L.CusadiError) as e:
            L.cusadi_batch_create([programs.listing2().to_bytes()], [16], _opt(ways=w))
        assert e.value.status == L.CUSADI_E_INVALID_ARG


def test_batch_satellites_compile_and_leave_the_scheduler():
    """A long program with few instances becomes a satellite under ways > 1:
    its instances leave the scheduler's tile table."""
    irs = [programs.random_program(n, seed=110 + j).to_bytes() for j, n in enumerate([400, 40000])]
    o = _opt(dtype=L.CUSADI_F32, segment_ops=9000, ways=8)
    b = L.cusadi_batch_create(irs, [1000, 300], o)
    try:
        n_tiles, block, _, _ = L.cusadi_batch_info(b)
        assert block == 128 and n_tiles == 8            # program 0 only: 1000 / 128
        assert L.cusadi_batch_op_counts(b, 1)[Op.ADD] > 0
    finally:
        L.cusadi_batch_free(b)
    b = L.cusadi_batch_create(irs, [1000, 300], _opt(dtype=L.CUSADI_F32, segment_ops=9000))
    try:
        assert L.cusadi_batch_info(b)[0] == 8 + 3        # no satellites without ways
    finally:
        L.cusadi_batch_free(b)


def test_cooperative_ways_validated():
    with pytest.raises(L.CusadiError):
        L.cusadi_load(programs.listing2().to_bytes(), _opt(ways=1))
    with pytest.raises(L.CusadiError):
        L.cusadi_load(programs.listing2().to_bytes(), _opt(ways=32))
