"""ctypes binding of libcusadi.so (include/cusadi.h): same names, argument
marshalling only.  Every step of an evaluation runs in the library's kernels.

Importing this module never falls back to anything: if libcusadi.so is
missing or fails to load, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcusadi.so")

c_int32, c_int64, c_uint32, c_size_t = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_size_t
c_void_p, c_char_p, c_double = ctypes.c_void_p, ctypes.c_char_p, ctypes.c_double

CUSADI_OK = 0
CUSADI_E_INVALID_ARG = 1
CUSADI_E_INVALID_IR = 2
CUSADI_E_COMPILE = 3
CUSADI_E_CUDA = 4
CUSADI_E_OOM = 5
CUSADI_E_TIMEOUT = 6
CUSADI_E_UNSUPPORTED = 7

CUSADI_F64, CUSADI_F32, CUSADI_MIXED = 0, 1, 2
CUSADI_PATH_AUTO, CUSADI_PATH_COMPILED, CUSADI_PATH_INTERP = 0, 1, 2
CUSADI_ADJ_ACCUMULATE = 1
CUSADI_ADJ_REDUCE_BROADCAST = 2
CUSADI_ADJ_ACCUMULATE_BROADCAST = 4
CUSADI_NOALLOC_SCRATCH_BYTES = 64 << 20
CUSADI_BATCH_PERSISTENT, CUSADI_BATCH_PLAIN = 0, 1


class cusadi_options(ctypes.Structure):
    _fields_ = [("dtype", c_int32), ("path", c_int32), ("compile_limit_ops", c_int64),
                ("segment_ops", c_int64), ("block", c_int32), ("maxrregcount", c_int32),
                ("fmad", c_int32), ("compile_threads", c_int32), ("schedule", c_int32),
                ("inline_math", c_int32), ("adjoint", c_int32), ("ways", c_int32), ("own_math", c_int32),
                ("debug_checks", c_int32), ("inst_per_thread", c_int32), ("coop_groups", c_int32),
                ("sync_every", c_int32), ("interp_shared_kb", c_int32), ("spill_values", c_int32),
                ("spill_shared_kb", c_int32), ("pair_calls", c_int32),
                ("cache_dir", c_char_p)]


class cusadi_fn_info(ctypes.Structure):
    _fields_ = [("n_in", c_int32), ("n_out", c_int32), ("nnz_in", c_int64), ("nnz_out", c_int64),
                ("n_instr", c_int64), ("n_work", c_int64), ("n_ops_ir", c_int64),
                ("n_ops", c_int64), ("n_slots", c_int64), ("path", c_int32),
                ("n_segments", c_int32), ("dtype", c_int32), ("n_bcast_in", c_int32),
                ("compile_seconds", c_double)]


class cusadi_arg(ctypes.Structure):
    _fields_ = [("nrow", c_uint32), ("ncol", c_uint32), ("nnz", c_uint32), ("flags", c_uint32),
                ("row_offset", c_int64), ("rowptr", ctypes.POINTER(c_uint32)),
                ("col", ctypes.POINTER(c_uint32)), ("name", c_char_p)]


class CusadiError(RuntimeError):
    def __init__(self, status: int, where: str):
        L = lib()
        msg = L.cusadi_last_error().decode(errors="replace")
        super().__init__(f"{where}: {L.cusadi_status_string(status).decode()}: {msg}")
        self.status = status


# name -> (restype, argtypes), mirroring include/cusadi.h
SIGNATURES = {
    "cusadi_default_options": (None, [ctypes.POINTER(cusadi_options)]),
    "cusadi_load": (c_int32, [c_void_p, c_size_t, ctypes.POINTER(cusadi_options), ctypes.POINTER(c_void_p)]),
    "cusadi_free": (None, [c_void_p]),
    "cusadi_info": (c_int32, [c_void_p, ctypes.POINTER(cusadi_fn_info)]),
    "cusadi_arg_info": (c_int32, [c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(cusadi_arg)]),
    "cusadi_op_counts": (c_int32, [c_void_p, ctypes.c_int, ctypes.POINTER(c_int64), ctypes.c_int]),
    "cusadi_workspace_bytes": (c_size_t, [c_void_p, c_int64, ctypes.c_int]),
    "cusadi_eval": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_int64, c_void_p, c_void_p]),
    "cusadi_adjoint": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_void_p, c_int64,
                                 c_int64, c_uint32, c_void_p, c_void_p]),
    "cusadi_adjoint_shared": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_void_p, c_int64,
                                        c_void_p, c_int64, c_uint32, c_void_p, c_void_p]),
    "cusadi_sum_instances": (c_int32, [c_int32, c_void_p, c_int64, c_int64, c_int64, c_void_p, c_int32,
                                       c_void_p]),
    "cusadi_eval_noalloc": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_int64, c_void_p]),
    "cusadi_debug_count": (c_int32, [c_void_p, ctypes.POINTER(ctypes.c_uint64)]),
    "cusadi_densify": (c_int32, [c_void_p, ctypes.c_int, c_void_p, c_int64, c_void_p, c_int64, c_int64,
                                 c_void_p]),
    "cusadi_eval_host": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_int64, c_void_p,
                                   c_void_p, c_void_p, c_int32, c_void_p]),
    "cusadi_stream_wait": (c_int32, [c_void_p, c_double]),
    "cusadi_source": (c_int32, [c_void_p, ctypes.c_int, ctypes.c_int, c_char_p, ctypes.POINTER(c_size_t)]),
    "cusadi_batch_create": (c_int32, [ctypes.POINTER(c_void_p), ctypes.POINTER(c_size_t),
                                      ctypes.POINTER(c_int64), ctypes.c_int,
                                      ctypes.POINTER(cusadi_options), ctypes.POINTER(c_void_p)]),
    "cusadi_batch_free": (None, [c_void_p]),
    "cusadi_batch_workspace_bytes": (c_size_t, [c_void_p]),
    "cusadi_batch_set_block": (c_int32, [c_void_p, ctypes.c_int]),
    "cusadi_batch_eval": (c_int32, [c_void_p, ctypes.POINTER(c_void_p), ctypes.POINTER(c_int64),
                                    ctypes.POINTER(c_void_p), ctypes.POINTER(c_int64), c_void_p,
                                    ctypes.c_int, c_void_p]),
    "cusadi_batch_info": (c_int32, [c_void_p, ctypes.POINTER(c_int64), ctypes.POINTER(c_int32),
                                    ctypes.POINTER(c_int32), ctypes.POINTER(c_int32)]),
    "cusadi_batch_op_counts": (c_int32, [c_void_p, ctypes.c_int, ctypes.POINTER(c_int64), ctypes.c_int]),
    "cusadi_status_string": (c_char_p, [c_int32]),
    "cusadi_last_error": (c_char_p, []),
}

_LIB = None


def lib():
    """The loaded libcusadi.so (raises if it is missing: there is no fallback)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libcusadi.so not built ({LIB_PATH}); run "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def check(status: int, where: str) -> None:
    if status != CUSADI_OK:
        raise CusadiError(status, where)


# thin same-name wrappers ----------------------------------------------------
def cusadi_default_options() -> cusadi_options:
    o = cusadi_options()
    lib().cusadi_default_options(ctypes.byref(o))
    return o


def cusadi_load(ir: bytes, opt: cusadi_options | None = None) -> int:
    h = c_void_p()
    buf = ctypes.create_string_buffer(bytes(ir), len(ir))
    check(lib().cusadi_load(buf, len(ir), ctypes.byref(opt) if opt is not None else None,
                            ctypes.byref(h)), "cusadi_load")
    return h.value


def cusadi_free(fn: int) -> None:
    if fn and _LIB is not None:
        _LIB.cusadi_free(fn)


def cusadi_info(fn: int) -> cusadi_fn_info:
    i = cusadi_fn_info()
    check(lib().cusadi_info(fn, ctypes.byref(i)), "cusadi_info")
    return i


def cusadi_arg_info(fn: int, is_output: bool, index: int) -> cusadi_arg:
    a = cusadi_arg()
    check(lib().cusadi_arg_info(fn, int(is_output), index, ctypes.byref(a)), "cusadi_arg_info")
    return a


def cusadi_op_counts(fn: int, adjoint: bool = False, n: int = 64, f64_only: bool = False) -> list:
    buf = (c_int64 * n)()
    check(lib().cusadi_op_counts(fn, int(adjoint) | (2 if f64_only else 0), buf, n),
          "cusadi_op_counts")
    return list(buf)


def cusadi_workspace_bytes(fn: int, N: int, adjoint: bool = False) -> int:
    return int(lib().cusadi_workspace_bytes(fn, N, int(adjoint)))


def cusadi_eval(fn: int, inp: int, ld_in: int, out: int, ld_out: int, N: int, workspace: int,
                stream: int) -> None:
    check(lib().cusadi_eval(fn, inp, ld_in, out, ld_out, N, workspace, stream), "cusadi_eval")


def cusadi_adjoint(fn: int, inp: int, ld_in: int, out_bar: int, ld_ob: int, in_bar: int,
                   ld_ib: int, N: int, flags: int, workspace: int, stream: int) -> None:
    check(lib().cusadi_adjoint(fn, inp, ld_in, out_bar, ld_ob, in_bar, ld_ib, N, flags,
                               workspace, stream), "cusadi_adjoint")


def cusadi_adjoint_shared(fn: int, inp: int, ld_in: int, out_bar: int, ld_ob: int, in_bar: int,
                          ld_ib: int, shared_bar: int, N: int, flags: int, workspace: int,
                          stream: int) -> None:
    check(lib().cusadi_adjoint_shared(fn, inp, ld_in, out_bar, ld_ob, in_bar, ld_ib, shared_bar, N,
                                      flags, workspace, stream), "cusadi_adjoint_shared")


def cusadi_sum_instances(dtype: int, y: int, ld_y: int, rows: int, N: int, sums: int,
                         accumulate: bool, stream: int) -> None:
    check(lib().cusadi_sum_instances(dtype, y, ld_y, rows, N, sums, int(accumulate), stream),
          "cusadi_sum_instances")


def cusadi_eval_noalloc(fn: int, inp: int, ld_in: int, out: int, ld_out: int, N: int,
                        stream: int) -> None:
    check(lib().cusadi_eval_noalloc(fn, inp, ld_in, out, ld_out, N, stream), "cusadi_eval_noalloc")


def cusadi_eval_host(fn: int, in_host: int, ld_in: int, out_host: int, ld_out: int, N: int,
                     dev_in: int, dev_out: int, workspace: int, chunks: int, stream: int) -> None:
    check(lib().cusadi_eval_host(fn, in_host, ld_in, out_host, ld_out, N, dev_in, dev_out,
                                 workspace, chunks, stream), "cusadi_eval_host")


def cusadi_debug_count(fn: int) -> int:
    n = ctypes.c_uint64(0)
    check(lib().cusadi_debug_count(fn, ctypes.byref(n)), "cusadi_debug_count")
    return int(n.value)


def cusadi_densify(fn: int, arg: int, y: int, ld_y: int, dense: int, ld_d: int, N: int,
                   stream: int) -> None:
    check(lib().cusadi_densify(fn, arg, y, ld_y, dense, ld_d, N, stream), "cusadi_densify")


def cusadi_stream_wait(stream: int, timeout_seconds: float) -> None:
    check(lib().cusadi_stream_wait(stream, timeout_seconds), "cusadi_stream_wait")


def cusadi_source(fn: int, adjoint: bool = False, segment: int = 0) -> str:
    n = c_size_t(0)
    check(lib().cusadi_source(fn, int(adjoint), segment, None, ctypes.byref(n)), "cusadi_source")
    buf = ctypes.create_string_buffer(n.value)
    check(lib().cusadi_source(fn, int(adjoint), segment, buf, ctypes.byref(n)), "cusadi_source")
    return buf.value.decode()


def cusadi_batch_create(irs: list, N: list, opt: cusadi_options | None = None) -> int:
    n = len(irs)
    bufs = [ctypes.create_string_buffer(bytes(b), len(b)) for b in irs]
    ptrs = (c_void_p * n)(*[ctypes.cast(b, c_void_p) for b in bufs])
    sizes = (c_size_t * n)(*[len(b) for b in irs])
    ns = (c_int64 * n)(*N)
    h = c_void_p()
    check(lib().cusadi_batch_create(ptrs, sizes, ns, n, ctypes.byref(opt) if opt is not None else None,
                                    ctypes.byref(h)), "cusadi_batch_create")
    return h.value


def cusadi_batch_free(b: int) -> None:
    if b and _LIB is not None:
        _LIB.cusadi_batch_free(b)


def cusadi_batch_workspace_bytes(b: int) -> int:
    return int(lib().cusadi_batch_workspace_bytes(b))


def cusadi_batch_set_block(b: int, block: int) -> None:
    check(lib().cusadi_batch_set_block(b, block), "cusadi_batch_set_block")


def cusadi_batch_eval(b: int, ins: list, ld_in: list, outs: list, ld_out: list, workspace: int,
                      mode: int, stream: int) -> None:
    n = len(ins)
    check(lib().cusadi_batch_eval(b, (c_void_p * n)(*ins), (c_int64 * n)(*ld_in), (c_void_p * n)(*outs),
                                  (c_int64 * n)(*ld_out), workspace, mode, stream), "cusadi_batch_eval")


def cusadi_batch_info(b: int) -> tuple:
    nt, blk, grid, regs = c_int64(), c_int32(), c_int32(), c_int32()
    check(lib().cusadi_batch_info(b, ctypes.byref(nt), ctypes.byref(blk), ctypes.byref(grid),
                                  ctypes.byref(regs)), "cusadi_batch_info")
    return nt.value, blk.value, grid.value, regs.value


def cusadi_batch_op_counts(b: int, prog: int, n: int = 64) -> list:
    arr = (c_int64 * n)()
    check(lib().cusadi_batch_op_counts(b, prog, arr, n), "cusadi_batch_op_counts")
    return list(arr)
