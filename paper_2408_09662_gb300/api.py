"""PyTorch-facing API (CusADi §III-B: torch tensors on the GPU are handed to
the compiled library; data never leaves the device).

``Function`` wraps one loaded program.  Buffers are torch CUDA tensors of
shape [rows, N] (row k of instance i at [k, i]); torch supplies memory and the
current stream, the library does every step of the evaluation.
"""
from __future__ import annotations

import os

import torch

from . import _lib as L
from .ir import ProgramIR

DTYPES = {"f64": L.CUSADI_F64, "f32": L.CUSADI_F32, "mixed": L.CUSADI_MIXED}
PATHS = {"auto": L.CUSADI_PATH_AUTO, "compiled": L.CUSADI_PATH_COMPILED,
         "interp": L.CUSADI_PATH_INTERP}
DEFAULT_CACHE = os.environ.get(
    "CUSADI_CACHE_DIR",
    os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "_build", "kernels"))


def _program_bytes(program) -> bytes:
    if isinstance(program, ProgramIR):
        return program.to_bytes()
    if isinstance(program, (bytes, bytearray)):
        return bytes(program)
    with open(program, "rb") as f:
        return f.read()


class Function:
    """A straight-line program loaded into the engine.

    dtype: "f64" | "f32" | "mixed";  path: "auto" | "compiled" | "interp".
    Other keyword options map onto ``cusadi_options`` fields.
    """

    def __init__(self, program, dtype: str = "f64", path: str = "auto", cache_dir=DEFAULT_CACHE,
                 **options):
        self._fn = None
        opt = L.cusadi_default_options()
        opt.dtype = DTYPES[dtype]
        opt.path = PATHS[path]
        for k, v in options.items():
            if not hasattr(opt, k):
                raise TypeError(f"unknown option {k}")
            setattr(opt, k, int(v))
        self._cache = cache_dir.encode() if cache_dir else None
        if cache_dir:
            os.makedirs(cache_dir, exist_ok=True)
        opt.cache_dir = self._cache
        self.dtype = dtype
        self._fn = L.cusadi_load(_program_bytes(program), opt)
        self.info = L.cusadi_info(self._fn)
        self.nnz_in = self.info.nnz_in
        self.nnz_out = self.info.nnz_out
        self.torch_dtype = torch.float64 if dtype == "f64" else torch.float32
        self.inputs = [L.cusadi_arg_info(self._fn, False, j) for j in range(self.info.n_in)]
        self.outputs = [L.cusadi_arg_info(self._fn, True, j) for j in range(self.info.n_out)]
        self._stage = {}

    def __del__(self):
        if getattr(self, "_fn", None):
            L.cusadi_free(self._fn)
            self._fn = None

    @property
    def handle(self) -> int:
        return self._fn

    @property
    def compiled(self) -> bool:
        return self.info.path == L.CUSADI_PATH_COMPILED

    def op_counts(self, adjoint: bool = False, f64_only: bool = False) -> list:
        return L.cusadi_op_counts(self._fn, adjoint, f64_only=f64_only)

    def source(self, adjoint: bool = False, segment: int = 0) -> str:
        return L.cusadi_source(self._fn, adjoint, segment)

    def workspace(self, N: int, adjoint: bool = False, device=None) -> torch.Tensor | None:
        """A fresh workspace for one call.  PyTorch's caching allocator ties the
        block to the current stream, so calls on different streams never share
        one (a single cached buffer would race between concurrent calls), and
        on the same stream the block is reused in stream order at no cost."""
        nb = L.cusadi_workspace_bytes(self._fn, N, adjoint)
        if nb == 0:
            return None
        return torch.empty(nb, dtype=torch.uint8, device=device)

    @staticmethod
    def _ld(t: torch.Tensor) -> int:
        # a single row's stride is meaningless (torch may report anything); use N
        return t.stride(0) if t.shape[0] > 1 else max(t.shape[1], 1)

    def _check(self, t: torch.Tensor, rows: int, name: str):
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor (data stays on the GPU)")
        if t.dtype != self.torch_dtype:
            raise TypeError(f"{name} must be {self.torch_dtype}, got {t.dtype}")
        if t.dim() != 2 or t.shape[0] != rows or t.stride(1) != 1:
            raise ValueError(f"{name} must be [{rows}, N] with unit stride along N")

    def __call__(self, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """y = f(x).  x: [nnz_in, N]; returns (or fills) y: [nnz_out, N]."""
        self._check(x, self.nnz_in, "x")
        N = x.shape[1]
        if out is None:
            out = torch.empty((self.nnz_out, N), dtype=self.torch_dtype, device=x.device)
        self._check(out, self.nnz_out, "out")
        ws = self.workspace(N, False, x.device)
        L.cusadi_eval(self._fn, x.data_ptr(), self._ld(x), out.data_ptr(), self._ld(out), N,
                      ws.data_ptr() if ws is not None else 0,
                      torch.cuda.current_stream(x.device).cuda_stream)
        return out

    def debug_count(self) -> int:
        """Non-finite values stored since the last call (needs debug_checks=1)."""
        return L.cusadi_debug_count(self._fn)

    def dense(self, y: torch.Tensor, arg: int) -> torch.Tensor:
        """Output argument `arg` of a result y [nnz_out, N] as a dense
        [nrow, ncol, N] tensor (structural zeros filled in on the GPU)."""
        self._check(y, self.nnz_out, "y")
        a = self.outputs[arg]
        N = y.shape[1]
        d = torch.empty((a.nrow, a.ncol, N), dtype=self.torch_dtype, device=y.device)
        L.cusadi_densify(self._fn, arg, y.data_ptr(), self._ld(y), d.data_ptr(), max(N, 1), N,
                         torch.cuda.current_stream(y.device).cuda_stream)
        return d

    def eval_host(self, x: torch.Tensor, out: torch.Tensor | None = None, chunks: int = 0,
                  sync: bool = True, device=None) -> torch.Tensor:
        """y = f(x) for host tensors: x [nnz_in, N] on the CPU (pinned for the
        copies to overlap the kernels), y returned (or filled) on the CPU.  The
        library copies chunks in, evaluates and copies them out on its own
        streams; device staging buffers are kept between calls.  With
        sync=False the result is valid once the current stream reaches this
        point (an event or a synchronize)."""
        if x.is_cuda:
            raise ValueError("x must be a host tensor (use __call__ for device tensors)")
        if x.dtype != self.torch_dtype:
            raise TypeError(f"x must be {self.torch_dtype}, got {x.dtype}")
        if x.dim() != 2 or x.shape[0] != self.nnz_in or x.stride(1) != 1:
            raise ValueError(f"x must be [{self.nnz_in}, N] with unit stride along N")
        N = x.shape[1]
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        if out is None:
            out = torch.empty((self.nnz_out, N), dtype=self.torch_dtype, pin_memory=x.is_pinned())
        if out.is_cuda or out.dtype != self.torch_dtype or out.dim() != 2 or \
                out.shape != (self.nnz_out, N) or out.stride(1) != 1:
            raise ValueError(f"out must be a host tensor [{self.nnz_out}, N] of {self.torch_dtype}")
        key = (N, str(dev))
        st = self._stage.get(key)
        if st is None:
            st = (torch.empty((self.nnz_in, N), dtype=self.torch_dtype, device=dev),
                  torch.empty((self.nnz_out, N), dtype=self.torch_dtype, device=dev))
            self._stage = {key: st}                 # keep one staging pair
        ws = self.workspace(N, False, dev)
        stream = torch.cuda.current_stream(dev)
        with torch.cuda.device(dev):
            L.cusadi_eval_host(self._fn, x.data_ptr(), self._ld(x), out.data_ptr(), self._ld(out), N,
                               st[0].data_ptr(), st[1].data_ptr(),
                               ws.data_ptr() if ws is not None else 0, chunks, stream.cuda_stream)
        if sync:
            stream.synchronize()
        return out

    def adjoint(self, x: torch.Tensor, ybar: torch.Tensor, out: torch.Tensor | None = None,
                accumulate: bool = False, reduce_broadcast: bool = False,
                accumulate_broadcast: bool = False,
                shared_out: torch.Tensor | None = None) -> torch.Tensor:
        """x_bar = J(x)^T y_bar per instance (broadcast rows summed when reduce_broadcast;
        accumulate_broadcast adds those sums into out instead of overwriting them).
        With shared_out (a CUDA vector of nnz_in entries), the broadcast rows'
        sums go to shared_out[row] instead (cusadi_adjoint_shared: always
        reduced, accumulated when accumulate_broadcast) and their rows of out
        are not written."""
        self._check(x, self.nnz_in, "x")
        N = x.shape[1]
        self._check(ybar, self.nnz_out, "ybar")
        if out is None:
            out = (torch.zeros if accumulate else torch.empty)(
                (self.nnz_in, N), dtype=self.torch_dtype, device=x.device)
        self._check(out, self.nnz_in, "out")
        flags = (L.CUSADI_ADJ_ACCUMULATE if accumulate else 0) | \
                (L.CUSADI_ADJ_ACCUMULATE_BROADCAST if accumulate_broadcast else 0)
        ws = self.workspace(N, True, x.device)
        stream = torch.cuda.current_stream(x.device).cuda_stream
        if shared_out is not None:
            if not shared_out.is_cuda or shared_out.dtype != self.torch_dtype or \
                    shared_out.numel() != self.nnz_in or not shared_out.is_contiguous():
                raise ValueError(f"shared_out must be a contiguous CUDA vector of {self.nnz_in} "
                                 f"{self.torch_dtype} entries")
            L.cusadi_adjoint_shared(self._fn, x.data_ptr(), self._ld(x), ybar.data_ptr(),
                                    self._ld(ybar), out.data_ptr(), self._ld(out),
                                    shared_out.data_ptr(), N, flags,
                                    ws.data_ptr() if ws is not None else 0, stream)
            return out
        if reduce_broadcast:
            flags |= L.CUSADI_ADJ_REDUCE_BROADCAST
        L.cusadi_adjoint(self._fn, x.data_ptr(), self._ld(x), ybar.data_ptr(), self._ld(ybar),
                         out.data_ptr(), self._ld(out), N, flags,
                         ws.data_ptr() if ws is not None else 0, stream)
        return out


def sum_instances(y: torch.Tensor, out: torch.Tensor | None = None,
                  accumulate: bool = False) -> torch.Tensor:
    """Per-row sums over the instances of a [rows, N] CUDA tensor (float32 or
    float64), computed by the library in a fixed order (cusadi_sum_instances):
    the same bits on every run."""
    if not y.is_cuda or y.dim() != 2 or y.stride(1) != 1 or y.dtype not in (torch.float32, torch.float64):
        raise ValueError("y must be a [rows, N] float32/float64 CUDA tensor with unit stride along N")
    rows, N = y.shape
    if out is None:
        out = (torch.zeros if accumulate else torch.empty)(rows, dtype=y.dtype, device=y.device)
    if not out.is_cuda or out.dtype != y.dtype or out.numel() != rows or not out.is_contiguous():
        raise ValueError("out must be a contiguous CUDA vector with one entry per row of y")
    dt = L.CUSADI_F64 if y.dtype == torch.float64 else L.CUSADI_F32
    L.cusadi_sum_instances(dt, y.data_ptr(), Function._ld(y), rows, N, out.data_ptr(), accumulate,
                           torch.cuda.current_stream(y.device).cuda_stream)
    return out


class _Apply(torch.autograd.Function):
    """y = f(x) with the reverse sweep of the library as its backward."""

    @staticmethod
    def forward(ctx, fn: Function, x: torch.Tensor):
        ctx.fn = fn
        ctx.save_for_backward(x)
        return fn(x.contiguous())

    @staticmethod
    def backward(ctx, ybar):
        (x,) = ctx.saved_tensors
        return None, ctx.fn.adjoint(x.contiguous(), ybar.contiguous())


def apply(fn: Function, x: torch.Tensor) -> torch.Tensor:
    """Differentiable evaluation (torch.autograd)."""
    return _Apply.apply(fn, x)


def tuned(program, x: torch.Tensor, dtype: str = "f64", candidates=(0, 2, 4), reps: int = 5,
          flush_bytes: int = 256 << 20, **options) -> Function:
    """The program compiled once per launch configuration in `candidates`
    (ways: 0 = one thread per instance, W = W warps per group of 32
    instances), the compiles running concurrently; each is timed on x (CUDA
    events, L2 flushed before each launch, median of `reps`) and the fastest
    is returned, with `.ways` and `.tuning_ms` recording the choice."""
    from concurrent.futures import ThreadPoolExecutor
    prog = _program_bytes(program)
    with ThreadPoolExecutor(len(candidates)) as ex:   # ctypes drops the GIL while compiling
        fns = dict(zip(candidates, ex.map(lambda w: Function(prog, dtype=dtype, ways=w, **options),
                                          candidates)))
    flush = torch.empty(flush_bytes, dtype=torch.uint8, device=x.device)
    y = torch.empty((fns[candidates[0]].nnz_out, x.shape[1]), dtype=x.dtype, device=x.device)
    ms = {}
    for w, fn in fns.items():
        for _ in range(2):
            fn(x, out=y)
        ts = []
        for _ in range(reps):
            flush.zero_()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            fn(x, out=y)
            e.record()
            e.synchronize()
            ts.append(s.elapsed_time(e))
        ms[w] = sorted(ts)[len(ts) // 2]
    best = min(ms, key=ms.get)
    fn = fns[best]
    fn.ways, fn.tuning_ms = best, ms
    return fn


class Batch:
    """Several programs, each over its own fixed instance count, evaluated by one
    persistent kernel replayed from a CUDA graph (mode "persistent") or by one
    plain kernel per program (mode "plain"); both run the same per-instance code.
    With ways = W > 1, long programs with few instances run as cooperative
    satellite kernels (W warps per group of 32 instances) beside the
    persistent kernel, on parallel branches of the same graph."""

    MODES = {"persistent": L.CUSADI_BATCH_PERSISTENT, "plain": L.CUSADI_BATCH_PLAIN}

    def __init__(self, programs, N, dtype: str = "f32", block: int = 128, cache_dir=DEFAULT_CACHE,
                 **options):
        self._b = None
        opt = L.cusadi_default_options()
        opt.dtype = DTYPES[dtype]
        opt.block = block
        for k, v in options.items():
            if not hasattr(opt, k):
                raise TypeError(f"unknown option {k}")
            setattr(opt, k, int(v))
        self._cache = cache_dir.encode() if cache_dir else None
        if cache_dir:
            os.makedirs(cache_dir, exist_ok=True)
        opt.cache_dir = self._cache
        irs = [_program_bytes(p) for p in programs]
        self.N = [int(n) for n in N]
        self._b = L.cusadi_batch_create(irs, self.N, opt)
        self.torch_dtype = torch.float64 if dtype == "f64" else torch.float32
        self.block = block
        self._ws = None

    def __del__(self):
        if getattr(self, "_b", None):
            L.cusadi_batch_free(self._b)
            self._b = None

    def info(self) -> dict:
        nt, blk, grid, regs = L.cusadi_batch_info(self._b)
        return {"tiles": nt, "block": blk, "grid": grid, "registers": regs}

    def set_block(self, block: int) -> None:
        L.cusadi_batch_set_block(self._b, block)
        self.block = block

    def op_counts(self, j: int) -> list:
        """Per-op-code counts of the ops program j evaluates per instance."""
        return L.cusadi_batch_op_counts(self._b, j)

    def workspace(self, device) -> torch.Tensor | None:
        """One workspace kept for the batch: calls on one batch must not overlap
        on the GPU anyway (its buffer table and tile counter are shared)."""
        nb = L.cusadi_batch_workspace_bytes(self._b)
        if nb == 0:
            return None
        if self._ws is None or self._ws.numel() < nb:
            self._ws = torch.empty(nb, dtype=torch.uint8, device=device)
        return self._ws

    def __call__(self, xs, outs, mode: str = "persistent"):
        """xs[j]: [nnz_in_j, N_j], outs[j]: [nnz_out_j, N_j] CUDA tensors."""
        for x, o, n in zip(xs, outs, self.N):
            for t in (x, o):
                if not t.is_cuda or t.dtype != self.torch_dtype or t.stride(1) != 1 or t.shape[1] != n:
                    raise ValueError("batch buffers must be CUDA [rows, N_j] tensors of the batch dtype")
        dev = xs[0].device
        ws = self.workspace(dev)
        L.cusadi_batch_eval(self._b, [x.data_ptr() for x in xs], [Function._ld(x) for x in xs],
                            [o.data_ptr() for o in outs], [Function._ld(o) for o in outs],
                            ws.data_ptr() if ws is not None else 0, self.MODES[mode],
                            torch.cuda.current_stream(dev).cuda_stream)
        return outs

    def tune(self, xs, outs, reps: int = 5) -> int:
        """Times the persistent launch at each tile size and keeps the fastest."""
        best = None
        for block in (32, 64, 128):
            self.set_block(block)
            self(xs, outs)
            torch.cuda.synchronize()
            ts = []
            for _ in range(reps):
                s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s.record()
                self(xs, outs)
                e.record()
                e.synchronize()
                ts.append(s.elapsed_time(e))
            t = min(ts)
            if best is None or t < best[0]:
                best = (t, block)
        self.set_block(best[1])
        return best[1]
