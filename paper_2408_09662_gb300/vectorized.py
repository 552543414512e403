"""One launch per instruction: the program's atomic ops applied one at a time
to length-N tensors (Fig. 2, right: each atomic operation vectorised over the
instances).  A comparator for the benchmarks, built from PyTorch eager ops; the
engine itself never uses it."""
from __future__ import annotations

import torch

from .ir import Op, ProgramIR


def _cmp(f):
    return lambda a, b: f(a, b).to(a.dtype)


_UN = {Op.NEG: torch.neg, Op.EXP: torch.exp, Op.LOG: torch.log, Op.SQ: torch.square,
       Op.SQRT: torch.sqrt, Op.SIN: torch.sin, Op.COS: torch.cos, Op.TAN: torch.tan,
       Op.ATAN: torch.atan, Op.TANH: torch.tanh, Op.FABS: torch.abs, Op.ASIN: torch.asin,
       Op.ACOS: torch.acos, Op.SINH: torch.sinh, Op.COSH: torch.cosh, Op.ERF: torch.erf,
       Op.SIGN: torch.sign, Op.FLOOR: torch.floor, Op.CEIL: torch.ceil, Op.INV: torch.reciprocal,
       Op.LOG1P: torch.log1p, Op.EXPM1: torch.expm1, Op.ASSIGN: lambda a: a,
       Op.NOT: lambda a: (a == 0).to(a.dtype)}
_BIN = {Op.ADD: torch.add, Op.SUB: torch.sub, Op.MUL: torch.mul, Op.DIV: torch.div,
        Op.POW: torch.pow, Op.ATAN2: torch.atan2, Op.FMIN: torch.fmin, Op.FMAX: torch.fmax,
        Op.FMOD: torch.fmod, Op.HYPOT: torch.hypot, Op.COPYSIGN: torch.copysign,
        Op.LT: _cmp(torch.lt), Op.LE: _cmp(torch.le), Op.EQ: _cmp(torch.eq), Op.NE: _cmp(torch.ne),
        Op.AND: lambda a, b: ((a != 0) & (b != 0)).to(a.dtype),
        Op.OR: lambda a, b: ((a != 0) | (b != 0)).to(a.dtype),
        Op.IF_ELSE_ZERO: lambda c, x: torch.where(c != 0, x, torch.zeros_like(x))}


class VectorizedProgram:
    def __init__(self, program):
        self.ir = program if isinstance(program, ProgramIR) else ProgramIR.from_bytes(program)

    def __call__(self, X: torch.Tensor) -> torch.Tensor:
        ir = self.ir
        N = X.shape[1]
        w = [None] * ir.n_work
        Y = torch.empty((ir.nnz_out, N), dtype=X.dtype, device=X.device)
        bc = []
        for s in ir.inputs:
            bc += [bool(s.flags & 1)] * s.nnz
        for ins in ir.instrs:
            op = ins.op
            if op == Op.INPUT:
                w[ins.out] = X[ins.a, :1].expand(N) if bc[ins.a] else X[ins.a]
            elif op == Op.OUTPUT:
                Y[ins.out] = w[ins.a]
            elif op == Op.CONST:
                w[ins.out] = torch.full((N,), ir.consts[ins.a], dtype=X.dtype, device=X.device)
            elif op == Op.FMA_CONST:
                w[ins.out] = torch.add(w[ins.b], w[ins.a], alpha=ir.consts[ins.c])
            elif op in _BIN:
                w[ins.out] = _BIN[op](w[ins.a], w[ins.b])
            else:
                w[ins.out] = _UN[op](w[ins.a])
        return Y
