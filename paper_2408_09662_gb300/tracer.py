"""Symbolic front end: trace scalar expressions into a straight-line program.

This plays the role CasADi's SX graph plays in the paper (§II-A): every value is
a node of a DAG of unary and binary atomic operations on scalars, matrices are
arrays of scalar nodes, and only structural non-zeros are ever computed.  Known
constants are folded while tracing and the structural identities 0*x = 0,
x+0 = x, x*1 = x are applied, which is how structural zeros of sparse matrix
algebra (e.g. a KKT matrix) disappear from the program.

``Function(inputs, outputs).to_ir()`` linearises the DAG into the work-vector
form of §III-A: it keeps the nodes the outputs need, orders them as traced,
and assigns work slots with reuse (an instruction may write the slot of an
operand it is the last reader of, as in Listing 2).
"""
from __future__ import annotations

import math
import struct
from contextlib import contextmanager

import numpy as np

from .ir import (ARG_BROADCAST, FLAG_F64, Instr, Op, ProgramIR, Sparsity)


class Graph:
    """Append-only SSA node store; node i may only reference nodes < i."""

    def __init__(self):
        self.op = []        # Op per node
        self.a = []         # operand node ids (-1 if unused)
        self.b = []
        self.k = []         # constant value (CONST, FMA_CONST) or input index (INPUT)
        self.flags = []
        self._consts = {}
        self._f64 = 0
        self.n_inputs = 0

    def node(self, op, a=-1, b=-1, k=0.0):
        self.op.append(op)
        self.a.append(a)
        self.b.append(b)
        self.k.append(k)
        self.flags.append(FLAG_F64 if self._f64 else 0)
        return len(self.op) - 1

    def const(self, v: float) -> "Sym":
        key = (struct.pack("<d", float(v)), self._f64)
        if key not in self._consts:
            self._consts[key] = self.node(Op.CONST, k=float(v))
        return Sym(self, self._consts[key])

    @contextmanager
    def fp64(self):
        """Tag every node created inside for FP64 evaluation (mixed precision)."""
        self._f64 += 1
        try:
            yield
        finally:
            self._f64 -= 1

    def symbols(self, n: int, name: str = "x"):
        """n fresh input scalars; their input index is assigned by Function."""
        return [Sym(self, self.node(Op.INPUT, k=-1.0)) for _ in range(n)]


def _is_num(x):
    return isinstance(x, (int, float, np.floating, np.integer))


class Sym:
    """A scalar node of a Graph, with arithmetic operators overloaded."""
    __slots__ = ("g", "i")
    __array_priority__ = 1000

    def __init__(self, g: Graph, i: int):
        self.g = g
        self.i = i

    # ---- binary arithmetic with structural simplification ----
    def __add__(self, o):
        if _is_num(o):
            return self if o == 0 else _bin(Op.ADD, self, o)
        return _bin(Op.ADD, self, o)

    def __radd__(self, o):
        if _is_num(o) and o == 0:
            return self
        return _bin(Op.ADD, o, self)

    def __sub__(self, o):
        if _is_num(o) and o == 0:
            return self
        return _bin(Op.SUB, self, o)

    def __rsub__(self, o):
        if _is_num(o) and o == 0:
            return -self
        return _bin(Op.SUB, o, self)

    def __mul__(self, o):
        if _is_num(o):
            if o == 0:
                return 0.0
            if o == 1:
                return self
            if o == -1:
                return -self
        return _bin(Op.MUL, self, o)

    __rmul__ = __mul__

    def __truediv__(self, o):
        if _is_num(o) and o == 1:
            return self
        return _bin(Op.DIV, self, o)

    def __rtruediv__(self, o):
        if _is_num(o) and o == 0:
            return 0.0
        return _bin(Op.DIV, o, self)

    def __pow__(self, o):
        if _is_num(o):
            if o == 1:
                return self
            if o == 2:
                return sq(self)
        return _bin(Op.POW, self, o)

    def __rpow__(self, o):
        return _bin(Op.POW, o, self)

    def __neg__(self):
        return Sym(self.g, self.g.node(Op.NEG, self.i))

    def __pos__(self):
        return self

    def __abs__(self):
        return fabs(self)

    def __lt__(self, o):
        return _bin(Op.LT, self, o)

    def __le__(self, o):
        return _bin(Op.LE, self, o)

    def __gt__(self, o):
        return _bin(Op.LT, o, self)

    def __ge__(self, o):
        return _bin(Op.LE, o, self)

    def __bool__(self):
        raise TypeError("a traced value has no truth value; use if_else_zero/fmin/fmax")

    def __repr__(self):
        return f"Sym({Op(self.g.op[self.i]).name}#{self.i})"


def _graph_of(*xs):
    for x in xs:
        if isinstance(x, Sym):
            return x.g
    return None


def _as_node(g, x):
    if isinstance(x, Sym):
        if x.g is not g:
            raise ValueError("mixing symbols of different graphs")
        return x.i
    return g.const(float(x)).i


_PY = {
    Op.ADD: lambda a, b: a + b, Op.SUB: lambda a, b: a - b, Op.MUL: lambda a, b: a * b,
    Op.DIV: lambda a, b: a / b, Op.POW: math.pow, Op.ATAN2: math.atan2,
    Op.FMIN: lambda a, b: min(a, b), Op.FMAX: lambda a, b: max(a, b),
    Op.LT: lambda a, b: float(a < b), Op.LE: lambda a, b: float(a <= b),
    Op.EQ: lambda a, b: float(a == b), Op.NE: lambda a, b: float(a != b),
    Op.AND: lambda a, b: float(bool(a) and bool(b)), Op.OR: lambda a, b: float(bool(a) or bool(b)),
    Op.IF_ELSE_ZERO: lambda c, x: x if c != 0 else 0.0, Op.FMOD: math.fmod,
    Op.HYPOT: math.hypot, Op.COPYSIGN: math.copysign,
    Op.NEG: lambda a: -a, Op.EXP: math.exp, Op.LOG: math.log, Op.SQ: lambda a: a * a,
    Op.SQRT: math.sqrt, Op.SIN: math.sin, Op.COS: math.cos, Op.TAN: math.tan,
    Op.ATAN: math.atan, Op.TANH: math.tanh, Op.FABS: abs, Op.NOT: lambda a: float(a == 0),
    Op.ASIN: math.asin, Op.ACOS: math.acos, Op.SINH: math.sinh, Op.COSH: math.cosh,
    Op.ERF: math.erf, Op.SIGN: lambda a: float((a > 0) - (a < 0)), Op.FLOOR: math.floor,
    Op.CEIL: math.ceil, Op.INV: lambda a: 1.0 / a, Op.LOG1P: math.log1p,
    Op.EXPM1: math.expm1,
}


def _bin(op, x, y):
    g = _graph_of(x, y)
    if g is None:
        return float(_PY[op](float(x), float(y)))
    return Sym(g, g.node(op, _as_node(g, x), _as_node(g, y)))


def _un(op, x):
    if not isinstance(x, Sym):
        return float(_PY[op](float(x)))
    return Sym(x.g, x.g.node(op, x.i))


def sq(x): return _un(Op.SQ, x)
def sqrt(x): return _un(Op.SQRT, x)
def exp(x): return _un(Op.EXP, x)
def log(x): return _un(Op.LOG, x)
def sin(x): return _un(Op.SIN, x)
def cos(x): return _un(Op.COS, x)
def tan(x): return _un(Op.TAN, x)
def atan(x): return _un(Op.ATAN, x)
def tanh(x): return _un(Op.TANH, x)
def fabs(x): return _un(Op.FABS, x)
def asin(x): return _un(Op.ASIN, x)
def acos(x): return _un(Op.ACOS, x)
def sinh(x): return _un(Op.SINH, x)
def cosh(x): return _un(Op.COSH, x)
def erf(x): return _un(Op.ERF, x)
def sign(x): return _un(Op.SIGN, x)
def floor(x): return _un(Op.FLOOR, x)
def ceil(x): return _un(Op.CEIL, x)
def inv(x): return _un(Op.INV, x)
def log1p(x): return _un(Op.LOG1P, x)
def expm1(x): return _un(Op.EXPM1, x)
def logical_not(x): return _un(Op.NOT, x)
def atan2(y, x): return _bin(Op.ATAN2, y, x)
def fmin(a, b): return _bin(Op.FMIN, a, b)
def fmax(a, b): return _bin(Op.FMAX, a, b)
def fmod(a, b): return _bin(Op.FMOD, a, b)
def hypot(a, b): return _bin(Op.HYPOT, a, b)
def copysign(a, b): return _bin(Op.COPYSIGN, a, b)
def eq(a, b): return _bin(Op.EQ, a, b)
def ne(a, b): return _bin(Op.NE, a, b)
def logical_and(a, b): return _bin(Op.AND, a, b)
def logical_or(a, b): return _bin(Op.OR, a, b)
def if_else_zero(c, x): return _bin(Op.IF_ELSE_ZERO, c, x)


def fma_const(c: float, a, b):
    """c*a + b with a single rounding, c a literal constant."""
    g = _graph_of(a, b)
    if g is None:
        return math.fma(c, float(a), float(b))
    return Sym(g, g.node(Op.FMA_CONST, _as_node(g, a), _as_node(g, b), float(c)))


# ---------------------------------------------------------------------------
# forward-mode differentiation of traced expressions (builds Jacobian programs)
# ---------------------------------------------------------------------------
def _tangent_rule(g, i, ta, tb):
    """Tangent of node i given tangents of its operands (Sym or 0.0)."""
    op = g.op[i]
    a = Sym(g, g.a[i]) if g.a[i] >= 0 else None
    b = Sym(g, g.b[i]) if g.b[i] >= 0 else None
    y = Sym(g, i)
    if op in (Op.ADD,):
        return ta + tb
    if op == Op.SUB:
        return ta - tb
    if op == Op.MUL:
        return ta * b + a * tb
    if op == Op.DIV:
        return (ta - y * tb) / b
    if op == Op.NEG:
        return -ta
    if op == Op.ASSIGN:
        return ta
    if op == Op.EXP:
        return y * ta
    if op == Op.LOG:
        return ta / a
    if op == Op.POW:
        t = b * pow_(a, b - 1.0) * ta
        return t + (y * log(a) * tb if not _zero(tb) else 0.0)
    if op == Op.SQ:
        return 2.0 * a * ta
    if op == Op.SQRT:
        return ta / (2.0 * y)
    if op == Op.SIN:
        return cos(a) * ta
    if op == Op.COS:
        return -sin(a) * ta
    if op == Op.TAN:
        return (1.0 + sq(y)) * ta
    if op == Op.ATAN:
        return ta / (1.0 + sq(a))
    if op == Op.ATAN2:
        return (b * ta - a * tb) / (sq(a) + sq(b))
    if op == Op.TANH:
        return (1.0 - sq(y)) * ta
    if op == Op.FABS:
        return sign(a) * ta
    if op == Op.FMIN:
        c = a <= b
        return if_else_zero(c, ta) + if_else_zero(logical_not(c), tb)
    if op == Op.FMAX:
        c = b <= a
        return if_else_zero(c, ta) + if_else_zero(logical_not(c), tb)
    if op == Op.FMA_CONST:
        return g.k[i] * ta + tb
    if op == Op.IF_ELSE_ZERO:
        return if_else_zero(a, tb)
    if op == Op.ASIN:
        return ta / sqrt(1.0 - sq(a))
    if op == Op.ACOS:
        return -ta / sqrt(1.0 - sq(a))
    if op == Op.SINH:
        return cosh(a) * ta
    if op == Op.COSH:
        return sinh(a) * ta
    if op == Op.ERF:
        return (2.0 / math.sqrt(math.pi)) * exp(-sq(a)) * ta
    if op == Op.INV:
        return -sq(y) * ta
    if op == Op.HYPOT:
        return (a * ta + b * tb) / y
    if op == Op.LOG1P:
        return ta / (1.0 + a)
    if op == Op.EXPM1:
        return (y + 1.0) * ta
    if op == Op.FMOD:
        return ta - ((a - y) / b) * tb
    if op == Op.COPYSIGN:
        return sign(a) * copysign(1.0, b) * ta
    # comparisons, logic, sign, floor, ceil: piecewise constant
    return 0.0


def pow_(a, b):
    return _bin(Op.POW, a, b)


def _zero(t):
    return _is_num(t) and t == 0


def forward_tangents(outputs, seeds):
    """Tangents of ``outputs`` for the input-node tangents in ``seeds``.

    ``seeds`` maps Sym -> tangent (Sym or float).  Returns a list with one
    tangent (Sym or 0.0) per output.
    """
    outs = [o for o in outputs if isinstance(o, Sym)]
    if not outs:
        return [0.0 for _ in outputs]
    g = outs[0].g
    top = max(o.i for o in outs)
    tan = {s.i: t for s, t in seeds.items()}
    for i in range(top + 1):
        if i in tan or g.op[i] in (Op.INPUT, Op.CONST):
            continue
        ta = tan.get(g.a[i], 0.0) if g.a[i] >= 0 else 0.0
        tb = tan.get(g.b[i], 0.0) if g.b[i] >= 0 else 0.0
        if _zero(ta) and _zero(tb):
            continue
        t = _tangent_rule(g, i, ta, tb)
        if not _zero(t):
            tan[i] = t
    return [tan.get(o.i, 0.0) if isinstance(o, Sym) else 0.0 for o in outputs]


def jacobian(ys, xs):
    """Dense list-of-rows Jacobian d ys / d xs by forward mode (one sweep per x)."""
    cols = [forward_tangents(ys, {x: 1.0}) for x in xs]
    return [[cols[j][r] for j in range(len(xs))] for r in range(len(ys))]


# ---------------------------------------------------------------------------
# linearisation into the work-vector IR
# ---------------------------------------------------------------------------
class Function:
    """A traced function: input arguments (lists of input Syms) -> output arguments.

    ``inputs``  list of (name, [Sym...]) or (name, [Sym...], flags) or
                (name, [Sym...], flags, Sparsity): the Syms are the argument's
                non-zeros in the pattern's storage order (default: a dense column)
    ``outputs`` list of (name, values, Sparsity or None); values are Sym or
                numbers.  With a Sparsity, values lists the non-zeros in its
                storage order; without one the output is a dense column.
    """

    def __init__(self, inputs, outputs):
        self.inputs = []
        self.in_sparsity = []
        for spec in inputs:
            name, syms = spec[0], list(spec[1])
            flags = spec[2] if len(spec) > 2 else 0
            sp = spec[3] if len(spec) > 3 and spec[3] is not None else None
            if sp is None:
                sp = Sparsity.dense(len(syms), 1, name, flags)
            elif sp.nnz != len(syms):
                raise ValueError(f"input {name}: {len(syms)} symbols for {sp.nnz} non-zeros")
            sp.name, sp.flags = name, flags
            self.inputs.append((name, syms, flags))
            self.in_sparsity.append(sp)
        self.outputs = []
        for spec in outputs:
            name, vals = spec[0], list(spec[1])
            sp = spec[2] if len(spec) > 2 and spec[2] is not None else None
            if sp is None:
                sp = Sparsity.dense(len(vals), 1, name)
            elif sp.nnz != len(vals):
                raise ValueError(f"output {name}: {len(vals)} values for {sp.nnz} non-zeros")
            sp.name = name
            self.outputs.append((name, vals, sp))
        g = None
        for _, syms, _ in self.inputs:
            for s in syms:
                g = s.g
        for _, vals, _ in self.outputs:
            for v in vals:
                if isinstance(v, Sym):
                    g = v.g
        self.g = g

    def to_ir(self) -> ProgramIR:
        g = self.g
        in_specs = list(self.in_sparsity)
        out_specs = [sp for _, _, sp in self.outputs]
        input_index = {}
        gi = 0
        for _, syms, _ in self.inputs:
            for s in syms:
                if s.i in input_index:
                    raise ValueError("a symbol appears twice among the inputs")
                input_index[s.i] = gi
                gi += 1
        # output non-zeros: node id or a literal number
        out_vals = [v for _, vals, _ in self.outputs for v in vals]
        n = len(g.op) if g is not None else 0
        # liveness from outputs
        need = bytearray(n)
        stack = [v.i for v in out_vals if isinstance(v, Sym)]
        while stack:
            i = stack.pop()
            if need[i]:
                continue
            need[i] = 1
            if g.op[i] == Op.INPUT and i not in input_index:
                raise ValueError("an output depends on a symbol that is not a declared input")
            for j in (g.a[i], g.b[i]):
                if j >= 0 and not need[j]:
                    stack.append(j)
        consts, const_ix = [], {}

        def cidx(v):
            key = struct.pack("<d", float(v))
            if key not in const_ix:
                const_ix[key] = len(consts)
                consts.append(float(v))
            return const_ix[key]

        # emission order: inputs first (argument order), then traced order
        order = [s.i for _, syms, _ in self.inputs for s in syms if need[s.i]]
        order += [i for i in range(n) if need[i] and g.op[i] != Op.INPUT]
        pos = {i: t for t, i in enumerate(order)}
        # outputs are emitted right after their value exists
        outs_at = {}
        lit_outs = []
        for oi, v in enumerate(out_vals):
            if isinstance(v, Sym):
                outs_at.setdefault(pos[v.i], []).append(oi)
            else:
                lit_outs.append((oi, float(v)))
        last_use = {}
        for t, i in enumerate(order):
            for j in (g.a[i], g.b[i]):
                if j >= 0:
                    last_use[j] = t
        for t, lst in outs_at.items():
            i = order[t]
            last_use[i] = max(last_use.get(i, t), t)
        free, n_work = [], 0
        slot = {}
        instrs = []

        def alloc():
            nonlocal n_work
            if free:
                return free.pop()
            n_work += 1
            return n_work - 1

        for t, i in enumerate(order):
            op = g.op[i]
            fl = g.flags[i]
            # operands whose last read is this instruction release their slot first
            ops_ = [j for j in (g.a[i], g.b[i]) if j >= 0]
            for j in dict.fromkeys(ops_):
                if last_use.get(j) == t:
                    free.append(slot[j])
            s = alloc()
            if op == Op.INPUT:
                instrs.append(Instr(Op.INPUT, s, input_index[i], 0, 0, fl))
            elif op == Op.CONST:
                instrs.append(Instr(Op.CONST, s, cidx(g.k[i]), 0, 0, fl))
            elif op == Op.FMA_CONST:
                instrs.append(Instr(Op.FMA_CONST, s, slot[g.a[i]], slot[g.b[i]], cidx(g.k[i]), fl))
            else:
                a = slot[g.a[i]] if g.a[i] >= 0 else 0
                b = slot[g.b[i]] if g.b[i] >= 0 else 0
                instrs.append(Instr(op, s, a, b, 0, fl))
            slot[i] = s
            for oi in outs_at.get(t, ()):
                instrs.append(Instr(Op.OUTPUT, oi, s, 0, 0, 0))
            if last_use.get(i, -1) <= t:
                free.append(s)
        for oi, v in lit_outs:
            s = alloc()
            instrs.append(Instr(Op.CONST, s, cidx(v), 0, 0, 0))
            instrs.append(Instr(Op.OUTPUT, oi, s, 0, 0, 0))
            free.append(s)
        return ProgramIR(max(n_work, 1), in_specs, out_specs, instrs, consts)
