"""Straight-line program IR: op codes and the binary wire format.

A program is a work vector plus an ordered list of instructions, each naming an
operation, the work-vector slots it reads and the slot it writes (CusADi §III-A,
the "instruction_id / instruction_input / instruction_output" triple).  Slots
are reused: an instruction reads its operands before it writes its result, so
``w[1] = w[1] + w[0]`` is legal (Listing 2).  Only the structural non-zeros of
each sparse input and output argument are read or written (§II-A).

Binary layout, little-endian, version 1::

    char  magic[4] = "CSDI"
    u32   version  = 1
    u32   n_work, n_in, n_out, n_instr, n_const, flags(=0)
    per argument (inputs first, then outputs):
        u32 nrow, ncol, nnz, arg_flags (bit 0: broadcast, inputs only)
        u32 name_len; u8 name[name_len]
        u32 rowptr[nrow + 1]; u32 col[nnz]          (CSR, row-major nz order)
    n_instr x { u16 op; u16 flags; u32 out; u32 a; u32 b; u32 c }   (20 bytes)
    n_const x f64

Input and output non-zeros are addressed by their index in the stack of all
input (resp. output) arguments' non-zeros, in argument order.  Instruction
semantics (w = work vector, x = stacked inputs, y = stacked outputs,
K = constant pool):

    INPUT       w[out] = x[a]
    OUTPUT      y[out] = w[a]
    CONST       w[out] = K[a]
    ASSIGN      w[out] = w[a]
    unary f     w[out] = f(w[a])
    binary f    w[out] = f(w[a], w[b])
    FMA_CONST   w[out] = fma(K[c], w[a], w[b])       (one rounding)
    IF_ELSE_ZERO w[out] = w[a] != 0 ? w[b] : 0

Every output non-zero is written exactly once.  Instruction flag bit 0 tags an
operation for FP64 evaluation in mixed-precision mode.
"""
from __future__ import annotations

import struct
from dataclasses import dataclass, field
from enum import IntEnum

MAGIC = b"CSDI"
VERSION = 1
FLAG_F64 = 1          # instruction flag: evaluate in FP64 under mixed precision
ARG_BROADCAST = 1     # argument flag: one value shared by every instance


class Op(IntEnum):
    INPUT = 0
    OUTPUT = 1
    CONST = 2
    ASSIGN = 3
    ADD = 4
    SUB = 5
    MUL = 6
    DIV = 7
    NEG = 8
    EXP = 9
    LOG = 10
    POW = 11
    SQ = 12
    SQRT = 13
    SIN = 14
    COS = 15
    TAN = 16
    ATAN = 17
    ATAN2 = 18
    TANH = 19
    FABS = 20
    FMIN = 21
    FMAX = 22
    FMA_CONST = 23
    IF_ELSE_ZERO = 24
    LT = 25
    LE = 26
    EQ = 27
    NE = 28
    NOT = 29
    AND = 30
    OR = 31
    ASIN = 32
    ACOS = 33
    SINH = 34
    COSH = 35
    ERF = 36
    SIGN = 37
    FLOOR = 38
    CEIL = 39
    FMOD = 40
    INV = 41
    HYPOT = 42
    LOG1P = 43
    EXPM1 = 44
    COPYSIGN = 45


UNARY = {Op.NEG, Op.EXP, Op.LOG, Op.SQ, Op.SQRT, Op.SIN, Op.COS, Op.TAN, Op.ATAN,
         Op.TANH, Op.FABS, Op.NOT, Op.ASIN, Op.ACOS, Op.SINH, Op.COSH, Op.ERF,
         Op.SIGN, Op.FLOOR, Op.CEIL, Op.INV, Op.LOG1P, Op.EXPM1, Op.ASSIGN}
BINARY = {Op.ADD, Op.SUB, Op.MUL, Op.DIV, Op.POW, Op.ATAN2, Op.FMIN, Op.FMAX,
          Op.IF_ELSE_ZERO, Op.LT, Op.LE, Op.EQ, Op.NE, Op.AND, Op.OR, Op.FMOD,
          Op.HYPOT, Op.COPYSIGN}
TRANSCENDENTAL = {Op.EXP, Op.LOG, Op.POW, Op.SIN, Op.COS, Op.TAN, Op.ATAN, Op.ATAN2,
                  Op.TANH, Op.ASIN, Op.ACOS, Op.SINH, Op.COSH, Op.ERF, Op.HYPOT,
                  Op.LOG1P, Op.EXPM1}


@dataclass
class Sparsity:
    """CSR pattern of one argument: only the listed (row, col) entries exist."""
    nrow: int
    ncol: int
    rowptr: list
    col: list
    name: str = ""
    flags: int = 0

    @property
    def nnz(self) -> int:
        return len(self.col)

    @staticmethod
    def dense(nrow: int, ncol: int = 1, name: str = "", flags: int = 0) -> "Sparsity":
        return Sparsity(nrow, ncol, [r * ncol for r in range(nrow + 1)],
                        [c for _ in range(nrow) for c in range(ncol)], name, flags)

    @staticmethod
    def from_mask(mask, name: str = "", flags: int = 0) -> "Sparsity":
        nrow = len(mask)
        ncol = len(mask[0]) if nrow else 0
        rowptr, col = [0], []
        for r in range(nrow):
            for c in range(ncol):
                if mask[r][c]:
                    col.append(c)
            rowptr.append(len(col))
        return Sparsity(nrow, ncol, rowptr, col, name, flags)

    def entries(self):
        """(row, col) of each non-zero in storage order."""
        out = []
        for r in range(self.nrow):
            for k in range(self.rowptr[r], self.rowptr[r + 1]):
                out.append((r, self.col[k]))
        return out


@dataclass
class Instr:
    op: int
    out: int = 0
    a: int = 0
    b: int = 0
    c: int = 0
    flags: int = 0


@dataclass
class ProgramIR:
    """In-memory form of one IR file."""
    n_work: int
    inputs: list
    outputs: list
    instrs: list = field(default_factory=list)
    consts: list = field(default_factory=list)

    @property
    def nnz_in(self) -> int:
        return sum(s.nnz for s in self.inputs)

    @property
    def nnz_out(self) -> int:
        return sum(s.nnz for s in self.outputs)

    def to_bytes(self) -> bytes:
        parts = [MAGIC, struct.pack("<7I", VERSION, self.n_work, len(self.inputs),
                                    len(self.outputs), len(self.instrs),
                                    len(self.consts), 0)]
        for s in list(self.inputs) + list(self.outputs):
            name = s.name.encode()
            parts.append(struct.pack("<5I", s.nrow, s.ncol, s.nnz, s.flags, len(name)))
            parts.append(name)
            parts.append(struct.pack(f"<{s.nrow + 1}I", *s.rowptr))
            parts.append(struct.pack(f"<{s.nnz}I", *s.col))
        rec = struct.Struct("<HHIIII")
        parts.append(b"".join(rec.pack(i.op, i.flags, i.out, i.a, i.b, i.c)
                              for i in self.instrs))
        parts.append(struct.pack(f"<{len(self.consts)}d", *self.consts))
        return b"".join(parts)

    def save(self, path) -> None:
        with open(path, "wb") as f:
            f.write(self.to_bytes())

    @staticmethod
    def from_bytes(buf: bytes) -> "ProgramIR":
        if buf[:4] != MAGIC:
            raise ValueError("not a CSDI program")
        off = 4
        ver, n_work, n_in, n_out, n_instr, n_const, _ = struct.unpack_from("<7I", buf, off)
        if ver != VERSION:
            raise ValueError(f"unsupported IR version {ver}")
        off += 28
        args = []
        for _ in range(n_in + n_out):
            nrow, ncol, nnz, flags, nl = struct.unpack_from("<5I", buf, off)
            off += 20
            name = buf[off:off + nl].decode()
            off += nl
            rowptr = list(struct.unpack_from(f"<{nrow + 1}I", buf, off))
            off += 4 * (nrow + 1)
            col = list(struct.unpack_from(f"<{nnz}I", buf, off))
            off += 4 * nnz
            args.append(Sparsity(nrow, ncol, rowptr, col, name, flags))
        rec = struct.Struct("<HHIIII")
        instrs = []
        for _ in range(n_instr):
            op, fl, o, a, b, c = rec.unpack_from(buf, off)
            off += 20
            instrs.append(Instr(op, o, a, b, c, fl))
        consts = list(struct.unpack_from(f"<{n_const}d", buf, off))
        return ProgramIR(n_work, args[:n_in], args[n_in:], instrs, consts)

    def count_ops(self) -> int:
        """Arithmetic instructions (everything except INPUT/OUTPUT/CONST/ASSIGN)."""
        skip = {Op.INPUT, Op.OUTPUT, Op.CONST, Op.ASSIGN}
        return sum(1 for i in self.instrs if i.op not in skip)
