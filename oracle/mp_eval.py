"""High-precision evaluation of an IR program with mpmath (test infrastructure).

Same semantics as the FP64 oracle (CusADi §III-A: traverse the instruction list
in order over a work vector), but every value is an mpmath number carrying
``dps`` significant digits, so its result is the exact value of the program to
far below double rounding.  Own parser; nothing is shared with other code.
"""
from __future__ import annotations

import struct

import mpmath


def _parse(buf: bytes):
    if buf[:4] != b"CSDI":
        raise ValueError("bad magic")
    ver, n_work, n_in, n_out, n_instr, n_const, _ = struct.unpack_from("<7I", buf, 4)
    off = 32
    bcast = []
    nnz_out = 0
    for j in range(n_in + n_out):
        nrow, ncol, nnz, flags, nl = struct.unpack_from("<5I", buf, off)
        off += 20 + nl + 4 * (nrow + 1) + 4 * nnz
        if j < n_in:
            bcast += [bool(flags & 1)] * nnz
        else:
            nnz_out += nnz
    code = [struct.unpack_from("<HHIIII", buf, off + 20 * t) for t in range(n_instr)]
    off += 20 * n_instr
    k = list(struct.unpack_from(f"<{n_const}d", buf, off))
    return n_work, bcast, nnz_out, code, k


def mp_eval(ir: bytes, x, dps: int = 40):
    """x: [nnz_in][N] numbers -> [nnz_out][N] mpf values."""
    n_work, bcast, nnz_out, code, K = _parse(ir)
    N = len(x[0]) if len(x) else 0
    mp = mpmath.mp
    old = mp.dps
    mp.dps = dps
    try:
        f = {
            4: lambda a, b: a + b, 5: lambda a, b: a - b, 6: lambda a, b: a * b,
            7: lambda a, b: a / b, 8: lambda a, b: -a, 9: lambda a, b: mpmath.exp(a),
            10: lambda a, b: mpmath.log(a), 11: lambda a, b: mpmath.power(a, b),
            12: lambda a, b: a * a, 13: lambda a, b: mpmath.sqrt(a),
            14: lambda a, b: mpmath.sin(a), 15: lambda a, b: mpmath.cos(a),
            16: lambda a, b: mpmath.tan(a), 17: lambda a, b: mpmath.atan(a),
            18: lambda a, b: mpmath.atan2(a, b), 19: lambda a, b: mpmath.tanh(a),
            20: lambda a, b: abs(a), 21: lambda a, b: min(a, b), 22: lambda a, b: max(a, b),
            24: lambda a, b: b if a != 0 else mpmath.mpf(0),
            25: lambda a, b: mpmath.mpf(a < b), 26: lambda a, b: mpmath.mpf(a <= b),
            27: lambda a, b: mpmath.mpf(a == b), 28: lambda a, b: mpmath.mpf(a != b),
            29: lambda a, b: mpmath.mpf(a == 0), 30: lambda a, b: mpmath.mpf(a != 0 and b != 0),
            31: lambda a, b: mpmath.mpf(a != 0 or b != 0),
            32: lambda a, b: mpmath.asin(a), 33: lambda a, b: mpmath.acos(a),
            34: lambda a, b: mpmath.sinh(a), 35: lambda a, b: mpmath.cosh(a),
            36: lambda a, b: mpmath.erf(a), 37: lambda a, b: mpmath.sign(a),
            38: lambda a, b: mpmath.floor(a), 39: lambda a, b: mpmath.ceil(a),
            40: lambda a, b: mpmath.sign(a) * (abs(a) % abs(b)), 41: lambda a, b: 1 / a,
            42: lambda a, b: mpmath.hypot(a, b), 43: lambda a, b: mpmath.log1p(a),
            44: lambda a, b: mpmath.expm1(a),
            45: lambda a, b: abs(a) if b >= 0 else -abs(a),
            3: lambda a, b: a,
        }
        y = [[None] * N for _ in range(nnz_out)]
        for i in range(N):
            w = [mpmath.mpf(0)] * n_work
            for op, fl, o, a, b, c in code:
                if op == 0:
                    w[o] = mpmath.mpf(x[a][0 if bcast[a] else i])
                elif op == 1:
                    y[o][i] = w[a]
                elif op == 2:
                    w[o] = mpmath.mpf(K[a])
                elif op == 23:
                    w[o] = mpmath.mpf(K[c]) * w[a] + w[b]
                else:
                    w[o] = f[op](w[a], w[b])
        return y
    finally:
        mp.dps = old
