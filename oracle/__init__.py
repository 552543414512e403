"""Oracle for the straight-line program engine.

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's CPU
baseline leg are the only code that may import this package.  Nothing here is
shared with the CUDA path, and nothing here imports it.

* ``Oracle``      ctypes front of cusadi_oracle.cpp: the plain FP64 sequential
                  interpreter of the IR (CusADi §III-A), FP32/mixed emulation,
                  the textbook reverse sweep, a first-order rounding bound
                  and Monte Carlo arithmetic (randomly perturbed evaluations).
* ``mp_eval``     the same interpreter in mpmath at high precision (truth for
                  rounding-sensitive pins).
* ``models``      direct numpy restatements of the benchmark workloads, used to
                  pin the generated programs.

Parity unpinned: none of the functions here; each is pinned by tests/.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import build as _build

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = _build()
        L = ctypes.CDLL(path)
        vp, i64, i32, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
        L.orc_load.argtypes = [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(vp)]
        L.orc_load.restype = i32
        L.orc_free.argtypes = [vp]
        L.orc_info.argtypes = [vp] + [ctypes.POINTER(i64)] * 4
        L.orc_eval.argtypes = [vp, dp, i64, dp, i64, i64, i32, i32]
        L.orc_eval.restype = i32
        L.orc_adjoint.argtypes = [vp, dp, i64, dp, i64, dp, i64, i64, i32]
        L.orc_adjoint.restype = i32
        L.orc_rounding_bound.argtypes = [vp, dp, i64, dp, i64, i64, i32, i32]
        L.orc_rounding_bound.restype = i32
        L.orc_eval_perturbed.argtypes = [vp, dp, i64, dp, i64, i64, i32, ctypes.c_uint64, i32]
        L.orc_eval_perturbed.restype = i32
        _LIB = L
    return _LIB


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


MODE_F64, MODE_F32, MODE_MIXED = 0, 1, 2


class OracleError(ValueError):
    pass


class Oracle:
    """One loaded program.  Arrays are [rows, N] float64, instance-fastest."""

    def __init__(self, ir: bytes):
        self._ir = bytes(ir)
        h = ctypes.c_void_p()
        rc = _lib().orc_load(self._ir, len(self._ir), ctypes.byref(h))
        if rc != 0:
            raise OracleError(f"oracle rejected the program (code {rc})")
        self._h = h
        a, b, c, d = (ctypes.c_int64() for _ in range(4))
        _lib().orc_info(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d))
        self.nnz_in, self.nnz_out, self.n_instr, self.n_work = a.value, b.value, c.value, d.value

    def __del__(self):
        if getattr(self, "_h", None) is not None and _LIB is not None:
            _LIB.orc_free(self._h)
            self._h = None

    def _x(self, x):
        x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
        if x.ndim == 1:
            x = x[:, None]
        if x.shape[0] != self.nnz_in:
            raise OracleError(f"expected {self.nnz_in} input rows, got {x.shape[0]}")
        return x

    def eval(self, x, mode: int = MODE_F64, threads: int = 0) -> np.ndarray:
        x = self._x(x)
        N = x.shape[1]
        y = np.zeros((self.nnz_out, N), dtype=np.float64)
        rc = _lib().orc_eval(self._h, _dp(x), N, _dp(y), N, N, mode, threads)
        if rc:
            raise OracleError(f"orc_eval failed ({rc})")
        return y

    def adjoint(self, x, ybar, threads: int = 0) -> np.ndarray:
        x = self._x(x)
        N = x.shape[1]
        ybar = np.ascontiguousarray(np.asarray(ybar, dtype=np.float64).reshape(self.nnz_out, N))
        xbar = np.zeros((self.nnz_in, N), dtype=np.float64)
        rc = _lib().orc_adjoint(self._h, _dp(x), N, _dp(ybar), N, _dp(xbar), N, N, threads)
        if rc:
            raise OracleError(f"orc_adjoint failed ({rc})")
        return xbar

    def rounding_bound(self, x, kind: int = 0, threads: int = 0) -> np.ndarray:
        """[nnz_out, N] first-order rounding bounds (kind 0: FP64 GPU vs oracle,
        kind 1: FP32 GPU vs exact)."""
        x = self._x(x)
        N = x.shape[1]
        B = np.zeros((self.nnz_out, N), dtype=np.float64)
        rc = _lib().orc_rounding_bound(self._h, _dp(x), N, _dp(B), N, N, kind, threads)
        if rc:
            raise OracleError(f"orc_rounding_bound failed ({rc})")
        return B

    def eval_perturbed(self, x, kind: int = 1, seed: int = 0, threads: int = 0) -> np.ndarray:
        """One Monte Carlo arithmetic run at FP32 sizes: FP64 evaluation with
        every result and stored output multiplied by (1 + eps_t * xi), xi
        uniform in [-1, 1) drawn per (seed, instance, instruction), eps_t as in
        rounding_bound(kind=1).  Only kind 1 exists: perturbations of FP64 size
        would drown in double's own rounding."""
        x = self._x(x)
        N = x.shape[1]
        y = np.zeros((self.nnz_out, N), dtype=np.float64)
        rc = _lib().orc_eval_perturbed(self._h, _dp(x), N, _dp(y), N, N, kind, seed, threads)
        if rc:
            raise OracleError(f"orc_eval_perturbed failed ({rc})")
        return y

    def mca_spread(self, x, y_ref, kind: int, runs: int = 8, seed: int = 1) -> np.ndarray:
        """max over `runs` Monte Carlo arithmetic runs of |y_run - y_ref|."""
        spread = np.zeros_like(y_ref)
        for r in range(runs):
            spread = np.fmax(spread, np.abs(self.eval_perturbed(x, kind, seed + r) - y_ref))
        return spread


def tolerance(oracle: Oracle, x, y_ref, tau: float, kind: int, kappa: float = 2.0,
              mca_runs: int = 0, kappa_mca: float = 4.0):
    """Per-element tolerance max(tau * s_k, kappa * B_k,i [, kappa_mca * S_k])
    with s_k = max_i |y_k,i|.

    tau is the stated relative tolerance (1e-12 FP64, 2e-4 FP32) scaled by the
    output's magnitude; B is the first-order rounding bound of the program at
    that instance, which dominates only where the program is deep enough that
    no correct implementation can meet tau.  With mca_runs > 0, S_k is the
    largest deviation from y_ref, over the instances of output row k, of that
    many Monte Carlo arithmetic runs: where errors have grown so large that the
    first-order bound no longer holds (a perturbed operand reaching a
    stationary point of the next operation, or a deep output with no correct
    digit left), S_k still measures how far a correct evaluation with rounding
    errors of the same size lands on that output.
    """
    s = np.max(np.abs(y_ref), axis=1, keepdims=True)
    B = oracle.rounding_bound(x, kind=kind)
    if kind == 1:
        B = B + np.ldexp(1.0, -24) * np.abs(y_ref)
    # where the bound is undefined (a derivative blows up at a discontinuity of
    # the program) only the stated relative tolerance applies
    tol = np.fmax(tau * s, kappa * B)
    if mca_runs:
        S = oracle.mca_spread(x, y_ref, kind, runs=mca_runs)
        tol = np.fmax(tol, kappa_mca * np.max(S, axis=1, keepdims=True))
    return tol
