"""Derives the polynomial coefficients of the engine's own single-precision
sin/cos/exp fast paths (printed as C hex-float literals for codegen.cpp).

Method (no library code involved):
* argument reduction after Cody & Waite ("Software Manual for the Elementary
  Functions", 1980): x = j*(pi/2) + r with pi/2 split into three floats, or
  x = k*ln2 + r with ln2 split into two, each subtraction done by an FMA;
* near-minimax polynomials on the reduced interval: least squares at Chebyshev
  nodes, refined by Lawson's iteratively reweighted least squares toward the
  minimax (relative-error) solution, with the target function evaluated in
  mpmath at 50 digits and the final coefficients rounded to float.

    sin r = r + r t S(t),     t = r^2,  |r| <= pi/4,  S of degree 2
    cos r = 1 + t C(t),                            C of degree 3
    exp r = 1 + r + r^2 E(r), |r| <= ln2/2,        E of degree 4
"""
from __future__ import annotations

import mpmath
import numpy as np

mpmath.mp.dps = 50


def _f32(v: float) -> float:
    return float(np.float32(v))


def lawson_fit(g, w, lo, hi, deg, n=400, iters=60):
    """Coefficients c (ascending) minimising max_t |w(t) (sum c_i t^i - g(t))|."""
    k = np.arange(n)
    t = (lo + hi) / 2 + (hi - lo) / 2 * np.cos(np.pi * (k + 0.5) / n)
    G = np.array([float(g(mpmath.mpf(x))) for x in t])
    W = np.array([float(w(mpmath.mpf(x))) for x in t])
    A = np.vander(t, deg + 1, increasing=True)
    lam = np.ones(n) / n
    for _ in range(iters):
        sw = np.sqrt(lam) * W
        c, *_ = np.linalg.lstsq(A * sw[:, None], G * sw, rcond=None)
        err = np.abs(W * (A @ c - G))
        lam = lam * err
        lam /= lam.sum()
    return c


def sin_coeffs():
    hi = float((mpmath.pi / 4) ** 2)
    g = lambda t: (mpmath.sin(mpmath.sqrt(t)) / mpmath.sqrt(t) - 1) / t if t > 0 else mpmath.mpf(-1) / 6
    # relative error of sin: weight r t / sin r
    w = lambda t: (mpmath.sqrt(t) * t / mpmath.sin(mpmath.sqrt(t))) if t > 0 else mpmath.mpf(0)
    return lawson_fit(g, w, 1e-12, hi, 2)


def cos_coeffs():
    hi = float((mpmath.pi / 4) ** 2)
    g = lambda t: (mpmath.cos(mpmath.sqrt(t)) - 1) / t if t > 0 else mpmath.mpf(-0.5)
    w = lambda t: t / mpmath.cos(mpmath.sqrt(t))
    return lawson_fit(g, w, 1e-12, hi, 3)


def exp_coeffs():
    h = float(mpmath.log(2) / 2)
    g = lambda r: (mpmath.exp(r) - 1 - r) / (r * r) if r != 0 else mpmath.mpf(0.5)
    w = lambda r: r * r / mpmath.exp(r)
    return lawson_fit(g, w, -h, h, 4)


def split(v, bits, parts):
    """v as a sum of `parts` floats: the leading ones keep `bits` significant bits
    (so k * part is exact in a float for |k| < 2^(24 - bits)), the last is v's
    float-rounded remainder."""
    out, rest = [], mpmath.mpf(v)
    for i in range(parts):
        if i < parts - 1:
            e = int(mpmath.floor(mpmath.log(abs(rest), 2)))
            q = mpmath.mpf(2) ** (e - bits + 1)
            f = float(mpmath.nint(rest / q) * q)
        else:
            f = _f32(float(rest))
        out.append(f)
        rest -= mpmath.mpf(f)
    return out


def max_rel_error(kind, c):
    """Max relative error of the float-rounded polynomial, evaluated exactly."""
    cf = [mpmath.mpf(_f32(x)) for x in c]
    if kind == "exp":
        xs = np.linspace(-float(mpmath.log(2) / 2), float(mpmath.log(2) / 2), 4001)
    else:
        xs = np.linspace(1e-6, float(mpmath.pi / 4), 4001)
    worst = 0
    for x in xs:
        r = mpmath.mpf(x)
        t = r * r
        if kind == "sin":
            p = r + r * t * (cf[0] + t * (cf[1] + t * cf[2]))
            f = mpmath.sin(r)
        elif kind == "cos":
            p = 1 + t * (cf[0] + t * (cf[1] + t * (cf[2] + t * cf[3])))
            f = mpmath.cos(r)
        else:
            p = 1 + r + t * (cf[0] + r * (cf[1] + r * (cf[2] + r * (cf[3] + r * cf[4]))))
            f = mpmath.exp(r)
        worst = max(worst, abs(p / f - 1))
    return float(worst)


def hexf(v: float) -> str:
    return float(np.float32(v)).hex() + "f"


if __name__ == "__main__":
    for kind, fn in (("sin", sin_coeffs), ("cos", cos_coeffs), ("exp", exp_coeffs)):
        c = fn()
        print(kind, [hexf(x) for x in c], "max rel err %.3g (ulp %.3g)" % (
            max_rel_error(kind, c), max_rel_error(kind, c) / 2.0 ** -24))
    # sin/cos fast path for |j| <= 128 (|x| <= 128 pi/2): 17-bit leading parts
    print("pi/2 split", [hexf(x) for x in split(mpmath.pi / 2, 17, 3)])
    print("2/pi", hexf(float(2 / mpmath.pi)))
    # exp: |k| <= 150 < 2^8: 16-bit leading part
    print("ln2 split", [hexf(x) for x in split(mpmath.log(2), 16, 2)])
    print("log2(e)", hexf(float(1 / mpmath.log(2))))
