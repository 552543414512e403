"""Program generators for the benchmark workloads (each returns a ProgramIR).

These build the straight-line programs that the engine evaluates; they are the
*inputs* of the method, traced with ``tracer``.  The paper publishes none of its
models, so every model below is the reading stated in its docstring.
"""
from __future__ import annotations

import numpy as np

from . import tracer as T
from .ir import Instr, Op, ProgramIR, Sparsity


# ---------------------------------------------------------------------------
# Listing 2 / Fig. 2: y = (sin x + x)^2, with in-place slot reuse
# ---------------------------------------------------------------------------
def listing2() -> ProgramIR:
    """The example function of Fig. 2 exactly as Listing 2 evaluates it:
    w0 = x; w1 = sin(w0); w1 = w1 + w0; w1 = w1 * w1; y = w1."""
    ins = [Instr(Op.INPUT, 0, 0), Instr(Op.SIN, 1, 0), Instr(Op.ADD, 1, 1, 0),
           Instr(Op.MUL, 1, 1, 1), Instr(Op.OUTPUT, 0, 1)]
    return ProgramIR(2, [Sparsity.dense(1, 1, "x")], [Sparsity.dense(1, 1, "y")], ins, [])


def single_op(op: Op, consts=(0.75,)) -> ProgramIR:
    """One elementary op on inputs x (and y): out = op(x[, y]).  FMA_CONST uses
    consts[0] as its literal."""
    from .ir import BINARY
    binary = op in BINARY or op == Op.FMA_CONST
    ins = [Instr(Op.INPUT, 0, 0)]
    n_in = 1
    if binary:
        ins.append(Instr(Op.INPUT, 1, 1))
        n_in = 2
    if op == Op.FMA_CONST:
        ins.append(Instr(Op.FMA_CONST, 2, 0, 1, 0))
        k = [float(consts[0])]
    else:
        ins.append(Instr(op, 2, 0, 1 if binary else 0))
        k = []
    ins.append(Instr(Op.OUTPUT, 0, 2))
    return ProgramIR(3, [Sparsity.dense(n_in, 1, "x")], [Sparsity.dense(1, 1, "y")], ins, k)


# ---------------------------------------------------------------------------
# RK4 helpers
# ---------------------------------------------------------------------------
def rk4_step(f, x, u, dt):
    """Classic 4-stage Runge-Kutta step with u held over the step."""
    k1 = f(x, u)
    k2 = f([xi + 0.5 * dt * ki for xi, ki in zip(x, k1)], u)
    k3 = f([xi + 0.5 * dt * ki for xi, ki in zip(x, k2)], u)
    k4 = f([xi + dt * ki for xi, ki in zip(x, k3)], u)
    return [xi + (dt / 6.0) * (a + 2.0 * b + 2.0 * c + d)
            for xi, a, b, c, d in zip(x, k1, k2, k3, k4)]


# ---------------------------------------------------------------------------
# Cart-pole: one RK4 step plus its 4x5 Jacobian
# ---------------------------------------------------------------------------
CARTPOLE = dict(m_c=1.0, m_p=0.1, l=0.5, g=9.81, dt=0.01)


def cartpole_dynamics(q, f, m_c=1.0, m_p=0.1, l=0.5, g=9.81):
    """Frictionless cart with a point-mass pole on a massless rod of length l;
    q = [x, th, xd, thd], th = 0 hanging straight down, f the cart force."""
    x, th, xd, thd = q
    s, c = T.sin(th), T.cos(th)
    den = m_c + m_p * s * s
    xdd = (f + m_p * s * (l * thd * thd + g * c)) / den
    thdd = (-f * c - m_p * l * thd * thd * c * s - (m_c + m_p) * g * s) / (l * den)
    return [xd, thd, xdd, thdd]


def cartpole_rk4(params=None) -> ProgramIR:
    """Inputs q (4) and f (1); outputs q+ (4) and the dense 4x5 Jacobian
    d q+ / d [q; f] (row-major non-zeros), traced by forward-mode AD."""
    p = dict(CARTPOLE)
    if params:
        p.update(params)
    g = T.Graph()
    q = g.symbols(4)
    (f,) = g.symbols(1)
    dyn = lambda x, u: cartpole_dynamics(x, u[0], p["m_c"], p["m_p"], p["l"], p["g"])
    qn = rk4_step(dyn, q, [f], p["dt"])
    J = T.jacobian(qn, q + [f])
    jvals = [J[r][c] for r in range(4) for c in range(5)]
    fn = T.Function([("q", q), ("f", [f])],
                    [("q_next", qn), ("jac", jvals, Sparsity.dense(4, 5))])
    return fn.to_ir()


# ---------------------------------------------------------------------------
# Pendulum and linear oscillator: RK4 over a fixed number of steps
# ---------------------------------------------------------------------------
def pendulum_rk4(steps: int, dt: float, g_over_l: float = 9.81) -> ProgramIR:
    """Frictionless pendulum th'' = -(g/l) sin th, `steps` RK4 steps of size dt.
    Inputs [th, om]; outputs [th, om] after the rollout."""
    g = T.Graph()
    x = g.symbols(2)
    f = lambda s, u: [s[1], -g_over_l * T.sin(s[0])]
    y = list(x)
    for _ in range(steps):
        y = rk4_step(f, y, [], dt)
    return T.Function([("x0", x)], [("xT", y)]).to_ir()


def oscillator_rk4(omega: float, dt: float) -> ProgramIR:
    """Linear oscillator x'' = -omega^2 x: one RK4 step, inputs [x, v]."""
    g = T.Graph()
    x = g.symbols(2)
    f = lambda s, u: [s[1], -(omega * omega) * s[0]]
    return T.Function([("x", x)], [("x_next", rk4_step(f, x, [], dt))]).to_ir()


# ---------------------------------------------------------------------------
# Seeded random straight-line program
# ---------------------------------------------------------------------------
RANDOM_MIX = (("add", 0.15), ("sub", 0.15), ("mul", 0.30), ("div", 0.05),
              ("sin", 0.05), ("cos", 0.05), ("gauss", 0.10), ("sqrt1p", 0.05),
              ("fma", 0.10))


def random_program(n_ops: int = 20000, n_in: int = 64, n_out: int = 32,
                   seed: int = 0, p_reuse: float = 0.01) -> ProgramIR:
    """Random program with the stated op mix, bounded so that it cannot overflow.

    Each of the n_ops draws appends one value.  Operands lie at a distance
    d ~ Geometric(p_reuse) behind the end of the value list (uniform over the
    list when d exceeds it).  Compound draws: div = a / (1 + b^2),
    sqrt1p = sqrt(1 + a^2), gauss = exp(-a^2), fma = c*a + b with c ~ U(-1, 1).
    The second factor of a mul is drawn, at geometric distance, from the values
    produced by sin, cos and gauss only (|.| <= 1), so products never grow.
    The outputs are the last n_out values.  Generator: numpy PCG64(seed).
    """
    rng = np.random.default_rng(seed)
    names = [k for k, _ in RANDOM_MIX]
    probs = np.array([p for _, p in RANDOM_MIX])
    kinds = rng.choice(len(names), size=n_ops, p=probs / probs.sum())
    g = T.Graph()
    x = g.symbols(n_in)
    vals = list(x)
    bounded = []

    def pick(lst):
        d = int(rng.geometric(p_reuse))
        L = len(lst)
        return lst[L - d] if d <= L else lst[int(rng.integers(L))]

    for kind in kinds:
        k = names[kind]
        a = pick(vals)
        if k == "add":
            v = a + pick(vals)
        elif k == "sub":
            v = a - pick(vals)
        elif k == "mul":
            v = a * (pick(bounded) if bounded else 0.5)
        elif k == "div":
            v = a / (1.0 + T.sq(pick(vals)))
        elif k == "sin":
            v = T.sin(a)
            bounded.append(v)
        elif k == "cos":
            v = T.cos(a)
            bounded.append(v)
        elif k == "gauss":
            v = T.exp(-T.sq(a))
            bounded.append(v)
        elif k == "sqrt1p":
            v = T.sqrt(1.0 + T.sq(a))
        else:
            v = T.fma_const(float(rng.uniform(-1.0, 1.0)), a, pick(vals))
        vals.append(v)
    return T.Function([("x", x)], [("y", vals[-n_out:])]).to_ir()
