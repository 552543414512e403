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


# ---------------------------------------------------------------------------
# Closed-form MPC: planar quadrotor, M unrolled barrier-Newton iterations
# ---------------------------------------------------------------------------
QUADROTOR = dict(mass=1.0, inertia=0.01, arm=0.2, g=9.81, dt=0.02, T=10,
                 q=(10.0, 10.0, 1.0, 1.0, 1.0, 1.0), r=0.1, u_max=15.0, mu0=0.1, mu_end=0.001,
                 M=5, delta=1e-9, tau=0.995)


def quadrotor_step(x, u, p):
    """Semi-implicit Euler step of the planar quadrotor (§V-C integrates its
    quadcopter this way): x = [px, pz, th, vx, vz, om], u = [u1, u2] thrusts."""
    px, pz, th, vx, vz, om = x
    u1, u2 = u
    thrust = u1 + u2
    ax = -thrust * T.sin(th) / p["mass"]
    az = thrust * T.cos(th) / p["mass"] - p["g"]
    al = p["arm"] * (u1 - u2) / p["inertia"]
    dt = p["dt"]
    vx1, vz1, om1 = vx + dt * ax, vz + dt * az, om + dt * al
    return [px + dt * vx1, pz + dt * vz1, th + dt * om1, vx1, vz1, om1]


def quadrotor_step_jacobian(x, u, p):
    """6x8 Jacobian of quadrotor_step w.r.t. [x; u], derived by hand; structural
    zeros are the float 0.0."""
    th = x[2]
    dt, m, arm, I = p["dt"], p["mass"], p["arm"], p["inertia"]
    s, c = T.sin(th), T.cos(th)
    thrust = u[0] + u[1]
    J = [[0.0] * 8 for _ in range(6)]
    # velocities
    dvx_dth = -dt * thrust * c / m
    dvz_dth = -dt * thrust * s / m
    dvx_du = -dt * s / m
    dvz_du = dt * c / m
    dom_du = (dt * arm / I, -dt * arm / I)
    J[3][3] = 1.0
    J[3][2] = dvx_dth
    J[4][4] = 1.0
    J[4][2] = dvz_dth
    J[5][5] = 1.0
    for j in range(2):
        J[3][6 + j] = dvx_du
        J[4][6 + j] = dvz_du
        J[5][6 + j] = dom_du[j]
    # positions and angle: p+ = p + dt * v+
    J[0][0] = 1.0
    J[0][2] = dt * dvx_dth
    J[0][3] = dt
    J[1][1] = 1.0
    J[1][2] = dt * dvz_dth
    J[1][4] = dt
    J[2][2] = 1.0
    J[2][5] = dt
    for j in range(2):
        J[0][6 + j] = dt * dvx_du
        J[1][6 + j] = dt * dvz_du
        J[2][6 + j] = dt * dom_du[j]
    return J


def kkt_order(Tn: int):
    """Stage ordering of the KKT unknowns: x0, lam0, then per stage k:
    u_k, x_{k+1}, lam_{k+1}.  Entries are (kind, stage, component).

    Every state block is eliminated before the multipliers of the constraint
    that defines it, so each multiplier pivot block picks up -(2Q)^-1 and stays
    well away from zero (placing lam_{k+1} before x_{k+1} instead leaves pivots
    of size delta, i.e. element growth of 1/delta)."""
    order = [("x", 0, i) for i in range(6)] + [("l", 0, i) for i in range(6)]
    for k in range(Tn):
        order += [("u", k, j) for j in range(2)]
        order += [("x", k + 1, i) for i in range(6)]
        order += [("l", k + 1, i) for i in range(6)]
    return order


def ldlt_solve(K, rhs, g, tag_pivots: bool):
    """Solve K s = rhs by an unrolled LDL^T factorisation without pivoting.

    K is a dense list-of-lists whose structural zeros are the float 0.0; the
    tracer drops every product with a structural zero, so only the fill that
    the ordering creates is ever computed.  Pivots, and every division by a
    pivot, are tagged FP64 when tag_pivots (mixed precision)."""
    from contextlib import nullcontext
    n = len(K)
    f64 = g.fp64 if tag_pivots else nullcontext
    L = [dict() for _ in range(n)]       # L[i][k], k < i, non-zeros only
    d = [None] * n
    cols = [set() for _ in range(n)]     # rows i > j with L[i][j] != 0
    for j in range(n):
        v = {k: L[j][k] * d[k] for k in L[j]}
        with f64():
            dj = K[j][j]
            for k in sorted(L[j]):
                dj = dj - L[j][k] * v[k]
            d[j] = dj
        # candidate rows: structural non-zeros of column j, plus fill from shared k
        rows = {i for i in range(j + 1, n) if not (isinstance(K[i][j], float) and K[i][j] == 0.0)}
        for k in L[j]:
            rows |= {i for i in cols[k] if i > j}
        for i in sorted(rows):
            s = K[i][j]
            for k in sorted(L[i].keys() & L[j].keys()):
                s = s - L[i][k] * v[k]
            if isinstance(s, float) and s == 0.0:
                continue
            with f64():
                L[i][j] = s / d[j]
            cols[j].add(i)
    y = [None] * n
    for i in range(n):
        acc = rhs[i]
        for k in sorted(L[i]):
            acc = acc - L[i][k] * y[k]
        y[i] = acc
    with f64():
        w = [y[i] / d[i] for i in range(n)]
    s = [None] * n
    for i in reversed(range(n)):
        acc = w[i]
        for r in sorted(cols[i]):
            acc = acc - L[r][i] * s[r]
        s[i] = acc
    return s


def quadrotor_mpc(params=None, mixed_tags: bool = True, debug_first_step: bool = False) -> ProgramIR:
    """Closed-form MPC (Eq. 8: M fixed solver iterations, no branches).

    Problem: states x_0..x_T, thrusts u_0..u_{T-1} of the planar quadrotor,
    x_0 = x0bar, x_{k+1} = step(x_k, u_k); cost sum_k (x_k - x_ref)' Q (x_k - x_ref)
    + sum_k (u_k - u_h)' R (u_k - u_h), u_h = m g / 2, x_ref = (wx, wz, 0, 0, 0, 0);
    thrust bounds 0 < u < u_max by the log barrier -mu sum [log u + log(u_max - u)].
    Iteration i (mu_i = mu0 (mu_end / mu0)^(i / (M-1))): Gauss-Newton Hessian
    (cost + barrier, dynamics curvature dropped), linearised constraints, KKT
    system [[H, A'], [A, -delta I]] solved by ldlt_solve in the stage ordering,
    step length alpha = min(1, tau * fraction-to-boundary), z += alpha dz.
    Initial guess: u = u_h and the rollout of u_h from x0bar.
    Inputs: x0bar (6), waypoint (2).  Output: z = (x_0..x_T, u_0..u_{T-1}).
    debug_first_step: output the first KKT solution (in kkt_order) instead.
    """
    from contextlib import nullcontext
    p = dict(QUADROTOR)
    if params:
        p.update(params)
    Tn, M = p["T"], p["M"]
    g = T.Graph()
    x0bar = g.symbols(6)
    wp = g.symbols(2)
    uh = p["mass"] * p["g"] / 2.0
    umax = p["u_max"]
    f64 = g.fp64 if mixed_tags else nullcontext
    xref = [wp[0], wp[1], 0.0, 0.0, 0.0, 0.0]
    u = [[uh, uh] for _ in range(Tn)]
    x = [list(x0bar)]
    for k in range(Tn):
        x.append(quadrotor_step(x[k], u[k], p))
    order = kkt_order(Tn)
    pos = {e: i for i, e in enumerate(order)}
    n = len(order)
    first = None
    for it in range(M):
        mu = p["mu0"] * (p["mu_end"] / p["mu0"]) ** (it / (M - 1)) if M > 1 else p["mu0"]
        K = [[0.0] * n for _ in range(n)]
        rhs = [0.0] * n
        for k in range(Tn + 1):
            for i in range(6):
                a = pos[("x", k, i)]
                K[a][a] = 2.0 * p["q"][i]
                rhs[a] = -2.0 * p["q"][i] * (x[k][i] - xref[i])
        for k in range(Tn):
            for j in range(2):
                a = pos[("u", k, j)]
                uk = u[k][j]
                with f64():
                    inv_lo = 1.0 / uk
                    inv_hi = 1.0 / (umax - uk)
                    hb = mu * (inv_lo * inv_lo + inv_hi * inv_hi)
                    gb = mu * (inv_lo - inv_hi)
                K[a][a] = 2.0 * p["r"] + hb
                rhs[a] = -(2.0 * p["r"] * (uk - uh) - gb)
        # constraints: lam0 -> x0 - x0bar;  lam_{k+1} -> x_{k+1} - step(x_k, u_k)
        for i in range(6):
            li, xi = pos[("l", 0, i)], pos[("x", 0, i)]
            K[li][xi] = K[xi][li] = 1.0
            K[li][li] = -p["delta"]
            rhs[li] = -(x[0][i] - x0bar[i])
        for k in range(Tn):
            fk = quadrotor_step(x[k], u[k], p)
            J = quadrotor_step_jacobian(x[k], u[k], p)
            for i in range(6):
                li = pos[("l", k + 1, i)]
                K[li][li] = -p["delta"]
                xn = pos[("x", k + 1, i)]
                K[li][xn] = K[xn][li] = 1.0
                for j in range(8):
                    col = pos[("x", k, j)] if j < 6 else pos[("u", k, j - 6)]
                    dv = J[i][j]
                    if isinstance(dv, float) and dv == 0.0:
                        continue
                    K[li][col] = K[col][li] = -dv
                rhs[li] = -(x[k + 1][i] - fk[i])
        s = ldlt_solve(K, rhs, g, mixed_tags)
        if it == 0:
            first = s
            if debug_first_step:
                break
        dx = [[s[pos[("x", k, i)]] for i in range(6)] for k in range(Tn + 1)]
        du = [[s[pos[("u", k, j)]] for j in range(2)] for k in range(Tn)]
        # fraction to the boundary of 0 < u < u_max, branch-free
        ratio = None
        for k in range(Tn):
            for j in range(2):
                lo = u[k][j] / T.fmax(-du[k][j], 0.0)
                hi = (umax - u[k][j]) / T.fmax(du[k][j], 0.0)
                r = T.fmin(lo, hi)
                ratio = r if ratio is None else T.fmin(ratio, r)
        alpha = T.fmin(1.0, p["tau"] * ratio)
        x = [[x[k][i] + alpha * dx[k][i] for i in range(6)] for k in range(Tn + 1)]
        u = [[u[k][j] + alpha * du[k][j] for j in range(2)] for k in range(Tn)]
    ins = [("x0", x0bar), ("waypoint", wp)]
    if debug_first_step:
        return T.Function(ins, [("kkt_solution", first)]).to_ir()
    z = [v for k in range(Tn + 1) for v in x[k]] + [v for k in range(Tn) for v in u[k]]
    return T.Function(ins, [("z", z)]).to_ir()


# ---------------------------------------------------------------------------
# Differentiable rollout: single-rigid-body quadruped under linear feedback
# ---------------------------------------------------------------------------
SRB = dict(mass=12.0, inertia=(0.07, 0.26, 0.28), g=9.81, dt=0.005,
           feet=((0.2, 0.15, -0.3), (0.2, -0.15, -0.3), (-0.2, 0.15, -0.3), (-0.2, -0.15, -0.3)))


def _rot_zyx(phi, th, psi):
    """R = Rz(psi) Ry(th) Rx(phi) (body -> world)."""
    cf, sf = T.cos(phi), T.sin(phi)
    ct, st = T.cos(th), T.sin(th)
    cp, sp = T.cos(psi), T.sin(psi)
    return [[cp * ct, cp * st * sf - sp * cf, cp * st * cf + sp * sf],
            [sp * ct, sp * st * sf + cp * cf, sp * st * cf - cp * sf],
            [-st, ct * sf, ct * cf]]


def srb_dynamics(x, u, p):
    """State [p(3), Theta(3) = roll, pitch, yaw (ZYX), v(3), omega(3)], world-frame
    velocities; u = four world-frame foot forces at body-fixed feet."""
    pos, ang, v, w = x[0:3], x[3:6], x[6:9], x[9:12]
    R = _rot_zyx(*ang)
    Ib = p["inertia"]
    # I_w^-1 = R Ib^-1 R'
    Iinv = [[sum(R[a][k] * R[b][k] / Ib[k] for k in range(3)) for b in range(3)] for a in range(3)]
    Iw = [[sum(R[a][k] * R[b][k] * Ib[k] for k in range(3)) for b in range(3)] for a in range(3)]
    F = [0.0, 0.0, 0.0]
    tau = [0.0, 0.0, 0.0]
    for i, foot in enumerate(p["feet"]):
        r = [sum(R[a][k] * foot[k] for k in range(3)) for a in range(3)]
        f = u[3 * i:3 * i + 3]
        F = [F[a] + f[a] for a in range(3)]
        tau = [tau[0] + r[1] * f[2] - r[2] * f[1], tau[1] + r[2] * f[0] - r[0] * f[2],
               tau[2] + r[0] * f[1] - r[1] * f[0]]
    Iww = [sum(Iw[a][b] * w[b] for b in range(3)) for a in range(3)]
    gyro = [w[1] * Iww[2] - w[2] * Iww[1], w[2] * Iww[0] - w[0] * Iww[2], w[0] * Iww[1] - w[1] * Iww[0]]
    rhs = [tau[a] - gyro[a] for a in range(3)]
    wd = [sum(Iinv[a][b] * rhs[b] for b in range(3)) for a in range(3)]
    vd = [F[0] / p["mass"], F[1] / p["mass"], F[2] / p["mass"] - p["g"]]
    phi, th, psi = ang
    cp, sp, ct, st = T.cos(psi), T.sin(psi), T.cos(th), T.sin(th)
    a = (cp * w[0] + sp * w[1]) / ct
    angd = [a, -sp * w[0] + cp * w[1], w[2] + st * a]
    return list(v) + angd + vd + wd


def srb_step(params=None) -> ProgramIR:
    """One RK4 step (dt, force held) of the SRB under u = u_grav - K x, plus the
    running loss.  Inputs: K (144, broadcast: one gain shared by all instances,
    row-major 12x12), x (12), L (1).  Outputs: x+ (12), L + ||x+||^2 (1).
    Output rows line up with input rows 144..156, so a rollout can ping-pong
    two buffers without copies."""
    from .ir import ARG_BROADCAST
    p = dict(SRB)
    if params:
        p.update(params)
    g = T.Graph()
    K = g.symbols(144)
    x = g.symbols(12)
    (L,) = g.symbols(1)
    ug = p["mass"] * p["g"] / 4.0
    u = [(ug if j % 3 == 2 else 0.0) - sum(K[12 * j + k] * x[k] for k in range(12))
         for j in range(12)]
    xn = rk4_step(lambda s, uu: srb_dynamics(s, uu, p), x, u, p["dt"])
    Ln = L + sum(v * v for v in xn)
    return T.Function([("K", K, ARG_BROADCAST), ("x", x), ("L", [L])],
                      [("x_next", xn), ("L_next", [Ln])]).to_ir()
