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
    """The example function of Fig. 2 (§III-A), y = (sin x + x)^2, as a two-slot
    work vector: slot 0 holds x, slot 1 holds sin x and then, reused in place,
    the sum and its square, which is the output."""
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
                 M=5, delta=1e-9, tau=0.995, penalty_mu0=10.0, penalty_growth=10.0)


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


def quadrotor_step_sparse_jacobian(params=None) -> ProgramIR:
    """x+ = step(x, u) of the planar quadrotor and its 6 x 8 Jacobian d x+ /
    d [x; u] by the tracer's forward mode, stored sparse: entries whose tangent
    is structurally zero are not in the output's CSR pattern (§II-A)."""
    p = dict(QUADROTOR)
    if params:
        p.update(params)
    g = T.Graph()
    x, u = g.symbols(6), g.symbols(2)
    xn = quadrotor_step(list(x), list(u), p)
    J = T.jacobian(xn, list(x) + list(u))
    mask = [[not (isinstance(v, float) and v == 0.0) for v in row] for row in J]
    vals = [v for row, mrow in zip(J, mask) for v, m in zip(row, mrow) if m]
    return T.Function([("x", x), ("u", u)],
                      [("x_next", xn), ("jac", vals, Sparsity.from_mask(mask))]).to_ir()


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


def quadrotor_mpc(params=None, mixed_tags: bool = True, debug_first_step: bool = False,
                  constraint: str = "barrier", warm_start: bool = False) -> ProgramIR:
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

    constraint = "penalty" is the paper's own form (Eq. 9): the bounds enter the
    cost as mu_i sum [max(0, u - u_max)^2 + max(0, -u)^2] with
    mu_i = penalty_mu0 * penalty_growth^i; its Gauss-Newton model uses the
    active set at the current iterate, and every step is taken in full.
    warm_start (real-time iteration, §V-A): an extra input z_prev (86) is the
    initial guess, with x_0 replaced by x0bar.
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
    if warm_start:
        zprev = g.symbols(6 * (Tn + 1) + 2 * Tn)
        x = [list(x0bar)] + [zprev[6 * k:6 * k + 6] for k in range(1, Tn + 1)]
        u = [zprev[6 * (Tn + 1) + 2 * k:6 * (Tn + 1) + 2 * k + 2] for k in range(Tn)]
    else:
        u = [[uh, uh] for _ in range(Tn)]
        x = [list(x0bar)]
        for k in range(Tn):
            x.append(quadrotor_step(x[k], u[k], p))
    order = kkt_order(Tn)
    pos = {e: i for i, e in enumerate(order)}
    n = len(order)
    first = None
    for it in range(M):
        if constraint == "penalty":
            mu = p["penalty_mu0"] * p["penalty_growth"] ** it
        else:
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
                if constraint == "penalty":
                    over, under = T.fmax(uk - umax, 0.0), T.fmax(-uk, 0.0)
                    active = T.logical_or(0.0 < over, 0.0 < under)
                    hb = 2.0 * mu * active
                    gb = 2.0 * mu * (under - over)      # minus the penalty gradient
                else:
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
        if constraint == "penalty":
            alpha = 1.0
        else:
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
    if warm_start:
        ins.append(("z_prev", zprev))
    if debug_first_step:
        return T.Function(ins, [("kkt_solution", first)]).to_ir()
    z = [v for k in range(Tn + 1) for v in x[k]] + [v for k in range(Tn) for v in u[k]]
    return T.Function(ins, [("z", z)]).to_ir()


def quadrotor_closed_loop_step(params=None) -> ProgramIR:
    """One closed-loop step of the planar quadrotor under the first input of an
    MPC solution, with the two quantities the paper plots against evaluation
    time for its MPC (§V-A, Fig. 4): accumulated cost and constraint violation.

    Inputs: x (6), waypoint (2), z (86, an MPC solution laid out as
    quadrotor_mpc's output: x_0..x_T then u_0..u_{T-1}), J (1), V (1).
    Outputs: x+ = step(x, u_0) (6), J+ = J + stage cost of (x, u_0) (the MPC's
    Q, R, x_ref and u_h), V+ = max(V, max_j max(0, u_0j - u_max, -u_0j)).
    """
    p = dict(QUADROTOR)
    if params:
        p.update(params)
    Tn = p["T"]
    g = T.Graph()
    x, wp, z, J, V = g.symbols(6), g.symbols(2), g.symbols(6 * (Tn + 1) + 2 * Tn), g.symbols(1), g.symbols(1)
    u = z[6 * (Tn + 1):6 * (Tn + 1) + 2]
    uh = p["mass"] * p["g"] / 2.0
    xref = [wp[0], wp[1], 0.0, 0.0, 0.0, 0.0]
    cost = J[0]
    for i in range(6):
        cost = cost + p["q"][i] * (x[i] - xref[i]) * (x[i] - xref[i])
    for j in range(2):
        cost = cost + p["r"] * (u[j] - uh) * (u[j] - uh)
    viol = V[0]
    for j in range(2):
        viol = T.fmax(viol, T.fmax(T.fmax(u[j] - p["u_max"], -u[j]), 0.0))
    xn = quadrotor_step(list(x), list(u), p)
    return T.Function([("x", x), ("waypoint", wp), ("z", z), ("J", J), ("V", V)],
                      [("x_next", xn), ("J_next", [cost]), ("V_next", [viol])]).to_ir()


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


# ---------------------------------------------------------------------------
# Quadcopter closed-loop step with an infinite-horizon LQR solved by a fixed
# number of structured-doubling iterations (§V-C)
# ---------------------------------------------------------------------------
LQR_PARAMS = ("u_max", "mass", "inertia", "q_px", "q_pz", "q_th", "q_vx", "q_vz", "q_om", "r")


def _mm(X, Y):
    """Product of traced matrices (lists of lists); structural zeros stay floats."""
    n, m, k = len(X), len(Y[0]), len(Y)
    out = []
    for i in range(n):
        row = []
        for j in range(m):
            acc = 0.0
            for l in range(k):
                a, b = X[i][l], Y[l][j]
                if (isinstance(a, float) and a == 0.0) or (isinstance(b, float) and b == 0.0):
                    continue
                acc = acc + a * b
            row.append(acc)
        out.append(row)
    return out


def _tr(X):
    return [list(r) for r in zip(*X)]


def _add(X, Y):
    return [[a + b for a, b in zip(r, s)] for r, s in zip(X, Y)]


def _lu_solve(W, Rhs):
    """Solve W Y = Rhs by Gaussian elimination without pivoting (W = I + G H
    with G, H positive semidefinite: its eigenvalues are >= 1)."""
    n = len(W)
    W = [list(r) for r in W]
    Y = [list(r) for r in Rhs]
    for j in range(n):
        for i in range(j + 1, n):
            if isinstance(W[i][j], float) and W[i][j] == 0.0:
                continue
            l = W[i][j] / W[j][j]
            for c in range(j + 1, n):
                W[i][c] = W[i][c] - l * W[j][c]
            Y[i] = [a - l * b for a, b in zip(Y[i], Y[j])]
    for j in reversed(range(n)):
        Y[j] = [a / W[j][j] for a in Y[j]]
        for i in range(j):
            if isinstance(W[i][j], float) and W[i][j] == 0.0:
                continue
            Y[i] = [a - W[i][j] * b for a, b in zip(Y[i], Y[j])]
    return Y


def sda_dare(A, B, Q, Rinv, iters):
    """Structured doubling for the DARE X = A'XA - A'XB(R + B'XB)^-1 B'XA + Q:
    A0 = A, G0 = B R^-1 B', H0 = Q; with W = I + G H,
    A+ = A W^-1 A, G+ = G + A W^-1 G A', H+ = H + A' H W^-1 A; H -> X
    quadratically.  A fixed number of iterations (no convergence test)."""
    n = len(A)
    G = _mm(_mm(B, Rinv), _tr(B))
    H = [list(r) for r in Q]
    Ak = [list(r) for r in A]
    I = [[1.0 if i == j else 0.0 for j in range(n)] for i in range(n)]
    for _ in range(iters):
        W = _add(I, _mm(G, H))
        Y = _lu_solve(W, [a + g for a, g in zip(Ak, G)])   # [W^-1 A | W^-1 G]
        YA = [r[:n] for r in Y]
        YG = [r[n:] for r in Y]
        A_next = _mm(Ak, YA)
        G = _add(G, _mm(_mm(Ak, YG), _tr(Ak)))
        H = _add(H, _mm(_mm(_tr(Ak), H), YA))
        Ak = A_next
    return H


def quadrotor_lqr_step(sda_iters: int = 12, debug_riccati: bool = False) -> ProgramIR:
    """z+ = step(z, clip(u_h - K z, 0, u_max)), K the infinite-horizon LQR gain of
    the hover linearisation, recomputed from the per-instance parameters
    theta = (u_max, mass, inertia, Q diagonal (6), r) with R = r I.
    debug_riccati: output the Riccati solution X (row-major) and K instead."""
    p = dict(QUADROTOR)
    g = T.Graph()
    z = g.symbols(6)
    th = g.symbols(len(LQR_PARAMS))
    prm = dict(zip(LQR_PARAMS, th))
    dt, grav, arm = p["dt"], p["g"], p["arm"]
    m, I = prm["mass"], prm["inertia"]
    # hover linearisation of the semi-implicit Euler step (theta = 0, F = m g)
    A = [[1.0 if i == j else 0.0 for j in range(6)] for i in range(6)]
    A[3][2] = -dt * grav
    A[0][2] = -dt * dt * grav
    A[0][3] = A[1][4] = A[2][5] = dt
    B = [[0.0, 0.0] for _ in range(6)]
    dvz = dt / m
    dom = dt * arm / I
    B[4] = [dvz, dvz]
    B[1] = [dt * dvz, dt * dvz]
    B[5] = [dom, -dom]
    B[2] = [dt * dom, -dt * dom]
    Q = [[prm[LQR_PARAMS[3 + i]] if i == j else 0.0 for j in range(6)] for i in range(6)]
    rinv = 1.0 / prm["r"]
    X = sda_dare(A, B, Q, [[rinv, 0.0], [0.0, rinv]], sda_iters)
    # K = (R + B'XB)^-1 B'XA
    BtX = _mm(_tr(B), X)
    S = _add([[prm["r"], 0.0], [0.0, prm["r"]]], _mm(BtX, B))
    det = S[0][0] * S[1][1] - S[0][1] * S[1][0]
    Sinv = [[S[1][1] / det, -S[0][1] / det], [-S[1][0] / det, S[0][0] / det]]
    K = _mm(Sinv, _mm(BtX, A))
    ins = [("z", z), ("theta", th)]
    if debug_riccati:
        return T.Function(ins, [("X", [X[i][j] for i in range(6) for j in range(6)]),
                                ("K", [K[i][j] for i in range(2) for j in range(6)])]).to_ir()
    uh = m * grav / 2.0
    u = []
    for i in range(2):
        v = uh - sum(K[i][j] * z[j] for j in range(6))
        u.append(T.fmin(T.fmax(v, 0.0), prm["u_max"]))
    pp = dict(p, mass=m, inertia=I)
    return T.Function(ins, [("z_next", quadrotor_step(z, u, pp))]).to_ir()


# ---------------------------------------------------------------------------
# §IV benchmark family: LDL^T solution of a symmetric positive definite system
# ---------------------------------------------------------------------------
def ldlt_spd_solve(n: int) -> ProgramIR:
    """x = A^-1 b for a dense SPD A (lower triangle row-major, n(n+1)/2 inputs)
    and b (n), by an unrolled LDL^T factorisation and two triangular solves.
    §IV benchmarks five such functions, each with about ten times the
    operations of the previous one (n = 5, 10, 22, 47, 100 here)."""
    g = T.Graph()
    low = g.symbols(n * (n + 1) // 2)
    b = g.symbols(n)
    K = [[0.0] * n for _ in range(n)]
    t = 0
    for i in range(n):
        for j in range(i + 1):
            K[i][j] = K[j][i] = low[t]
            t += 1
    x = ldlt_solve(K, list(b), g, tag_pivots=False)
    lower = Sparsity.from_mask([[j <= i for j in range(n)] for i in range(n)])
    return T.Function([("A", low, 0, lower), ("b", b)], [("x", x)]).to_ir()


LDLT_SIZES = (5, 10, 22, 47, 100)
