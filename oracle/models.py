"""Direct numpy restatements of the benchmark models (test infrastructure).

These do not trace anything and share no code with the program generators:
they restate each model from its definition, with derivatives derived by hand,
so that a generated program can be checked against them through the oracle.
"""
from __future__ import annotations

import math

import numpy as np


# ---------------------------------------------------------------------------
# cart-pole (frictionless cart, point-mass pole on a massless rod of length l,
# theta = 0 hanging down); state [x, th, xd, thd], input f
# ---------------------------------------------------------------------------
def cartpole_f(q, f, m_c=1.0, m_p=0.1, l=0.5, g=9.81):
    x, th, xd, thd = q
    s, c = np.sin(th), np.cos(th)
    D = m_c + m_p * s ** 2
    xdd = (f + m_p * s * (l * thd ** 2 + g * c)) / D
    thdd = (-f * c - m_p * l * thd ** 2 * c * s - (m_c + m_p) * g * s) / (l * D)
    return np.array([xd, thd, xdd, thdd])


def cartpole_jf(q, f, m_c=1.0, m_p=0.1, l=0.5, g=9.81):
    """4x5 Jacobian of the continuous dynamics w.r.t. [x, th, xd, thd, f], by hand."""
    _, th, _, w = q
    s, c = math.sin(th), math.cos(th)
    D = m_c + m_p * s * s
    dD = 2 * m_p * s * c
    Nx = f + m_p * s * l * w * w + m_p * g * s * c
    dNx = m_p * c * l * w * w + m_p * g * (c * c - s * s)
    Nt = -f * c - m_p * l * w * w * c * s - (m_c + m_p) * g * s
    dNt = f * s - m_p * l * w * w * (c * c - s * s) - (m_c + m_p) * g * c
    J = np.zeros((4, 5))
    J[0, 2] = 1.0
    J[1, 3] = 1.0
    J[2, 1] = (dNx * D - Nx * dD) / D ** 2
    J[2, 3] = 2 * m_p * s * l * w / D
    J[2, 4] = 1.0 / D
    J[3, 1] = (dNt * D - Nt * dD) / (l * D ** 2)
    J[3, 3] = -2 * m_p * l * w * c * s / (l * D)
    J[3, 4] = -c / (l * D)
    return J


def cartpole_rk4_with_jacobian(q, f, dt=0.01, **p):
    """RK4 step and d q+ / d [q; f], the stage Jacobians chained by hand."""
    q = np.asarray(q, dtype=np.float64)
    E = np.hstack([np.eye(4), np.zeros((4, 1))])   # d q / d z
    eu = np.array([[0, 0, 0, 0, 1.0]])              # d f / d z
    k1 = cartpole_f(q, f, **p)
    dk1 = cartpole_jf(q, f, **p) @ np.vstack([E, eu])
    q2 = q + 0.5 * dt * k1
    dq2 = E + 0.5 * dt * dk1
    k2 = cartpole_f(q2, f, **p)
    dk2 = cartpole_jf(q2, f, **p) @ np.vstack([dq2, eu])
    q3 = q + 0.5 * dt * k2
    dq3 = E + 0.5 * dt * dk2
    k3 = cartpole_f(q3, f, **p)
    dk3 = cartpole_jf(q3, f, **p) @ np.vstack([dq3, eu])
    q4 = q + dt * k3
    dq4 = E + dt * dk3
    k4 = cartpole_f(q4, f, **p)
    dk4 = cartpole_jf(q4, f, **p) @ np.vstack([dq4, eu])
    qn = q + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    Jn = E + dt / 6.0 * (dk1 + 2 * dk2 + 2 * dk3 + dk4)
    return qn, Jn


def cartpole_linearization(m_c=1.0, m_p=0.1, l=0.5, g=9.81):
    """A_c, B_c of the dynamics at the hanging equilibrium, in closed form."""
    A = np.array([[0, 0, 1, 0], [0, 0, 0, 1],
                  [0, m_p * g / m_c, 0, 0],
                  [0, -(m_c + m_p) * g / (l * m_c), 0, 0]], dtype=np.float64)
    B = np.array([[0], [0], [1 / m_c], [-1 / (l * m_c)]], dtype=np.float64)
    return A, B


def rk4_linear_maps(A, B, dt):
    """RK4 on x' = A x + B u with u held: x+ = T4(A dt) x + S4 B u where
    T4 = sum_{k<=4} (A dt)^k / k! and S4 = sum_{k=1..4} A^(k-1) dt^k / k!."""
    n = A.shape[0]
    T4 = np.zeros((n, n))
    S4 = np.zeros((n, n))
    P = np.eye(n)
    for k in range(0, 5):
        T4 += np.linalg.matrix_power(A * dt, k) / math.factorial(k)
        if k >= 1:
            S4 += np.linalg.matrix_power(A, k - 1) * dt ** k / math.factorial(k)
    return T4, S4 @ B


# ---------------------------------------------------------------------------
# pendulum: th'' = -(g/l) sin th; energy E = om^2 / 2 - (g/l) cos th
# ---------------------------------------------------------------------------
def pendulum_energy(th, om, g_over_l=9.81):
    return 0.5 * np.asarray(om) ** 2 - g_over_l * np.cos(th)


# ---------------------------------------------------------------------------
# closed-form MPC of the planar quadrotor (barrier Newton, M fixed iterations)
# restated densely: z = (x_0..x_T, u_0..u_{T-1}), KKT solved by LAPACK
# ---------------------------------------------------------------------------
QUAD = dict(mass=1.0, inertia=0.01, arm=0.2, g=9.81, dt=0.02, T=10,
            q=(10.0, 10.0, 1.0, 1.0, 1.0, 1.0), r=0.1, u_max=15.0, mu0=0.1, mu_end=0.001,
            M=5, delta=1e-9, tau=0.995, penalty_mu0=10.0, penalty_growth=10.0)


def quad_step(x, u, p):
    px, pz, th, vx, vz, om = x
    F = u[0] + u[1]
    vx1 = vx + p["dt"] * (-F * math.sin(th) / p["mass"])
    vz1 = vz + p["dt"] * (F * math.cos(th) / p["mass"] - p["g"])
    om1 = om + p["dt"] * (p["arm"] * (u[0] - u[1]) / p["inertia"])
    return np.array([px + p["dt"] * vx1, pz + p["dt"] * vz1, th + p["dt"] * om1, vx1, vz1, om1])


def quad_step_jac(x, u, p):
    """(A, B) = d step / d x, d step / d u, by hand."""
    th = x[2]
    F = u[0] + u[1]
    dt, m = p["dt"], p["mass"]
    s, c = math.sin(th), math.cos(th)
    B = np.zeros((6, 2))
    B[3, :] = -dt * s / m
    B[4, :] = dt * c / m
    B[5, :] = [dt * p["arm"] / p["inertia"], -dt * p["arm"] / p["inertia"]]
    B[0:3, :] = dt * B[3:6, :]
    A = np.eye(6)
    A[3, 2] = -dt * F * c / m
    A[4, 2] = -dt * F * s / m
    A[0, 3] = A[1, 4] = A[2, 5] = dt
    A[0, 2] = dt * A[3, 2]
    A[1, 2] = dt * A[4, 2]
    return A, B


def quad_kkt(x, u, x0bar, wp, mu, p, penalty=False):
    """KKT matrix and right-hand side at (x, u): unknowns (dz, lambda)."""
    Tn = p["T"]
    nx, nu = 6 * (Tn + 1), 2 * Tn
    nz, nl = nx + nu, 6 * (Tn + 1)
    Q = np.diag(p["q"])
    xref = np.array([wp[0], wp[1], 0, 0, 0, 0.0])
    uh = p["mass"] * p["g"] / 2
    H = np.zeros((nz, nz))
    g = np.zeros(nz)
    for k in range(Tn + 1):
        H[6 * k:6 * k + 6, 6 * k:6 * k + 6] = 2 * Q
        g[6 * k:6 * k + 6] = 2 * Q @ (x[k] - xref)
    for k in range(Tn):
        for j in range(2):
            a = nx + 2 * k + j
            if penalty:
                # quadratic penalty of the bound violation, active set at u
                over, under = max(u[k][j] - p["u_max"], 0.0), max(-u[k][j], 0.0)
                H[a, a] = 2 * p["r"] + (2 * mu if (over > 0 or under > 0) else 0.0)
                g[a] = 2 * p["r"] * (u[k][j] - uh) + 2 * mu * (over - under)
                continue
            lo, hi = 1 / u[k][j], 1 / (p["u_max"] - u[k][j])
            H[a, a] = 2 * p["r"] + mu * (lo * lo + hi * hi)
            g[a] = 2 * p["r"] * (u[k][j] - uh) - mu * (lo - hi)
    A = np.zeros((nl, nz))
    c = np.zeros(nl)
    A[0:6, 0:6] = np.eye(6)
    c[0:6] = x[0] - x0bar
    for k in range(Tn):
        Ak, Bk = quad_step_jac(x[k], u[k], p)
        r = 6 * (k + 1)
        A[r:r + 6, 6 * (k + 1):6 * (k + 2)] = np.eye(6)
        A[r:r + 6, 6 * k:6 * k + 6] = -Ak
        A[r:r + 6, nx + 2 * k:nx + 2 * k + 2] = -Bk
        c[r:r + 6] = x[k + 1] - quad_step(x[k], u[k], p)
    K = np.block([[H, A.T], [A, -p["delta"] * np.eye(nl)]])
    rhs = np.concatenate([-g, -c])
    return K, rhs


def quadrotor_mpc(x0bar, wp, M=None, penalty=False, z_prev=None, **over):
    """z after M Newton iterations (the reading documented with the program
    generator), with every KKT system solved densely by LAPACK.  penalty: the
    quadratic-penalty form with full steps; z_prev: warm start."""
    p = dict(QUAD)
    p.update(over)
    if M is not None:
        p["M"] = M
    Tn = p["T"]
    nx = 6 * (Tn + 1)
    uh = p["mass"] * p["g"] / 2
    if z_prev is not None:
        x = [np.asarray(x0bar, dtype=np.float64)] + [np.array(z_prev[6 * k:6 * k + 6]) for k in range(1, Tn + 1)]
        u = [np.array(z_prev[nx + 2 * k:nx + 2 * k + 2]) for k in range(Tn)]
    else:
        u = [np.array([uh, uh]) for _ in range(Tn)]
        x = [np.asarray(x0bar, dtype=np.float64)]
        for k in range(Tn):
            x.append(quad_step(x[k], u[k], p))
    for it in range(p["M"]):
        if penalty:
            mu = p["penalty_mu0"] * p["penalty_growth"] ** it
        else:
            mu = p["mu0"] * (p["mu_end"] / p["mu0"]) ** (it / (p["M"] - 1)) if p["M"] > 1 else p["mu0"]
        K, rhs = quad_kkt(x, u, x0bar, wp, mu, p, penalty=penalty)
        s = np.linalg.solve(K, rhs)
        du = s[nx:nx + 2 * Tn].reshape(Tn, 2)
        dx = s[:nx].reshape(Tn + 1, 6)
        U = np.array(u)
        with np.errstate(divide="ignore"):
            lo = np.where(du < 0, U / np.maximum(-du, 0), np.inf)
            hi = np.where(du > 0, (p["u_max"] - U) / np.maximum(du, 0), np.inf)
        alpha = 1.0 if penalty else min(1.0, p["tau"] * float(np.min(np.minimum(lo, hi))))
        x = [x[k] + alpha * dx[k] for k in range(Tn + 1)]
        u = [u[k] + alpha * du[k] for k in range(Tn)]
    return np.concatenate([np.concatenate(x), np.concatenate(u)])


# ---------------------------------------------------------------------------
# single-rigid-body quadruped under u = u_grav - K x, RK4, running loss
# (vectorised over instances: arrays [12, N])
# ---------------------------------------------------------------------------
SRB = dict(mass=12.0, inertia=(0.07, 0.26, 0.28), g=9.81, dt=0.005,
           feet=((0.2, 0.15, -0.3), (0.2, -0.15, -0.3), (-0.2, 0.15, -0.3), (-0.2, -0.15, -0.3)))


def _rz_ry_rx(phi, th, psi):
    """[3, 3, N] rotation Rz(psi) @ Ry(th) @ Rx(phi), built from the factors."""
    N = np.shape(phi)[0]
    one, zero = np.ones(N), np.zeros(N)
    Rx = np.array([[one, zero, zero], [zero, np.cos(phi), -np.sin(phi)], [zero, np.sin(phi), np.cos(phi)]])
    Ry = np.array([[np.cos(th), zero, np.sin(th)], [zero, one, zero], [-np.sin(th), zero, np.cos(th)]])
    Rz = np.array([[np.cos(psi), -np.sin(psi), zero], [np.sin(psi), np.cos(psi), zero], [zero, zero, one]])
    return np.einsum("abn,bcn,cdn->adn", Rz, Ry, Rx)


def srb_f(x, u, p=SRB):
    pos, ang, v, w = x[0:3], x[3:6], x[6:9], x[9:12]
    R = _rz_ry_rx(ang[0], ang[1], ang[2])
    Ib = np.array(p["inertia"])
    Iw = np.einsum("akn,k,bkn->abn", R, Ib, R)
    F = np.zeros_like(v)
    tau = np.zeros_like(v)
    for i, foot in enumerate(p["feet"]):
        r = np.einsum("akn,k->an", R, np.array(foot))
        f = u[3 * i:3 * i + 3]
        F = F + f
        tau = tau + np.cross(r, f, axis=0)
    Iww = np.einsum("abn,bn->an", Iw, w)
    rhs = tau - np.cross(w, Iww, axis=0)
    wd = np.stack([np.linalg.solve(Iw[:, :, n], rhs[:, n]) for n in range(x.shape[1])], axis=1)
    vd = F / p["mass"] - np.array([0, 0, p["g"]])[:, None]
    phi, th, psi = ang
    # world angular velocity = E(Theta) dTheta/dt for ZYX angles; invert E
    E = np.array([[np.cos(psi) * np.cos(th), -np.sin(psi), np.zeros_like(psi)],
                  [np.sin(psi) * np.cos(th), np.cos(psi), np.zeros_like(psi)],
                  [-np.sin(th), np.zeros_like(psi), np.ones_like(psi)]])
    angd = np.stack([np.linalg.solve(E[:, :, n], w[:, n]) for n in range(x.shape[1])], axis=1)
    return np.vstack([v, angd, vd, wd])


def srb_rollout_loss(x0, K, steps=50, p=SRB):
    """sum over instances and t = 1..steps of ||x_t||^2, u = u_grav - K x held per RK4 step.
    Complex inputs are carried through unchanged (every step is analytic), which
    gives complex-step derivatives: d L / d K_ab = Im L(K + i h e_ab) / h."""
    x = np.array(x0, dtype=np.result_type(x0, K, np.float64))
    ug = np.zeros((12, 1))
    ug[2::3] = p["mass"] * p["g"] / 4
    total = 0.0
    dt = p["dt"]
    for _ in range(steps):
        u = ug - K @ x
        k1 = srb_f(x, u, p)
        k2 = srb_f(x + 0.5 * dt * k1, u, p)
        k3 = srb_f(x + 0.5 * dt * k2, u, p)
        k4 = srb_f(x + dt * k3, u, p)
        x = x + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        total = total + np.sum(x * x)
    return total, x


# ---------------------------------------------------------------------------
# quadcopter LQR closed-loop step (infinite horizon, DARE by scipy)
# ---------------------------------------------------------------------------
def quad_hover_AB(mass, inertia, p=QUAD):
    """Linearisation of the semi-implicit Euler step at hover (theta = 0, F = m g)."""
    dt, g, arm = p["dt"], p["g"], p["arm"]
    A = np.eye(6)
    A[0, 3] = A[1, 4] = A[2, 5] = dt
    A[3, 2] = -dt * g
    A[0, 2] = dt * A[3, 2]
    B = np.zeros((6, 2))
    B[4, :] = dt / mass
    B[5, :] = [dt * arm / inertia, -dt * arm / inertia]
    B[0:3, :] = dt * B[3:6, :]
    return A, B


def quad_lqr_step(z, theta, p=QUAD):
    """theta = (u_max, mass, inertia, q (6), r); returns (z_next, X, K)."""
    import scipy.linalg as sl
    u_max, mass, inertia = theta[0], theta[1], theta[2]
    Q, R = np.diag(theta[3:9]), theta[9] * np.eye(2)
    A, B = quad_hover_AB(mass, inertia, p)
    X = sl.solve_discrete_are(A, B, Q, R)
    K = np.linalg.solve(R + B.T @ X @ B, B.T @ X @ A)
    u = np.clip(mass * p["g"] / 2 - K @ z, 0.0, u_max)
    pp = dict(p, mass=mass, inertia=inertia)
    return quad_step(z, u, pp), X, K
