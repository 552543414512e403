"""Pins of the closed-form MPC program (Eq. 8: a fixed number of solver
iterations written as one straight-line program) against the dense numpy
restatement in oracle/models.py and against the KKT conditions."""
import numpy as np
import pytest

from oracle import MODE_MIXED, Oracle
from oracle import models as M
from paper_2408_09662_gb300 import programs


def mpc_inputs(N, seed=0):
    """x0bar = hover (origin, at rest) + U(-0.5, 0.5) per state; waypoint U(-1, 1)^2."""
    rng = np.random.default_rng(seed)
    return np.vstack([rng.uniform(-0.5, 0.5, (6, N)), rng.uniform(-1, 1, (2, N))])


@pytest.fixture(scope="module")
def mpc():
    return programs.quadrotor_mpc().to_bytes()


def test_program_matches_dense_lapack_restatement(mpc):
    X = mpc_inputs(16, seed=1)
    y = Oracle(mpc).eval(X)
    for i in range(16):
        ref = M.quadrotor_mpc(X[:6, i], X[6:, i])
        np.testing.assert_allclose(y[:, i], ref, rtol=0, atol=1e-11 * np.max(np.abs(ref)))


def test_thrusts_stay_strictly_inside_bounds(mpc):
    X = mpc_inputs(64, seed=2)
    X[2] *= 2.0                                  # larger tilts push thrusts toward the bounds
    y = Oracle(mpc).eval(X)
    u = y[66:]
    assert np.all(u > 0) and np.all(u < 15)


def test_first_newton_step_solves_its_kkt_system():
    """The unrolled LDL^T solution s satisfies K s = rhs (K, rhs assembled densely
    at the initial guess) to a relative residual of 1e-10."""
    ir = programs.quadrotor_mpc({"M": 1}, debug_first_step=True).to_bytes()
    X = mpc_inputs(8, seed=3)
    S = Oracle(ir).eval(X)
    order = programs.kkt_order(10)
    p = dict(M.QUAD)
    Tn = p["T"]
    nx = 6 * (Tn + 1)
    for i in range(8):
        x0bar, wp = X[:6, i], X[6:, i]
        uh = p["mass"] * p["g"] / 2
        u = [np.array([uh, uh]) for _ in range(Tn)]
        x = [x0bar]
        for k in range(Tn):
            x.append(M.quad_step(x[k], u[k], p))
        K, rhs = M.quad_kkt(x, u, x0bar, wp, p["mu0"], p)
        # map the program's stage ordering onto (z, lambda) of the dense system
        idx = []
        for kind, k, c in order:
            idx.append(6 * k + c if kind == "x" else (nx + 2 * k + c if kind == "u" else
                                                      nx + 2 * Tn + 6 * k + c))
        s = np.zeros(len(order))
        s[idx] = S[:, i]
        res = np.linalg.norm(K @ s - rhs) / np.linalg.norm(rhs)
        assert res < 1e-10, res


def test_without_barrier_one_step_is_the_equality_constrained_qp():
    """mu = 0, delta = 0 and one iteration: the step solves min 1/2 dz'H dz + g'dz
    s.t. A dz = -c exactly; checked against the null-space solution (scipy)."""
    import scipy.linalg as sl
    X = mpc_inputs(4, seed=4)
    ir = programs.quadrotor_mpc({"M": 1, "mu0": 0.0, "mu_end": 0.0, "tau": 1e30,
                                 "delta": 0.0}).to_bytes()
    y = Oracle(ir).eval(X)
    p = dict(M.QUAD, mu0=0.0, delta=0.0)
    Tn = p["T"]
    nx, nz = 6 * (Tn + 1), 6 * (Tn + 1) + 2 * Tn
    for i in range(4):
        x0bar, wp = X[:6, i], X[6:, i]
        uh = p["mass"] * p["g"] / 2
        u = [np.array([uh, uh]) for _ in range(Tn)]
        x = [x0bar]
        for k in range(Tn):
            x.append(M.quad_step(x[k], u[k], p))
        K, rhs = M.quad_kkt(x, u, x0bar, wp, 0.0, p)
        H, A = K[:nz, :nz], K[nz:, :nz]
        g, c = -rhs[:nz], -rhs[nz:]
        # null-space method: dz = dz_p + Z w
        dz_p = np.linalg.lstsq(A, -c, rcond=None)[0]
        Z = sl.null_space(A)
        w = np.linalg.solve(Z.T @ H @ Z, -Z.T @ (g + H @ dz_p))
        dz = dz_p + Z @ w
        z0 = np.concatenate([np.concatenate(x), np.concatenate(u)])
        np.testing.assert_allclose(y[:, i], z0 + dz, rtol=0, atol=1e-10)


def test_mixed_precision_emulation_error_is_small(mpc):
    """FP32 bulk with FP64 pivots/divisions/barrier terms stays close to FP64."""
    X = mpc_inputs(32, seed=5)
    orc = Oracle(mpc)
    y64 = orc.eval(X)
    ym = orc.eval(X, mode=MODE_MIXED)
    scale = np.max(np.abs(y64), axis=1, keepdims=True)
    assert np.max(np.abs(ym - y64) / scale) < 1e-3


# ---------------------------------------------------------------------------
# the paper's own form (Eq. 9): quadratic penalty, growing mu, full steps;
# real-time-iteration warm start
# ---------------------------------------------------------------------------
def tight_inputs(N, seed):
    """Targets far away so the unconstrained thrusts leave [0, u_max]."""
    rng = np.random.default_rng(seed)
    X = np.vstack([rng.uniform(-0.5, 0.5, (6, N)), rng.uniform(-1, 1, (2, N))])
    X[6:] *= 6.0
    return X


def test_penalty_program_matches_dense_restatement():
    params = {"u_max": 12.0}
    ir = programs.quadrotor_mpc(params, constraint="penalty").to_bytes()
    X = tight_inputs(12, seed=6)
    y = Oracle(ir).eval(X)
    for i in range(12):
        ref = M.quadrotor_mpc(X[:6, i], X[6:, i], penalty=True, u_max=12.0)
        np.testing.assert_allclose(y[:, i], ref, rtol=0, atol=1e-10 * np.max(np.abs(ref)))


def test_penalty_violation_shrinks_as_mu_grows():
    """For large enough mu the penalised problem solves the constrained one
    (Eq. 9's justification): the worst bound violation falls with each
    iteration's tenfold larger mu."""
    X = tight_inputs(16, seed=7)
    viol = []
    for Mi in (2, 3, 4, 5):
        ir = programs.quadrotor_mpc({"u_max": 12.0, "M": Mi}, constraint="penalty").to_bytes()
        u = Oracle(ir).eval(X)[66:]
        viol.append(np.max(np.maximum(u - 12.0, 0) + np.maximum(-u, 0)))
    assert viol[0] > 0.05
    assert all(b < a for a, b in zip(viol, viol[1:]))
    assert viol[-1] < 0.05 * viol[0]


def test_warm_start_matches_dense_restatement_and_converges():
    """Real-time iteration: one Newton step from the previous solution.  From a
    converged solution the step barely moves it."""
    # one step at the final barrier weight, from the 8-iteration solution
    ir1 = programs.quadrotor_mpc({"M": 1, "mu0": 0.001}, warm_start=True).to_bytes()
    X = mpc_inputs(8, seed=8)
    z_full = np.stack([M.quadrotor_mpc(X[:6, i], X[6:, i], M=8) for i in range(8)], axis=1)
    y = Oracle(ir1).eval(np.vstack([X, z_full]))
    for i in range(8):
        ref = M.quadrotor_mpc(X[:6, i], X[6:, i], M=1, z_prev=z_full[:, i], mu0=0.001)
        np.testing.assert_allclose(y[:, i], ref, rtol=0, atol=1e-10 * np.max(np.abs(ref)))
    cold = Oracle(programs.quadrotor_mpc({"M": 1, "mu0": 0.001}).to_bytes()).eval(X)
    assert np.max(np.abs(y - z_full)) < 0.01 * np.max(np.abs(cold - z_full))


def test_closed_loop_step_matches_model():
    """The closed-loop step (Fig. 4's cost and constraint-violation axes) against
    the numpy model's step, a stage cost written out, and the bound violation
    at hand-picked thrusts (inside, above u_max, below 0)."""
    ir = programs.quadrotor_closed_loop_step().to_bytes()
    p = M.QUAD
    rng = np.random.default_rng(21)
    N = 6
    x = rng.uniform(-0.5, 0.5, (6, N))
    wp = rng.uniform(-1, 1, (2, N))
    z = rng.uniform(0, 1, (86, N))
    z[66:68] = np.array([[5.0, 16.5, -0.25, 4.9, 15.0, 0.0], [5.1, 3.0, 7.0, -2.0, 0.0, 14.0]])
    J, V = rng.uniform(0, 2, (1, N)), np.array([[0.0, 0.0, 0.0, 3.0, 0.0, 0.0]])
    y = Oracle(ir).eval(np.vstack([x, wp, z, J, V]))
    uh = p["mass"] * p["g"] / 2
    want_v = [0.0, 1.5, 0.25, 3.0, 0.0, 0.0]
    for i in range(N):
        u = z[66:68, i]
        xref = np.array([wp[0, i], wp[1, i], 0, 0, 0, 0])
        cost = J[0, i] + np.sum(np.array(p["q"]) * (x[:, i] - xref) ** 2) + p["r"] * np.sum((u - uh) ** 2)
        np.testing.assert_allclose(y[:6, i], M.quad_step(x[:, i], u, p), rtol=1e-14, atol=1e-15)
        assert abs(y[6, i] - cost) <= 1e-13 * cost
        assert y[7, i] == want_v[i]
