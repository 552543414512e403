"""Pins of the quadcopter LQR closed-loop step (§V-C): the fixed-iteration
structured-doubling solution of the DARE against scipy's solver, and the
closed-loop step against a numpy restatement."""
import numpy as np
import pytest

from oracle import Oracle
from oracle import models as M
from paper_2408_09662_gb300 import programs


def lqr_inputs(N, seed=0):
    rng = np.random.default_rng(seed)
    z = rng.uniform(-0.5, 0.5, (6, N))
    theta = np.vstack([rng.uniform(10, 20, (1, N)), rng.uniform(0.8, 1.2, (1, N)),
                       rng.uniform(0.008, 0.012, (1, N)), rng.uniform(0.5, 10, (6, N)),
                       rng.uniform(0.05, 0.5, (1, N))])
    return np.vstack([z, theta])


def test_sda_matches_scipy_dare():
    ir = programs.quadrotor_lqr_step(debug_riccati=True).to_bytes()
    X = lqr_inputs(12, seed=1)
    y = Oracle(ir).eval(X)
    for i in range(12):
        _, Xr, Kr = M.quad_lqr_step(X[:6, i], X[6:, i])
        np.testing.assert_allclose(y[:36, i].reshape(6, 6), Xr, rtol=1e-8, atol=1e-8 * np.abs(Xr).max())
        np.testing.assert_allclose(y[36:, i].reshape(2, 6), Kr, rtol=1e-8, atol=1e-8 * np.abs(Kr).max())


def test_sda_converges_quadratically():
    """Doubling: the error of H_k roughly squares per iteration, so a few more
    iterations than needed change nothing while too few leave a visible error."""
    X = lqr_inputs(4, seed=2)
    errs = []
    for it in (3, 5, 12):
        y = Oracle(programs.quadrotor_lqr_step(sda_iters=it, debug_riccati=True).to_bytes()).eval(X)
        e = 0.0
        for i in range(4):
            Xr = M.quad_lqr_step(X[:6, i], X[6:, i])[1]
            e = max(e, np.abs(y[:36, i].reshape(6, 6) - Xr).max() / np.abs(Xr).max())
        errs.append(e)
    assert errs[0] > 1e-3 and errs[2] < 1e-9 and errs[1] < errs[0]


def test_closed_loop_step_matches_numpy():
    ir = programs.quadrotor_lqr_step().to_bytes()
    X = lqr_inputs(32, seed=3)
    y = Oracle(ir).eval(X)
    for i in range(32):
        zn = M.quad_lqr_step(X[:6, i], X[6:, i])[0]
        np.testing.assert_allclose(y[:, i], zn, rtol=1e-9, atol=1e-11)


def test_closed_loop_is_stable():
    """The program's gain K makes A - B K a contraction (spectral radius < 1),
    and near hover the Lyapunov function V = z' X z of the Riccati solution
    decreases at every closed-loop step of the nonlinear program."""
    dbg = Oracle(programs.quadrotor_lqr_step(debug_riccati=True).to_bytes())
    orc = Oracle(programs.quadrotor_lqr_step().to_bytes())
    X = lqr_inputs(16, seed=4)
    X[:6] *= 0.1
    RK = dbg.eval(X)
    z = X[:6].copy()
    V = lambda z, i: z[:, i] @ RK[:36, i].reshape(6, 6) @ z[:, i]
    for i in range(16):
        A, B = M.quad_hover_AB(X[7, i], X[8, i])
        K = RK[36:, i].reshape(2, 6)
        assert max(abs(np.linalg.eigvals(A - B @ K))) < 1.0
    for _ in range(40):
        zn = orc.eval(np.vstack([z, X[6:]]))
        for i in range(16):
            assert V(zn, i) < V(z, i)
        z = zn


def test_thrust_limits_clip_the_control():
    """A large tilt saturates a thrust at 0 or u_max; the step then equals the
    numpy step with the clipped control."""
    ir = programs.quadrotor_lqr_step().to_bytes()
    X = lqr_inputs(16, seed=5)
    X[2] = np.linspace(-1.2, 1.2, 16)
    X[6] = 12.0
    y = Oracle(ir).eval(X)
    saturated = 0
    for i in range(16):
        zn, _, K = M.quad_lqr_step(X[:6, i], X[6:, i])
        u = X[7, i] * 9.81 / 2 - K @ X[:6, i]
        saturated += int(np.any((u < 0) | (u > 12.0)))
        np.testing.assert_allclose(y[:, i], zn, rtol=1e-9, atol=1e-11)
    assert saturated > 0
