"""GPU parity of the quadcopter LQR closed-loop step (SDA Riccati solve inside
the program) and a 10,000-instance closed-loop rollout for a region-of-
attraction sweep over initial momenta and thrust limits.

Tolerances: FP64 vs the FP64 oracle max(1e-12 * s_k, 2 * B_k,i); FP32 vs the
FP64 oracle max(2e-4 * s_k, 2 * B32_k,i)."""
import numpy as np
import pytest
import torch

from oracle import Oracle, tolerance
from paper_2408_09662_gb300 import programs
from paper_2408_09662_gb300.api import Function

pytestmark = pytest.mark.gpu


def lqr_inputs(N, seed=0):
    rng = np.random.default_rng(seed)
    z = rng.uniform(-0.5, 0.5, (6, N))
    theta = np.vstack([rng.uniform(10, 20, (1, N)), rng.uniform(0.8, 1.2, (1, N)),
                       rng.uniform(0.008, 0.012, (1, N)), rng.uniform(0.5, 10, (6, N)),
                       rng.uniform(0.05, 0.5, (1, N))])
    return np.vstack([z, theta])


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_lqr_step_parity(dtype):
    ir = programs.quadrotor_lqr_step().to_bytes()
    N = 10000
    X = lqr_inputs(N, seed=1)
    if dtype == "f32":
        X = X.astype(np.float32).astype(np.float64)
    fn = Function(ir, dtype=dtype)
    y = fn(torch.tensor(X, dtype=fn.torch_dtype, device="cuda")).double().cpu().numpy()
    idx = np.unique(np.concatenate([np.random.default_rng(2).choice(N, 128, replace=False), [N - 1]]))
    orc = Oracle(ir)
    ref = orc.eval(X[:, idx])
    tol = tolerance(orc, X[:, idx], ref, 1e-12 if dtype == "f64" else 2e-4, kind=0 if dtype == "f64" else 1)
    assert np.all(np.abs(y[:, idx] - ref) <= tol)


def test_region_of_attraction_rollout():
    """10,000 instances from zero position/angle with different linear and
    angular momenta and thrust limits, 250 closed-loop steps on the GPU; the
    stable set matches the oracle's rollout on a sample."""
    ir = programs.quadrotor_lqr_step().to_bytes()
    fn = Function(ir, dtype="f64")
    N = 10000
    rng = np.random.default_rng(3)
    X = lqr_inputs(N, seed=4)
    X[:3] = 0.0
    X[3:6] = rng.uniform(-3, 3, (3, N)) * np.array([[1.0], [1.0], [8.0]])
    X[6] = rng.choice([6.0, 10.0, 20.0], N)
    X[9:15] = 5.0
    X[15] = 0.1
    buf = [torch.tensor(X, device="cuda"), torch.tensor(X, device="cuda")]
    for t in range(250):
        fn(buf[t % 2], out=buf[(t + 1) % 2][:6])
    zT = buf[250 % 2][:6].cpu().numpy()
    stable = np.all(np.abs(zT) < 0.5, axis=0) & np.all(np.isfinite(zT), axis=0)
    assert 0.05 < stable.mean() < 0.999
    # stability grows with the thrust limit
    rates = [stable[X[6] == u].mean() for u in (6.0, 10.0, 20.0)]
    assert rates[0] <= rates[1] <= rates[2]
    orc = Oracle(ir)
    idx = rng.choice(N, 48, replace=False)
    Z = X[:, idx].copy()
    for t in range(250):
        Z[:6] = orc.eval(Z)
    ref_stable = np.all(np.abs(Z[:6]) < 0.5, axis=0) & np.all(np.isfinite(Z[:6]), axis=0)
    # trajectories near the boundary of the region may split on rounding alone
    assert np.mean(ref_stable == stable[idx]) >= 0.95
