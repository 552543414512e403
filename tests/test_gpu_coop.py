"""Within-instance parallelism (options.ways = W): W warps split each program
over 32 instances, exchanging values through shared memory between barrier-
separated phases.  Same parity rule as the one-instance-per-thread kernels:
FP64 max(1e-12 * s_k, 2 * B_k,i), FP32 max(2e-4 * s_k, 2 * B32_k,i)."""
import numpy as np
import pytest
import torch

from oracle import Oracle, tolerance
from paper_2408_09662_gb300 import inputs, programs
from paper_2408_09662_gb300.api import Function

pytestmark = pytest.mark.gpu


def _check(ir, X, fn, tau, kind):
    y = fn(torch.tensor(X, dtype=fn.torch_dtype, device="cuda")).double().cpu().numpy()
    orc = Oracle(ir)
    ref = orc.eval(X)
    tol = tolerance(orc, X, ref, tau, kind=kind)
    same = (y == ref) | (np.isnan(y) & np.isnan(ref))
    bad = ~((np.abs(y - ref) <= tol) | same)
    assert not np.any(bad), int(bad.sum())


@pytest.mark.parametrize("ways", [2, 4, 8])
def test_coop_cartpole(ways):
    ir = programs.cartpole_rk4().to_bytes()
    fn = Function(ir, dtype="f64", ways=ways)
    assert "__syncthreads();" in fn.source()
    for N in (1, 31, 1000, 4096):
        _check(ir, inputs.cartpole(N, seed=N), fn, 1e-12, 0)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_coop_random_program_segmented(dtype):
    ir = programs.random_program(6000, seed=13).to_bytes()
    fn = Function(ir, dtype=dtype, ways=4, segment_ops=2500)
    assert fn.info.n_segments >= 2
    X = inputs.normal(64, 2049, seed=14)
    if dtype == "f32":
        X = X.astype(np.float32).astype(np.float64)
    _check(ir, X, fn, 1e-12 if dtype == "f64" else 2e-4, 0 if dtype == "f64" else 1)


def test_coop_mpc_mixed_and_lqr():
    rng = np.random.default_rng(3)
    mpc = programs.quadrotor_mpc().to_bytes()
    X = np.vstack([rng.uniform(-0.5, 0.5, (6, 300)), rng.uniform(-1, 1, (2, 300))])
    _check(mpc, X, Function(mpc, dtype="f64", ways=4), 1e-12, 0)
    Xm = X.astype(np.float32).astype(np.float64)
    _check(mpc, Xm, Function(mpc, dtype="mixed", ways=4), 2e-4, 1)
    lqr = programs.quadrotor_lqr_step().to_bytes()
    Z = np.vstack([rng.uniform(-0.5, 0.5, (6, 500)), rng.uniform(10, 20, (1, 500)),
                   rng.uniform(0.8, 1.2, (1, 500)), rng.uniform(0.008, 0.012, (1, 500)),
                   rng.uniform(0.5, 10, (6, 500)), rng.uniform(0.05, 0.5, (1, 500))])
    for ways in (4, 6, 8):
        _check(lqr, Z, Function(lqr, dtype="f64", ways=ways), 1e-12, 0)
