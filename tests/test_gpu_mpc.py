"""GPU parity of the closed-form MPC program (unrolled barrier-Newton with an
unrolled LDL^T per iteration) in FP64, FP32 and mixed precision.

Tolerances: FP64 kernels vs the FP64 oracle: max(1e-12 * s_k, 2 * B_k,i);
FP32 and mixed kernels vs the FP64 oracle: max(2e-4 * s_k, 2 * B32_k,i) (the
FP32 bound covers mixed, whose FP64-tagged ops are only more accurate).
"""
import numpy as np
import pytest
import torch

from oracle import MODE_MIXED, Oracle, tolerance
from paper_2408_09662_gb300 import programs
from paper_2408_09662_gb300.api import Function

pytestmark = pytest.mark.gpu


def mpc_inputs(N, seed=0):
    rng = np.random.default_rng(seed)
    return np.vstack([rng.uniform(-0.5, 0.5, (6, N)), rng.uniform(-1, 1, (2, N))])


@pytest.fixture(scope="module")
def mpc():
    return programs.quadrotor_mpc().to_bytes()


def _run(fn, X):
    x = torch.tensor(X, dtype=fn.torch_dtype, device="cuda")
    y = fn(x)
    torch.cuda.synchronize()
    return y.double().cpu().numpy()


def _check(y, ref, tol):
    bad = ~(np.abs(y - ref) <= tol)
    assert not np.any(bad), (int(bad.sum()), float(np.max(np.abs(y - ref) - tol)))


@pytest.mark.parametrize("dtype", ["f64", "mixed", "f32"])
def test_mpc_full_batch_sampled(mpc, dtype):
    """N = 16384 instances; the program is split over two kernels that pass
    their live values through the workspace."""
    N = 16384
    X = mpc_inputs(N, seed=1)
    fn = Function(mpc, dtype=dtype)
    assert fn.info.n_segments >= 2
    if dtype != "f64":
        X = X.astype(np.float32).astype(np.float64)
    y = _run(fn, X)
    assert np.all(np.isfinite(y))
    assert np.all((y[66:] > 0) & (y[66:] < 15))
    idx = np.unique(np.concatenate([np.random.default_rng(2).choice(N, 96, replace=False),
                                    [0, N - 1]]))
    orc = Oracle(mpc)
    ref = orc.eval(X[:, idx])
    if dtype == "f64":
        tol = tolerance(orc, X[:, idx], ref, 1e-12, kind=0)
    else:
        tol = tolerance(orc, X[:, idx], ref, 2e-4, kind=1)
    _check(y[:, idx], ref, tol)


def test_mixed_tracks_its_emulation_more_closely_than_fp32(mpc):
    N = 2048
    X = mpc_inputs(N, seed=3).astype(np.float32).astype(np.float64)
    orc = Oracle(mpc)
    ref64 = orc.eval(X)
    refm = orc.eval(X, mode=MODE_MIXED)
    ym = _run(Function(mpc, dtype="mixed"), X)
    scale = np.max(np.abs(ref64), axis=1, keepdims=True)
    # the GPU's mixed result and the oracle's mixed emulation round the same
    # FP32 ops, so they agree far better than either agrees with FP64
    assert np.max(np.abs(ym - refm) / scale) < 2e-5
    assert np.max(np.abs(ym - ref64) / scale) < 2e-4


def test_mpc_interpreter_matches(mpc):
    N = 1000
    X = mpc_inputs(N, seed=4)
    y = _run(Function(mpc, dtype="f64", path="interp"), X)
    orc = Oracle(mpc)
    ref = orc.eval(X)
    _check(y, ref, tolerance(orc, X, ref, 1e-12, kind=0))


@pytest.mark.parametrize("kw", [dict(constraint="penalty"), dict(warm_start=True)],
                         ids=["penalty", "warm_start"])
def test_mpc_variants_parity(kw):
    """The paper's quadratic-penalty form and the warm-started (real-time
    iteration) form, FP64 on the GPU against the oracle."""
    ir = programs.quadrotor_mpc({"u_max": 12.0}, **kw).to_bytes()
    N = 4096
    X = mpc_inputs(N, seed=5)
    X[6:] *= 6.0
    if kw.get("warm_start"):
        z0 = Oracle(programs.quadrotor_mpc({"u_max": 12.0, "M": 2}).to_bytes()).eval(X)
        X = np.vstack([X, z0])
    fn = Function(ir, dtype="f64")
    y = _run(fn, X)
    orc = Oracle(ir)
    idx = np.random.default_rng(6).choice(N, 64, replace=False)
    ref = orc.eval(X[:, idx])
    _check(y[:, idx], ref, tolerance(orc, X[:, idx], ref, 1e-12, kind=0))


def test_closed_loop_step_parity():
    ir = programs.quadrotor_closed_loop_step().to_bytes()
    N = 4096
    rng = np.random.default_rng(12)
    X = np.vstack([rng.uniform(-0.5, 0.5, (6, N)), rng.uniform(-1, 1, (2, N)),
                   rng.uniform(-1, 16, (86, N)), rng.uniform(0, 5, (2, N))])
    y = _run(Function(ir, dtype="f64"), X)
    orc = Oracle(ir)
    ref = orc.eval(X)
    _check(y, ref, tolerance(orc, X, ref, 1e-12, kind=0))


def test_closed_loop_pareto_small():
    """The Fig. 4 experiment at a small size: the barrier form keeps every
    thrust strictly inside its bounds, the penalty form's violation shrinks as
    its weight grows with M, and more iterations do not raise the cost of a
    stable closed loop."""
    from paper_2408_09662_gb300.experiments import mpc_pareto
    rows = mpc_pareto(N=256, steps=25, Ms=(1, 4), warm_Ms=(1,))
    by = {(r[0], r[1], r[2]): r for r in rows}
    for M in (1, 4):
        assert by[("barrier", "cold", M)][7] == 0.0
        assert by[("barrier", "cold", M)][8] == 0.0
    assert by[("penalty", "cold", 4)][7] < 1e-2 * by[("penalty", "cold", 1)][7]
    assert by[("barrier", "cold", 4)][6] <= by[("barrier", "cold", 1)][6] * 1.05
    assert all(np.isfinite(r[5]) and r[5] > 0 for r in rows)
