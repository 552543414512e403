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


@pytest.mark.parametrize("ways", [4, 8])
def test_cooperative_adjoint_equals_plain_adjoint(ways):
    """The SRB step's adjoint split over W warps per 32 instances: with FMA
    contraction off every op rounds once in either layout, so the per-instance
    rows and the 144 reduced gain rows agree bit for bit with
    the one-thread-per-instance adjoint, for every flag combination (the
    reduced rows' per-instance terms are summed by the same finishing kernel)."""
    ir = programs.srb_step().to_bytes()
    a = Function(ir, dtype="f64", fmad=0, adjoint=1)
    b = Function(ir, dtype="f64", fmad=0, adjoint=1, ways=ways)
    N = 4100
    rng = np.random.default_rng(50 + ways)
    X = np.vstack([np.tile(rng.normal(0, 0.1, (144, 1)), (1, N)), rng.uniform(-0.1, 0.1, (12, N)),
                   np.zeros((1, N))])
    x = torch.tensor(X, device="cuda")
    ybar = torch.tensor(rng.normal(0, 1, (13, N)), device="cuda")
    for kw in (dict(), dict(reduce_broadcast=True), dict(accumulate=True),
               dict(reduce_broadcast=True, accumulate_broadcast=True)):
        outs = []
        for fn in (a, b):
            o = torch.ones((157, N), dtype=torch.float64, device="cuda")
            fn.adjoint(x, ybar, out=o, **kw)
            outs.append(o)
        torch.cuda.synchronize()
        assert torch.equal(outs[0], outs[1]), kw


def test_cooperative_rollout_gradient_equals_plain():
    from paper_2408_09662_gb300.rollout import StepProgram, rollout
    ir = programs.srb_step().to_bytes()
    res = []
    for ways in (0, 8):
        prog = StepProgram(Function(ir, dtype="f64", fmad=0, adjoint=1, ways=ways), 144, 12)
        rng = np.random.default_rng(60)
        x0 = torch.tensor(rng.uniform(-0.1, 0.1, (12, 2048)), device="cuda", requires_grad=True)
        K = torch.tensor(rng.normal(0, 0.1, 144), device="cuda", requires_grad=True)
        L, xT = rollout(prog, x0, K, 20)
        L.backward()
        res.append((L.item(), xT.detach().cpu(), x0.grad.cpu(), K.grad.cpu()))
    assert res[0][0] == res[1][0]
    for u, v in zip(res[0][1:], res[1][1:]):
        assert torch.equal(u, v)


def test_tuned_picks_the_fastest_configuration_and_keeps_results():
    from paper_2408_09662_gb300.api import tuned
    ir = programs.cartpole_rk4().to_bytes()
    x = torch.tensor(inputs.cartpole(4096, seed=70), device="cuda")
    fn = tuned(ir, x, "f64", candidates=(0, 4), fmad=0)
    assert fn.ways in (0, 4) and set(fn.tuning_ms) == {0, 4}
    assert fn.tuning_ms[fn.ways] == min(fn.tuning_ms.values())
    ref = Function(ir, dtype="f64", fmad=0)(x)
    torch.cuda.synchronize()
    assert torch.equal(fn(x), ref)
