"""Differentiable SRB-quadruped rollout on the GPU: 50 RK4 steps of a linear
feedback policy with a shared 12x12 gain, loss = sum of squared states.

Checks: the loss and final state against the numpy model; dL/dK and dL/dx0
against central differences of the numpy model (h = 1e-6, FP64) and against
the oracle's reverse sweep of each step; checkpointed == stored-state
gradients bitwise (the shared-gain reduction sums warp partials in a fixed
order); repeated runs bitwise.
"""
import numpy as np
import pytest
import torch

from oracle import Oracle
from oracle import models as M
from paper_2408_09662_gb300 import programs
from paper_2408_09662_gb300.api import Function
from paper_2408_09662_gb300.rollout import StepProgram, rollout

pytestmark = pytest.mark.gpu
STEPS = 50


def srb_inputs(N, seed=0):
    rng = np.random.default_rng(seed)
    return rng.uniform(-0.1, 0.1, (12, N)), rng.normal(0.0, 0.1, (12, 12))


@pytest.fixture(scope="module")
def prog64():
    return StepProgram(Function(programs.srb_step(), dtype="f64"), 144, 12)


def _grad(prog, x0, K, ce):
    x = torch.tensor(x0, dtype=prog.fn.torch_dtype, device="cuda", requires_grad=True)
    k = torch.tensor(K.reshape(144), dtype=prog.fn.torch_dtype, device="cuda", requires_grad=True)
    L, xT = rollout(prog, x, k, STEPS, checkpoint_every=ce)
    L.backward()
    return float(L), xT.detach().cpu().numpy(), x.grad.cpu().numpy(), k.grad.cpu().numpy().reshape(12, 12)


def test_rollout_loss_matches_numpy_model(prog64):
    x0, K = srb_inputs(64, seed=1)
    L, xT, _, _ = _grad(prog64, x0, K, 10)
    ref_L, ref_x = M.srb_rollout_loss(x0, K, STEPS)
    assert abs(L - float(ref_L)) <= 1e-11 * abs(ref_L)
    np.testing.assert_allclose(xT, ref_x, rtol=1e-10, atol=1e-12)


def test_rollout_gradient_matches_central_differences(prog64):
    """Central differences, h = 1e-6, FP64.  Their own error is rounding of the
    loss, ~eps * |L| / h per difference, so that is added to the tolerance."""
    N = 16
    x0, K = srb_inputs(N, seed=2)
    L, _, gx, gK = _grad(prog64, x0, K, 10)
    h = 1e-6
    fd_noise = 10 * np.finfo(np.float64).eps * abs(L) / h
    rng = np.random.default_rng(3)
    for (a, b) in [tuple(rng.integers(12, size=2)) for _ in range(16)]:
        Kp, Km = K.copy(), K.copy()
        Kp[a, b] += h
        Km[a, b] -= h
        fd = (M.srb_rollout_loss(x0, Kp, STEPS)[0] - M.srb_rollout_loss(x0, Km, STEPS)[0]) / (2 * h)
        assert abs(gK[a, b] - fd) <= 1e-6 * abs(fd) + fd_noise, (a, b, gK[a, b], fd)
    for k in range(12):
        xp, xm = x0.copy(), x0.copy()
        xp[k, 5] += h
        xm[k, 5] -= h
        fd = (M.srb_rollout_loss(xp, K, STEPS)[0] - M.srb_rollout_loss(xm, K, STEPS)[0]) / (2 * h)
        assert abs(gx[k, 5] - fd) <= 1e-6 * abs(fd) + fd_noise, (k, gx[k, 5], fd)


def test_rollout_gradient_matches_complex_step(prog64):
    """Complex-step derivatives of the numpy model are exact to rounding, so the
    reverse sweep must agree to ~1e-10 of the largest gradient entry."""
    N = 8
    x0, K = srb_inputs(N, seed=8)
    _, _, gx, gK = _grad(prog64, x0, K, 10)
    h = 1e-30
    rng = np.random.default_rng(9)
    for (a, b) in [tuple(rng.integers(12, size=2)) for _ in range(12)]:
        Kc = K.astype(np.complex128)
        Kc[a, b] += 1j * h
        cs = M.srb_rollout_loss(x0, Kc, STEPS)[0].imag / h
        assert abs(gK[a, b] - cs) <= 1e-10 * np.max(np.abs(gK)), (a, b, gK[a, b], cs)
    for k in range(0, 12, 3):
        xc = x0.astype(np.complex128)
        xc[k, 3] += 1j * h
        cs = M.srb_rollout_loss(xc, K, STEPS)[0].imag / h
        assert abs(gx[k, 3] - cs) <= 1e-10 * np.max(np.abs(gx)), (k, gx[k, 3], cs)


def test_step_adjoint_matches_oracle_reverse_sweep(prog64):
    N = 2048
    x0, K = srb_inputs(N, seed=4)
    X = np.vstack([np.tile(K.reshape(144, 1), (1, N)), x0, np.zeros((1, N))])
    ybar = np.random.default_rng(5).standard_normal((13, N))
    ref = Oracle(programs.srb_step().to_bytes()).adjoint(X, ybar)
    fn = prog64.fn
    xb = fn.adjoint(torch.tensor(X, device="cuda"), torch.tensor(ybar, device="cuda"),
                    reduce_broadcast=True).cpu().numpy()
    s = np.max(np.abs(ref[144:]))
    np.testing.assert_allclose(xb[144:], ref[144:], rtol=0, atol=1e-12 * s)
    Kref = ref[:144].sum(axis=1)
    np.testing.assert_allclose(xb[:144, 0], Kref, rtol=1e-11, atol=1e-12 * np.max(np.abs(Kref)))


def test_fp32_step_adjoint_matches_oracle_reverse_sweep():
    """The FP32 adjoint kernel of one SRB step against the oracle's FP64 reverse
    sweep on the same FP32-rounded inputs, under the FP32 rule: per input row
    k, 2e-4 of the row's largest adjoint; for the shared gain reduced over the
    2,048 instances, 2e-4 of the sum of the magnitudes it adds up."""
    N = 2048
    x0, K = srb_inputs(N, seed=14)
    X = np.vstack([np.tile(K.reshape(144, 1), (1, N)), x0, np.zeros((1, N))])
    X = X.astype(np.float32).astype(np.float64)
    ybar = np.random.default_rng(15).standard_normal((13, N)).astype(np.float32).astype(np.float64)
    ref = Oracle(programs.srb_step().to_bytes()).adjoint(X, ybar)
    fn = Function(programs.srb_step(), dtype="f32")
    xb = fn.adjoint(torch.tensor(X, dtype=torch.float32, device="cuda"),
                    torch.tensor(ybar, dtype=torch.float32, device="cuda"),
                    reduce_broadcast=True).double().cpu().numpy()
    s = np.max(np.abs(ref[144:]), axis=1, keepdims=True)
    assert np.all(np.abs(xb[144:] - ref[144:]) <= 2e-4 * s)
    Kref = ref[:144].sum(axis=1)
    scale = np.abs(ref[:144]).sum(axis=1)
    assert np.all(np.abs(xb[:144, 0] - Kref) <= 2e-4 * scale)


def _oracle_rollout_gradient(x0, K, steps):
    """dL/dx0 and dL/dK of the rollout from the oracle alone: FP64 forward steps
    with every state kept, then the oracle's reverse sweep of each step in
    reverse order, the shared gain's per-instance adjoints summed over
    instances and steps."""
    orc = Oracle(programs.srb_step().to_bytes())
    N = x0.shape[1]
    X = np.vstack([np.tile(K.reshape(144, 1), (1, N)), x0, np.zeros((1, N))])
    states = []
    for _ in range(steps):
        states.append(X.copy())
        X[144:] = orc.eval(X)
    ybar = np.zeros((13, N))
    ybar[12] = 1.0                        # dL/dL_T; the final states carry no gradient
    gK = np.zeros(144)
    for X in reversed(states):
        xb = orc.adjoint(X, ybar)
        gK += xb[:144].sum(axis=1)
        ybar = xb[144:]
    return ybar[:12], gK.reshape(12, 12)


def test_fp32_rollout_gradient_against_oracle():
    """50 steps in FP32 through the checkpointed reverse pass against the
    oracle's FP64 reverse sweeps on the same FP32-rounded x0 and K: per state
    row, 2e-4 of the row's largest gradient; the gain, 2e-4 of its largest
    entry."""
    x0, K = srb_inputs(256, seed=16)
    x0 = x0.astype(np.float32).astype(np.float64)
    K = K.astype(np.float32).astype(np.float64)
    prog32 = StepProgram(Function(programs.srb_step(), dtype="f32"), 144, 12)
    _, _, gx, gK = _grad(prog32, x0, K, 10)
    rgx, rgK = _oracle_rollout_gradient(x0, K, STEPS)
    s = np.max(np.abs(rgx), axis=1, keepdims=True)
    rel_x = float(np.max(np.abs(gx - rgx) / s))
    rel_K = float(np.max(np.abs(gK - rgK)) / np.max(np.abs(rgK)))
    assert rel_x <= 2e-4 and rel_K <= 2e-4, (rel_x, rel_K)


def test_adjoint_shared_equals_reduced_rows_bitwise():
    """cusadi_adjoint_shared writes the same sums, bit for bit, to its own
    vector that cusadi_adjoint with the reduction writes to column 0 of the
    broadcast rows, leaves those rows of in_bar alone, and accumulates."""
    fn = Function(programs.srb_step(), dtype="f64")
    N = 3000
    x0, K = srb_inputs(N, seed=17)
    X = torch.tensor(np.vstack([np.tile(K.reshape(144, 1), (1, N)), x0, np.zeros((1, N))]), device="cuda")
    ybar = torch.tensor(np.random.default_rng(18).standard_normal((13, N)), device="cuda")
    red = fn.adjoint(X, ybar, reduce_broadcast=True)
    out = torch.full((157, N), 7.0, dtype=torch.float64, device="cuda")
    shared = torch.full((157,), -1.0, dtype=torch.float64, device="cuda")
    fn.adjoint(X, ybar, out=out, shared_out=shared)
    torch.cuda.synchronize()
    assert torch.equal(shared[:144], red[:144, 0])
    assert torch.all(shared[144:] == -1.0) and torch.all(out[:144] == 7.0)
    assert torch.equal(out[144:], red[144:])
    fn.adjoint(X, ybar, out=out, shared_out=shared, accumulate_broadcast=True)
    torch.cuda.synchronize()
    assert torch.equal(shared[:144], red[:144, 0] + red[:144, 0])


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_sum_instances_is_reproducible_and_accurate(dtype):
    from paper_2408_09662_gb300.api import sum_instances
    rng = np.random.default_rng(19)
    y = rng.standard_normal((5, 100003))
    yt = torch.tensor(y, dtype=dtype, device="cuda")
    a, b = sum_instances(yt), sum_instances(yt)
    c = sum_instances(yt, out=a.clone(), accumulate=True)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(c, a + a)
    exact = y.astype(np.float32 if dtype == torch.float32 else np.float64).astype(np.float64).sum(axis=1)
    u = 2.0 ** (-24 if dtype == torch.float32 else -53)
    bound = (200 + 9) * u * np.abs(y).sum(axis=1)      # per-thread chains of <= 196, tree of 9
    assert np.all(np.abs(a.double().cpu().numpy() - exact) <= bound)


def test_rollout_loss_sum_is_bitwise_reproducible(prog64):
    x0, K = srb_inputs(4096, seed=20)
    Ls = [_grad(prog64, x0, K, 10)[0] for _ in range(3)]
    assert Ls[0] == Ls[1] == Ls[2]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_rollout_at_the_benchmark_batch_against_oracle(dtype):
    """The benchmark's rollout configuration itself: N = 4,096 instances, 50
    RK4 steps, checkpoints every 10, shared 12x12 gain.  Loss, dL/dx0 and dL/dK
    against the oracle's FP64 forward steps and reverse sweeps on the same
    (for FP32: FP32-rounded) x0 and K; FP64 to 1e-11 of each row's scale, FP32
    under the FP32 rule 2e-4 of each row's scale."""
    N = 4096
    x0, K = srb_inputs(N, seed=21)
    tau = 1e-11 if dtype == "f64" else 2e-4
    if dtype == "f32":
        x0 = x0.astype(np.float32).astype(np.float64)
        K = K.astype(np.float32).astype(np.float64)
    prog = StepProgram(Function(programs.srb_step(), dtype=dtype), 144, 12)
    L, _, gx, gK = _grad(prog, x0, K, 10)
    orc = Oracle(programs.srb_step().to_bytes())
    X = np.vstack([np.tile(K.reshape(144, 1), (1, N)), x0, np.zeros((1, N))])
    for _ in range(STEPS):
        X[144:] = orc.eval(X)
    assert abs(L - X[156].sum()) <= tau * abs(X[156].sum())
    rgx, rgK = _oracle_rollout_gradient(x0, K, STEPS)
    assert np.all(np.abs(gx - rgx) <= tau * np.max(np.abs(rgx), axis=1, keepdims=True))
    assert np.max(np.abs(gK - rgK)) <= tau * np.max(np.abs(rgK))


def test_checkpointing_does_not_change_the_gradient(prog64):
    x0, K = srb_inputs(512, seed=6)
    L1, _, gx1, gK1 = _grad(prog64, x0, K, 10)
    L2, _, gx2, gK2 = _grad(prog64, x0, K, 1)      # every state stored, no recompute
    assert L1 == L2
    np.testing.assert_array_equal(gx1, gx2)
    np.testing.assert_array_equal(gK1, gK2)


def test_fp32_rollout_gradient_close_to_fp64(prog64):
    x0, K = srb_inputs(1024, seed=7)
    prog32 = StepProgram(Function(programs.srb_step(), dtype="f32"), 144, 12)
    L64, _, gx64, gK64 = _grad(prog64, x0, K, 10)
    L32, _, gx32, gK32 = _grad(prog32, x0, K, 10)
    assert abs(L32 - L64) <= 1e-4 * abs(L64)
    assert np.max(np.abs(gK32 - gK64)) <= 2e-3 * np.max(np.abs(gK64))


def test_graph_replayed_rollout_matches_eager(prog64):
    from paper_2408_09662_gb300.rollout import GraphRollout
    x0, K = srb_inputs(1024, seed=11)
    L, xT, gx, gK = _grad(prog64, x0, K, 10)
    gr = GraphRollout(prog64, 1024, STEPS, 10)
    for _ in range(2):                       # replay twice with the same inputs
        Lg, xTg = gr.forward(torch.tensor(x0, device="cuda"), torch.tensor(K.reshape(144), device="cuda"))
        gxg, gKg = gr.backward()
        torch.cuda.synchronize()
        assert float(Lg) == L
        np.testing.assert_array_equal(xTg.cpu().numpy(), xT)
        np.testing.assert_array_equal(gxg.cpu().numpy(), gx)
        np.testing.assert_array_equal(gKg.cpu().numpy().reshape(12, 12), gK)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_shared_gain_reduction_is_reproducible(dtype):
    """The 144 broadcast rows summed over 65,536 instances: repeated adjoints
    give the same bits, with and without
    accumulation, and the sum matches a float64 sum of the per-instance
    adjoints (reduce_broadcast off) to rounding."""
    fn = Function(programs.srb_step(), dtype=dtype, adjoint=1)
    N = 65536
    rng = np.random.default_rng(12)
    X = np.vstack([np.tile(rng.normal(0, 0.1, (144, 1)), (1, N)), rng.uniform(-0.1, 0.1, (12, N)),
                   np.zeros((1, N))])
    x = torch.tensor(X, dtype=fn.torch_dtype, device="cuda")
    ybar = torch.tensor(rng.normal(0, 1, (13, N)), dtype=fn.torch_dtype, device="cuda")
    a = fn.adjoint(x, ybar, reduce_broadcast=True)
    b = fn.adjoint(x, ybar, reduce_broadcast=True)
    c = fn.adjoint(x, ybar, reduce_broadcast=True)
    fn.adjoint(x, ybar, out=c, reduce_broadcast=True, accumulate_broadcast=True)
    per = fn.adjoint(x, ybar)
    torch.cuda.synchronize()
    # written entries only: column 0 of the reduced rows, every column of the others
    assert torch.equal(a[:144, 0], b[:144, 0]) and torch.equal(a[144:], b[144:])
    assert torch.equal(c[:144, 0], (a[:144, 0].double() * 2).to(fn.torch_dtype)) or \
        np.allclose(c[:144, 0].double().cpu().numpy(), 2 * a[:144, 0].double().cpu().numpy(), rtol=1e-6)
    want = per[:144].double().sum(dim=1).cpu().numpy()
    got = a[:144, 0].double().cpu().numpy()
    tol = (1e-12 if dtype == "f64" else 2e-5) * per[:144].double().abs().sum(dim=1).cpu().numpy()
    assert np.all(np.abs(got - want) <= tol)
