"""Launch shapes of the compiled path: several instances per thread (with
vector loads and stores), CTA barriers every few hundred ops, several groups
of 32 instances per cooperative CTA, and the engine's own FP32 math as
out-of-line functions.

Each shape evaluates every instance with the same ops in the same order as
the one-instance-per-thread kernel, so with FMA contraction off the results
must be the same bits; one case per shape is also checked against the oracle
under the parity tolerances (max(1e-12 s_k, 2 B) in FP64, max(2e-4 s_k, 2 B32)
in FP32).  Ragged batches (N not a multiple of the instances per thread),
buffers whose alignment rules out vector accesses, and columns past N (never
written) are covered.
"""
import numpy as np
import pytest
import torch

from oracle import Oracle, tolerance
from paper_2408_09662_gb300 import inputs, programs
from paper_2408_09662_gb300.api import Function

pytestmark = pytest.mark.gpu

TDT = {"f64": torch.float64, "f32": torch.float32, "mixed": torch.float32}


def _eval(fn, x, ld=None, offset=0):
    """fn on x [rows, N] held in a [rows, ld] buffer starting `offset` elements
    into its storage; the output likewise; returns (y, the whole output buffer)."""
    rows, N = x.shape
    ld = ld or N
    xs = torch.zeros(rows * ld + offset + 8, dtype=fn.torch_dtype, device="cuda")
    xb = xs[offset:offset + rows * ld].view(rows, ld)
    xb[:, :N] = torch.tensor(x, dtype=fn.torch_dtype, device="cuda")
    ys = torch.full((fn.nnz_out * ld + offset + 8,), 7.0, dtype=fn.torch_dtype, device="cuda")
    yb = ys[offset:offset + fn.nnz_out * ld].view(fn.nnz_out, ld)
    fn(xb[:, :N], out=yb[:, :N])
    torch.cuda.synchronize()
    return yb[:, :N].double().cpu().numpy(), yb


@pytest.fixture(scope="module")
def rand3k():
    return programs.random_program(3000, seed=61).to_bytes()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("lanes", [2, 4])
def test_lanes_equal_one_lane_bitwise(rand3k, dtype, lanes):
    one = Function(rand3k, dtype=dtype, fmad=0)
    many = Function(rand3k, dtype=dtype, fmad=0, inst_per_thread=lanes)
    many_seg = Function(rand3k, dtype=dtype, fmad=0, inst_per_thread=lanes, segment_ops=700)
    assert many_seg.info.n_segments > 1
    for N in (1, 2, 3, 5, 33, 4099):
        x = inputs.normal(64, N, seed=N).astype(np.float32).astype(np.float64)
        ref, _ = _eval(one, x)
        for fn in (many, many_seg):
            got, buf = _eval(fn, x)
            np.testing.assert_array_equal(got, ref, err_msg=f"N={N}")
    # vector accesses ruled out: odd leading dimension, base one element off
    x = inputs.normal(64, 1001, seed=3).astype(np.float32).astype(np.float64)
    ref, _ = _eval(one, x)
    for ld, off in ((1003, 0), (1004, 1), (1004, 0)):
        got, buf = _eval(many, x, ld=ld, offset=off)
        np.testing.assert_array_equal(got, ref, err_msg=f"ld={ld} offset={off}")
        assert torch.all(buf[:, 1001:] == 7.0)           # nothing written past N


def test_lanes_against_the_oracle():
    ir = programs.cartpole_rk4().to_bytes()
    orc = Oracle(ir)
    x = inputs.cartpole(4099, seed=11)
    ref = orc.eval(x)
    y, _ = _eval(Function(ir, dtype="f64", inst_per_thread=2), x)
    assert np.all(np.abs(y - ref) <= tolerance(orc, x, ref, 1e-12, kind=0))
    x32 = x.astype(np.float32).astype(np.float64)
    ref32 = orc.eval(x32)
    y, _ = _eval(Function(ir, dtype="f32", inst_per_thread=4), x32)
    assert np.all(np.abs(y - ref32) <= tolerance(orc, x32, ref32, 2e-4, kind=1))


def test_mixed_precision_lanes_equal_one_lane_bitwise():
    ir = programs.quadrotor_mpc(dict(programs.QUADROTOR, M=1)).to_bytes()
    rng = np.random.default_rng(5)
    N = 1027
    x = np.vstack([rng.uniform(-0.5, 0.5, (6, N)), rng.uniform(-1, 1, (2, N))])
    x = x.astype(np.float32).astype(np.float64)
    ref, _ = _eval(Function(ir, dtype="mixed", fmad=0), x)
    got, _ = _eval(Function(ir, dtype="mixed", fmad=0, inst_per_thread=2), x)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("lanes", [2, 4])
def test_adjoint_lanes_equal_one_lane_bitwise(lanes):
    """The SRB step's reverse sweep with its 144 broadcast gain rows reduced
    over instances (per-instance terms, fixed-order sum) and accumulated."""
    ir = programs.srb_step().to_bytes()
    rng = np.random.default_rng(13)
    N = 2051
    X = np.vstack([np.tile(rng.normal(0, 0.1, (144, 1)), (1, N)), rng.uniform(-0.1, 0.1, (12, N)),
                   np.zeros((1, N))])
    ybar = rng.standard_normal((13, N))
    res = []
    for R in (1, lanes):
        fn = Function(ir, dtype="f64", fmad=0, inst_per_thread=R)
        xd = torch.tensor(X, device="cuda")
        yd = torch.tensor(ybar, device="cuda")
        a = fn.adjoint(xd, yd, reduce_broadcast=True)
        b = torch.ones((157, N), dtype=torch.float64, device="cuda")
        fn.adjoint(xd, yd, out=b, accumulate=True, reduce_broadcast=True)
        torch.cuda.synchronize()
        res.append((a[:144, 0].cpu().numpy(), a[144:].cpu().numpy(), b[:144, 0].cpu().numpy(),
                    b[144:].cpu().numpy()))
    for u, v in zip(*res):
        np.testing.assert_array_equal(u, v)
    ref = Oracle(ir).adjoint(X, ybar)
    np.testing.assert_allclose(res[1][1], ref[144:], rtol=0, atol=1e-12 * np.max(np.abs(ref[144:])))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_cta_barriers_do_not_change_results(rand3k, dtype):
    one = Function(rand3k, dtype=dtype, fmad=0)
    x = inputs.normal(64, 4099, seed=21).astype(np.float32).astype(np.float64)
    ref, _ = _eval(one, x)
    for block, every in ((256, 200), (512, 1000), (128, 1)):
        fn = Function(rand3k, dtype=dtype, fmad=0, block=block, sync_every=every)
        got, buf = _eval(fn, x, ld=4099 + 29)
        np.testing.assert_array_equal(got, ref, err_msg=f"block={block} every={every}")
        assert torch.all(buf[:, 4099:] == 7.0)
    fn = Function(rand3k, dtype=dtype, fmad=0, block=256, sync_every=100, inst_per_thread=2)
    np.testing.assert_array_equal(_eval(fn, x)[0], ref)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_cooperative_groups_per_cta_equal_one_group_bitwise(rand3k, dtype):
    x = inputs.normal(64, 4099, seed=23).astype(np.float32).astype(np.float64)
    ref, _ = _eval(Function(rand3k, dtype=dtype, fmad=0, ways=4), x)
    for G in (2, 4):
        fn = Function(rand3k, dtype=dtype, fmad=0, ways=4, coop_groups=G)
        got, buf = _eval(fn, x, ld=4099 + 3)
        np.testing.assert_array_equal(got, ref, err_msg=f"groups={G}")
        assert torch.all(buf[:, 4099:] == 7.0)


def test_own_math_out_of_line_equals_inlined(rand3k):
    x = inputs.normal(64, 4099, seed=25).astype(np.float32).astype(np.float64)
    ref, _ = _eval(Function(rand3k, dtype="f32", fmad=0, own_math=1), x)
    got, _ = _eval(Function(rand3k, dtype="f32", fmad=0, own_math=2), x)
    np.testing.assert_array_equal(got, ref)
    got4, _ = _eval(Function(rand3k, dtype="f32", fmad=0, own_math=2, ways=4), x)
    np.testing.assert_array_equal(got4, ref)
    orc = Oracle(rand3k)
    y = orc.eval(x)
    assert np.all(np.abs(got - y) <= tolerance(orc, x, y, 2e-4, kind=1))


@pytest.mark.parametrize("dtype", ["f64", "f32", "mixed"])
def test_register_budget_spills_give_the_same_bits(rand3k, dtype):
    """spill_values caps the values a thread keeps in registers; the rest live
    in shared-memory slots, in workspace rows (a 4 KB shared budget forces
    those) or are re-read from their input / carried row.  Only where values
    live changes, so the results keep their bits."""
    ir = rand3k if dtype != "mixed" else programs.quadrotor_mpc(dict(programs.QUADROTOR, M=1)).to_bytes()
    x = (inputs.normal(64, 4099, seed=27) if dtype != "mixed" else
         np.vstack([np.random.default_rng(3).uniform(-0.5, 0.5, (6, 4099)),
                    np.random.default_rng(4).uniform(-1, 1, (2, 4099))]))
    x = x.astype(np.float32).astype(np.float64)
    ref, _ = _eval(Function(ir, dtype=dtype, fmad=0), x)
    for opts in (dict(spill_values=24), dict(spill_values=24, spill_shared_kb=4, segment_ops=900)):
        fn = Function(ir, dtype=dtype, fmad=0, **opts)
        got, buf = _eval(fn, x, ld=4099 + 5)
        np.testing.assert_array_equal(got, ref, err_msg=str(opts))
        assert torch.all(buf[:, 4099:] == 7.0)


def test_register_budget_in_the_adjoint():
    ir = programs.srb_step().to_bytes()
    rng = np.random.default_rng(29)
    N = 2051
    X = np.vstack([np.tile(rng.normal(0, 0.1, (144, 1)), (1, N)), rng.uniform(-0.1, 0.1, (12, N)),
                   np.zeros((1, N))])
    ybar = rng.standard_normal((13, N))
    res = []
    for opts in ({}, dict(spill_values=32, spill_shared_kb=8)):
        fn = Function(ir, dtype="f64", fmad=0, **opts)
        a = fn.adjoint(torch.tensor(X, device="cuda"), torch.tensor(ybar, device="cuda"), reduce_broadcast=True)
        torch.cuda.synchronize()
        res.append((a[:144, 0].cpu().numpy(), a[144:].cpu().numpy()))
    for u, v in zip(*res):
        np.testing.assert_array_equal(u, v)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_paired_math_calls_give_the_same_bits(rand3k, dtype):
    """pair_calls evaluates two calls of the same out-of-line function in one
    call (the second hoisted from a few ops later): the same function on the
    same argument, so the same bits."""
    x = inputs.normal(64, 4099, seed=31).astype(np.float32).astype(np.float64)
    ref, _ = _eval(Function(rand3k, dtype=dtype, fmad=0), x)
    for window in (8, 256):
        fn = Function(rand3k, dtype=dtype, fmad=0, pair_calls=window)
        assert "2_" + ("d" if dtype == "f64" else "f") + "(" in fn.source()
        got, buf = _eval(fn, x, ld=4099 + 1)
        np.testing.assert_array_equal(got, ref, err_msg=f"window {window}")
        assert torch.all(buf[:, 4099:] == 7.0)
