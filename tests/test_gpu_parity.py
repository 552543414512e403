"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, element
by element on the same seeded inputs.

Tolerances (per output row k and instance i), written out in each test:
* FP64 kernels vs the FP64 oracle: max(1e-12 * s_k, 2 * B_k,i), s_k = max_i |y_k,i|,
  B the first-order rounding bound of the program at that instance (GPU ulp
  table + host libm); it only exceeds 1e-12 * s_k on deep programs.
* FP32 kernels vs the FP64 oracle: max(2e-4 * s_k, 2 * B32_k,i), B32 the FP32
  bound (u = 2^-24 plus the GPU's FP32 ulp table).
* FP32 kernels built without contraction vs the oracle's FP32 emulation, on
  programs of correctly rounded ops only: bit-exact.
"""
import numpy as np
import pytest
import torch

from oracle import MODE_F32, Oracle, tolerance
from paper_2408_09662_gb300 import inputs, programs
from paper_2408_09662_gb300.api import Function, apply
from paper_2408_09662_gb300.ir import BINARY, Op

pytestmark = pytest.mark.gpu

TAU64, TAU32 = 1e-12, 2e-4


def dev(x, fn):
    return torch.tensor(np.ascontiguousarray(x), dtype=fn.torch_dtype, device="cuda")


def run(fn, x):
    y = fn(dev(x, fn))
    torch.cuda.synchronize()
    return y.double().cpu().numpy()


def assert_within(y, ref, tol, what=""):
    err = np.abs(y - ref)
    same = (y == ref) | (np.isnan(y) & np.isnan(ref))   # equal infinities, NaN for NaN
    bad = ~((err <= tol) | same)
    if np.any(bad):
        k, i = np.argwhere(bad)[0]
        raise AssertionError(f"{what}: {bad.sum()} of {bad.size} outside tolerance; first at row {k} "
                             f"instance {i}: got {y[k, i]!r} want {ref[k, i]!r} tol {tol[k, i]!r}")


def check_f64(ir, x, fn):
    orc = Oracle(ir)
    ref = orc.eval(x)
    y = run(fn, x)
    assert_within(y, ref, tolerance(orc, x, ref, TAU64, kind=0), "f64")
    return y, ref


def check_f32(ir, x, fn):
    orc = Oracle(ir)
    x32 = x.astype(np.float32).astype(np.float64)   # the float buffer holds rounded inputs
    ref = orc.eval(x32)
    y = run(fn, x32)
    assert_within(y, ref, tolerance(orc, x32, ref, TAU32, kind=1), "f32")
    return y, ref


# ---------------------------------------------------------------------------
def test_listing2():
    ir = programs.listing2().to_bytes()
    x = np.linspace(-5, 5, 1000)[None, :]
    for dt in ("f64", "f32"):
        fn = Function(ir, dtype=dt)
        (check_f64 if dt == "f64" else check_f32)(ir, x, fn)
    y = run(Function(ir), x)
    np.testing.assert_allclose(y[0], (np.sin(x[0]) + x[0]) ** 2, rtol=1e-15)


_UNARY_DOMAIN = {Op.LOG: (0.1, 5), Op.SQRT: (0, 9), Op.ASIN: (-0.99, 0.99), Op.ACOS: (-0.99, 0.99),
                 Op.LOG1P: (-0.9, 4), Op.INV: (0.5, 3), Op.TAN: (-1.4, 1.4), Op.POW: (0.1, 3)}
ALL_OPS = [op for op in Op if op not in (Op.INPUT, Op.OUTPUT, Op.CONST, Op.ASSIGN)]


@pytest.mark.parametrize("path", ["compiled", "interp"])
@pytest.mark.parametrize("op", ALL_OPS, ids=lambda o: o.name)
def test_single_op(op, path):
    ir = programs.single_op(op).to_bytes()
    lo, hi = _UNARY_DOMAIN.get(op, (-3, 3))
    rng = np.random.default_rng(int(op))
    N = 1000
    x = rng.uniform(lo, hi, size=(2, N))
    x[:, ::7] = np.round(x[:, ::7])             # ties, zeros and equal operands
    if op in (Op.DIV, Op.FMOD):
        x[1] = np.where(np.abs(x[1]) < 0.2, 0.7, x[1])
    binary = op in BINARY or op == Op.FMA_CONST
    xin = x if binary else x[:1]
    check_f64(ir, xin, Function(ir, dtype="f64", path=path))
    check_f32(ir, xin, Function(ir, dtype="f32", path=path))


def test_cartpole_rk4_jacobian_f64():
    ir = programs.cartpole_rk4().to_bytes()
    x = inputs.cartpole(4096, seed=0)
    check_f64(ir, x, Function(ir, dtype="f64"))


def test_cartpole_f32_and_interp():
    ir = programs.cartpole_rk4().to_bytes()
    x = inputs.cartpole(4096 + 17, seed=1)
    check_f32(ir, x, Function(ir, dtype="f32"))
    check_f64(ir, x, Function(ir, dtype="f64", path="interp"))


@pytest.mark.parametrize("N", [1, 31, 32, 33, 4096 + 37])
def test_random_program_ragged_batches(N):
    ir = programs.random_program(2500, seed=3).to_bytes()
    x = inputs.normal(64, N, seed=4)
    check_f64(ir, x, Function(ir, dtype="f64"))
    check_f32(ir, x, Function(ir, dtype="f32"))


def test_fp32_without_contraction_is_bit_exact_on_correctly_rounded_ops():
    """Only add/sub/mul/div/sqrt/fma: every op is correctly rounded in IEEE float."""
    from paper_2408_09662_gb300 import tracer as T
    g = T.Graph()
    x = g.symbols(8)
    rng = np.random.default_rng(5)
    vals = list(x)
    for t in range(3000):
        a, b = vals[-1 - int(rng.integers(min(len(vals), 50)))], vals[-1 - int(rng.integers(min(len(vals), 50)))]
        k = t % 5
        v = [a + b, a - b, a * 0.75 + b * 0.25, a / (1.5 + T.sq(b)), T.sqrt(1.0 + T.sq(a))][k]
        vals.append(v)
    ir = T.Function([("x", x)], [("y", vals[-16:])]).to_ir().to_bytes()
    X = inputs.normal(8, 5000, seed=6).astype(np.float32).astype(np.float64)
    ref = Oracle(ir).eval(X, mode=MODE_F32)
    for path in ("compiled", "interp"):
        y = run(Function(ir, dtype="f32", path=path, fmad=0), X)
        np.testing.assert_array_equal(y, ref, err_msg=path)


def test_segmented_kernels_equal_single_kernel_bitwise():
    ir = programs.random_program(4000, seed=7).to_bytes()
    x = inputs.normal(64, 3000, seed=8)
    one = run(Function(ir, dtype="f64", fmad=0), x)
    for seg in (500, 1500):
        fn = Function(ir, dtype="f64", fmad=0, segment_ops=seg)
        assert fn.info.n_segments > 1
        np.testing.assert_array_equal(run(fn, x), one)


def test_interpreter_equals_compiled():
    ir = programs.random_program(3000, seed=9).to_bytes()
    x = inputs.normal(64, 2000, seed=10)
    a = run(Function(ir, dtype="f64", fmad=0), x)
    b = run(Function(ir, dtype="f64", path="interp"), x)
    np.testing.assert_allclose(b, a, rtol=1e-13, atol=1e-13)


def test_strided_buffers_and_zero_batch():
    ir = programs.cartpole_rk4().to_bytes()
    fn = Function(ir, dtype="f64")
    N = 1000
    x = inputs.cartpole(N, seed=2)
    xb = torch.zeros((5, N + 24), dtype=torch.float64, device="cuda")
    xb[:, :N] = torch.from_numpy(x)
    yb = torch.full((24, N + 40), 7.0, dtype=torch.float64, device="cuda")
    fn(xb[:, :N], out=yb[:, :N])
    torch.cuda.synchronize()
    ref = Oracle(ir).eval(x)
    np.testing.assert_allclose(yb[:, :N].cpu().numpy(), ref, rtol=1e-12, atol=1e-14)
    assert torch.all(yb[:, N:] == 7.0)                 # nothing written past N
    empty = fn(torch.zeros((5, 0), dtype=torch.float64, device="cuda"))
    assert empty.shape == (24, 0)


@pytest.mark.slow
@pytest.mark.parametrize("dtype,launch", [
    ("f64", dict(ways=0)), ("f64", dict(ways=2)), ("f64", dict(ways=4)),
    ("f64", dict(ways=4, coop_groups=2)), ("f64", dict(ways=0, maxrregcount=128)),
    ("f32", dict(ways=0)), ("f32", dict(ways=2)), ("f32", dict(ways=4)), ("f32", dict(ways=8)),
    ("f32", dict(ways=0, maxrregcount=128)), ("f32", dict(ways=0, maxrregcount=128, pair_calls=256)),
    ("f32", dict(ways=0, inst_per_thread=2))], ids=lambda v: str(v))
def test_random_20k_program_full_batch_sampled(dtype, launch):
    """The 20,000-op workload at N = 65536 in the launch configurations the
    bench's autotuner chooses from (one thread per instance, with register
    caps, paired math calls or two instances per thread; or 2, 4, 8 warps per
    group of 32 instances, 1 or 2 groups per CTA), including the ones it
    picks on GB300 (FP64: 4 warps, 2 groups; FP32: 128-register cap with
    paired calls); 256 sampled instances (and the ragged tail) are checked
    against the oracle."""
    ir = programs.random_program(20000, seed=0).to_bytes()
    N = 65536
    x = inputs.normal(64, N, seed=1)
    fn = Function(ir, dtype=dtype, **launch)
    if dtype == "f32":
        x = x.astype(np.float32).astype(np.float64)
    y = run(fn, x)
    idx = np.unique(np.concatenate([np.random.default_rng(0).choice(N, 256, replace=False),
                                    np.arange(N - 8, N)]))
    orc = Oracle(ir)
    xs = x[:, idx]
    ref = orc.eval(xs)
    kind, tau = (0, TAU64) if dtype == "f64" else (1, TAU32)
    tol = tolerance(orc, xs, ref, tau, kind=kind)
    assert_within(y[:, idx], ref, tol, dtype)
    assert np.all(np.isfinite(y))


# ---------------------------------------------------------------------------
# reverse mode
# ---------------------------------------------------------------------------
def test_adjoint_cartpole_matches_oracle_reverse_sweep():
    ir = programs.cartpole_rk4().to_bytes()
    orc = Oracle(ir)
    N = 3000
    x = inputs.cartpole(N, seed=5)
    ybar = np.random.default_rng(1).standard_normal((24, N))
    ref = orc.adjoint(x, ybar)
    for path in ("compiled", "interp"):
        fn = Function(ir, dtype="f64", path=path)
        xb = fn.adjoint(dev(x, fn), dev(ybar, fn))
        torch.cuda.synchronize()
        s = np.max(np.abs(ref), axis=1, keepdims=True)
        np.testing.assert_allclose(xb.cpu().numpy(), ref, rtol=0, atol=1e-11 * float(s.max()), err_msg=path)


def test_adjoint_broadcast_reduction_and_accumulate():
    from paper_2408_09662_gb300 import tracer as T
    from paper_2408_09662_gb300.ir import ARG_BROADCAST
    g = T.Graph()
    x = g.symbols(3)
    k = g.symbols(4)
    y = [T.sin(x[0] * k[0]) + k[1] * x[1] * x[2], T.exp(-T.sq(x[2] - k[2])) * k[3]]
    ir = T.Function([("x", x), ("k", k, ARG_BROADCAST)], [("y", y)]).to_ir().to_bytes()
    N = 5000
    rng = np.random.default_rng(3)
    X = np.vstack([rng.standard_normal((3, N)), np.tile(rng.standard_normal((4, 1)), (1, N))])
    ybar = rng.standard_normal((2, N))
    ref = Oracle(ir).adjoint(X, ybar)
    for path in ("compiled", "interp"):
        fn = Function(ir, dtype="f64", path=path)
        xd, yd = dev(X, fn), dev(ybar, fn)
        per = fn.adjoint(xd, yd).cpu().numpy()
        np.testing.assert_allclose(per, ref, rtol=1e-12, atol=1e-14, err_msg=path)
        red = fn.adjoint(xd, yd, reduce_broadcast=True).cpu().numpy()
        np.testing.assert_allclose(red[:3], ref[:3], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(red[3:, 0], ref[3:].sum(axis=1), rtol=1e-11)
        acc = torch.ones((7, N), dtype=torch.float64, device="cuda")
        fn.adjoint(xd, yd, out=acc, accumulate=True, reduce_broadcast=True)
        a = acc.cpu().numpy()
        np.testing.assert_allclose(a[:3], ref[:3] + 1, rtol=1e-12)
        np.testing.assert_allclose(a[3:, 0], ref[3:].sum(axis=1) + 1, rtol=1e-11)


def test_autograd_through_function():
    ir = programs.cartpole_rk4().to_bytes()
    fn = Function(ir, dtype="f64")
    x = torch.tensor(inputs.cartpole(64, seed=9), device="cuda", requires_grad=True)
    y = apply(fn, x)
    loss = (y[:4] ** 2).sum()
    loss.backward()
    g = x.grad.cpu().numpy()
    yn = y.detach().cpu().numpy()
    ybar = np.zeros_like(yn)
    ybar[:4] = 2 * yn[:4]
    ref = Oracle(ir).adjoint(x.detach().cpu().numpy(), ybar)
    np.testing.assert_allclose(g, ref, rtol=1e-12, atol=1e-14)


def test_stream_wait_times_out_then_completes():
    """A bounded wait: a long evaluation is still running after 1 ms (TIMEOUT,
    work left running), and a second wait with a generous limit sees it finish.
    Garbage collection is kept out of the window: freeing an earlier test's
    function (cudaFree, module unload) would synchronise the device."""
    import gc
    from paper_2408_09662_gb300 import _lib as L
    ir = programs.random_program(20000, seed=0).to_bytes()
    fn = Function(ir, dtype="f64")
    x = torch.tensor(inputs.normal(64, 65536, seed=1), device="cuda")
    y = fn(x)
    gc.collect()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream().cuda_stream
    gc.disable()
    try:
        fn(x, out=y)
        with pytest.raises(L.CusadiError) as e:
            L.cusadi_stream_wait(s, 0.001)
    finally:
        gc.enable()
    assert e.value.status == L.CUSADI_E_TIMEOUT
    L.cusadi_stream_wait(s, 60.0)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_densified_sparse_output_matches_oracle(dtype):
    """cusadi_densify: the structural non-zeros of the quadrotor step's sparse
    Jacobian land at their (row, col) and every other entry is exactly 0."""
    ir = programs.quadrotor_step_sparse_jacobian()
    fn = Function(ir.to_bytes(), dtype=dtype)
    N = 10007
    rng = np.random.default_rng(32)
    X = np.vstack([rng.uniform(-1, 1, (6, N)), rng.uniform(0, 10, (2, N))])
    if dtype == "f32":
        X = X.astype(np.float32).astype(np.float64)
    x = torch.tensor(X, dtype=fn.torch_dtype, device="cuda")
    y = fn(x)
    D = fn.dense(y, 1)
    Dx = fn.dense(y, 0)
    torch.cuda.synchronize()
    D, Dx, y = D.double().cpu().numpy(), Dx.double().cpu().numpy(), y.double().cpu().numpy()
    sp = ir.outputs[1]
    mask = np.zeros((6, 8), bool)
    for r in range(6):
        for q in range(sp.rowptr[r], sp.rowptr[r + 1]):
            assert np.array_equal(D[r, sp.col[q]], y[6 + q])    # a copy, bit for bit
            mask[r, sp.col[q]] = True
    assert np.all(D[~mask] == 0.0)
    np.testing.assert_array_equal(Dx[:, 0], y[:6])
    orc = Oracle(ir.to_bytes())
    idx = np.random.default_rng(33).choice(N, 64, replace=False)
    ref = orc.eval(X[:, idx])
    tol = tolerance(orc, X[:, idx], ref, 1e-12 if dtype == "f64" else 2e-4, kind=0 if dtype == "f64" else 1)
    assert np.all(np.abs(y[:, idx] - ref) <= tol)


def test_concurrent_calls_on_different_streams():
    """A segmented program (kernels pass values through the workspace) called
    on eight streams at once: each call gets its own workspace from the
    stream-ordered allocator, so every chunk equals the single-call result."""
    ir = programs.quadrotor_mpc().to_bytes()
    fn = Function(ir, dtype="f64")
    assert fn.info.n_segments >= 2
    N = 16384
    rng = np.random.default_rng(40)
    X = np.vstack([rng.uniform(-0.5, 0.5, (6, N)), rng.uniform(-1, 1, (2, N))])
    x = torch.tensor(X, device="cuda")
    ref = fn(x)
    y = torch.empty_like(ref)
    streams = [torch.cuda.Stream() for _ in range(8)]
    cur = torch.cuda.current_stream()
    start = torch.cuda.Event()
    start.record(cur)
    ch = N // 8
    for c, st in enumerate(streams):
        st.wait_stream(cur)
        with torch.cuda.stream(st):
            fn(x[:, c * ch:(c + 1) * ch], out=y[:, c * ch:(c + 1) * ch])
    for st in streams:
        cur.wait_stream(st)
    torch.cuda.synchronize()
    assert torch.equal(y, ref)


@pytest.mark.parametrize("ways", [0, 4])
def test_debug_checks_count_non_finite_results(ways):
    """debug_checks=1: log and sqrt of negative inputs give NaN; the kernels
    count every non-finite value they store, cusadi_debug_count reads and
    resets the counter, and finite results count nothing."""
    from paper_2408_09662_gb300 import tracer as T
    g = T.Graph()
    x = g.symbols(2)
    ir = T.Function([("x", x)], [("y", [T.log(x[0]), T.sqrt(x[1]), x[0] * x[1]])]).to_ir().to_bytes()
    fn = Function(ir, dtype="f64", debug_checks=1, ways=ways)
    N = 5000
    X = np.ones((2, N))
    X[0, :37] = -1.0                       # log(-1) = NaN
    X[1, 100:112] = -4.0                   # sqrt(-4) = NaN
    X[0, 200] = 0.0                        # log(0) = -inf
    x_d = torch.tensor(X, device="cuda")
    y = fn(x_d)
    assert fn.debug_count() == 37 + 12 + 1
    assert np.isnan(y.cpu().numpy()[0, :37]).all()
    assert fn.debug_count() == 0           # read and reset
    fn(torch.ones((2, N), dtype=torch.float64, device="cuda"), out=y)
    assert fn.debug_count() == 0


@pytest.mark.parametrize("path,ways", [("compiled", 0), ("interp", 0), ("compiled", 2)])
def test_degenerate_programs(path, ways):
    """Outputs that are a constant, a copy of an input and a product; one
    instance and a ragged batch; a program whose inputs are all broadcast,
    read from a one-column buffer (ld_in = 1), gives the same value everywhere."""
    from paper_2408_09662_gb300 import tracer as T
    from paper_2408_09662_gb300.ir import ARG_BROADCAST
    g = T.Graph()
    x = g.symbols(2)
    ir = T.Function([("x", x)], [("y", [2.5, x[1], x[0] * x[1]])]).to_ir().to_bytes()
    fn = Function(ir, dtype="f64", path=path, ways=ways)
    for N in (1, 37):
        X = np.random.default_rng(N).standard_normal((2, N))
        y = fn(torch.tensor(X, device="cuda")).cpu().numpy()
        np.testing.assert_array_equal(y[0], np.full(N, 2.5))
        np.testing.assert_array_equal(y[1], X[1])
        np.testing.assert_array_equal(y[2], X[0] * X[1])
    g = T.Graph()
    k = g.symbols(2)
    irb = T.Function([("k", k, ARG_BROADCAST)], [("y", [T.sin(k[0]) * k[1]])]).to_ir().to_bytes()
    fb = Function(irb, dtype="f64", path=path, ways=ways)
    kk = torch.tensor([[0.5], [3.0]], dtype=torch.float64, device="cuda")        # [2, 1]
    out = torch.empty((1, 100), dtype=torch.float64, device="cuda")
    from paper_2408_09662_gb300 import _lib as L
    L.cusadi_eval(fb._fn, kk.data_ptr(), 1, out.data_ptr(), 100, 100,
                  0, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert np.allclose(out.cpu().numpy(), np.sin(0.5) * 3.0, rtol=1e-15, atol=0)
    assert len(set(out.cpu().numpy().ravel().tolist())) == 1
