"""Host-buffer evaluation (cusadi_eval_host): chunks copied in, evaluated and
copied out on the library's own streams give exactly the device-buffer
results — every chunk count, ragged chunks, broadcast input rows, segmented
programs (workspace), the interpreter path, pinned and pageable host memory."""
import numpy as np
import pytest
import torch

from paper_2408_09662_gb300 import inputs, programs
from paper_2408_09662_gb300.api import Function

pytestmark = pytest.mark.gpu


def _device(fn, X):
    x = torch.tensor(X, dtype=fn.torch_dtype, device="cuda")
    y = fn(x)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("chunks", [0, 1, 3, 7])
@pytest.mark.parametrize("pinned", [True, False])
def test_cartpole_host_matches_device(chunks, pinned):
    fn = Function(programs.cartpole_rk4(), dtype="f64")
    N = 70001                                  # not a multiple of 32 or of any chunk count
    X = inputs.cartpole(N, seed=3)
    xh = torch.tensor(X)
    if pinned:
        xh = xh.pin_memory()
    y = fn.eval_host(xh, chunks=chunks)
    np.testing.assert_array_equal(y.numpy(), _device(fn, X))


def test_broadcast_rows_reach_every_chunk():
    """The SRB step's 144 gain entries are broadcast rows (read at column 0
    only): each chunk must see them."""
    fn = Function(programs.srb_step(), dtype="f64")
    N = 5000
    rng = np.random.default_rng(4)
    X = np.vstack([np.zeros((144, N)), rng.uniform(-0.1, 0.1, (12, N)), np.zeros((1, N))])
    X[:144, 0] = rng.normal(0, 0.1, 144)       # only column 0 of a broadcast row is read
    y = fn.eval_host(torch.tensor(X).pin_memory(), chunks=3)
    Xd = X.copy()
    Xd[:144] = X[:144, :1]                     # device reference: same values everywhere
    np.testing.assert_array_equal(y.numpy(), _device(fn, Xd))


def test_segmented_program_with_workspace():
    ir = programs.random_program(3000, n_in=16, n_out=8, seed=5).to_bytes()
    fn = Function(ir, dtype="f32", segment_ops=700)
    assert fn.info.n_segments >= 3
    N = 40000
    X = inputs.normal(16, N, seed=6).astype(np.float32)
    y = fn.eval_host(torch.tensor(X).pin_memory(), chunks=4)
    np.testing.assert_array_equal(y.numpy(), _device(fn, X))


def test_interpreter_path_and_tiny_batches():
    ir = programs.random_program(2000, seed=8).to_bytes()
    fn = Function(ir, dtype="f64", path="interp")
    for N in (1, 5, 33, 1000):
        X = inputs.normal(64, N, seed=N)
        y = fn.eval_host(torch.tensor(X), chunks=4)
        np.testing.assert_array_equal(y.numpy(), _device(fn, X))


def test_asynchronous_call_orders_with_the_stream():
    """sync=False: the result is valid after the current stream's event."""
    fn = Function(programs.cartpole_rk4(), dtype="f64")
    N = 65536
    X = inputs.cartpole(N, seed=9)
    xh = torch.tensor(X).pin_memory()
    out = torch.empty((24, N), dtype=torch.float64).pin_memory()
    fn.eval_host(xh, out=out, sync=False)
    ev = torch.cuda.Event()
    ev.record()
    ev.synchronize()
    np.testing.assert_array_equal(out.numpy(), _device(fn, X))


@pytest.mark.parametrize("chunks", [2, 5])
def test_segmented_mpc_chunks_run_concurrently(chunks):
    """The MPC program passes values between its two kernels through the
    workspace; concurrent chunks use disjoint columns of it."""
    fn = Function(programs.quadrotor_mpc().to_bytes(), dtype="f64")
    assert fn.info.n_segments >= 2
    N = 20000
    rng = np.random.default_rng(41)
    X = np.vstack([rng.uniform(-0.5, 0.5, (6, N)), rng.uniform(-1, 1, (2, N))])
    y = fn.eval_host(torch.tensor(X).pin_memory(), chunks=chunks)
    np.testing.assert_array_equal(y.numpy(), _device(fn, X))


def test_interpreter_with_global_workspace_chunks():
    """A work vector too long for shared memory: the interpreter keeps it in the
    workspace, 128-column grain per chunk."""
    ir = programs.ldlt_spd_solve(47).to_bytes()        # 1,176 live slots
    fn = Function(ir, dtype="f64", path="interp")
    assert fn.workspace(1000) is not None
    N = 3000
    rng = np.random.default_rng(10)
    X = rng.uniform(-1, 1, (fn.nnz_in, N))
    X[[k * (k + 3) // 2 for k in range(47)]] += 60.0      # diagonal entries: diagonally dominant
    y = fn.eval_host(torch.tensor(X).pin_memory(), chunks=3)
    np.testing.assert_array_equal(y.numpy(), _device(fn, X))
