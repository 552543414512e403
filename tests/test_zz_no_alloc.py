"""cusadi_eval_noalloc: evaluation for callers that cannot allocate device
memory once they run (a real-time control loop under a no-allocation rule, a
plugin whose host application owns all device memory).  Its workspace is the
library's static scratch array.

Two programs exercise both layouts of that workspace: a random program split
into several compiled kernels, whose carried values go through the array, and
an LDL^T solve on the interpreter path with more work slots than shared memory
holds, whose work vector lives in the array ([slots x round_up(N, 128)]).  Two
calls in a row must match cusadi_eval on the same inputs within the FP64 parity
tolerance of the other GPU tests (1e-12 relative to each output row's
magnitude).  This file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

from paper_2408_09662_gb300 import _lib as L
from paper_2408_09662_gb300 import inputs, programs
from paper_2408_09662_gb300.api import Function

pytestmark = pytest.mark.gpu


def test_noalloc_matches_eval_on_two_calls_in_a_row():
    fn = Function(programs.random_program(3000, seed=41), dtype="f64", segment_ops=600)
    assert fn.info.n_segments >= 3
    N = 4099
    assert 0 < L.cusadi_workspace_bytes(fn.handle, N, False) <= L.CUSADI_NOALLOC_SCRATCH_BYTES
    x = torch.tensor(inputs.normal(64, N, seed=42), device="cuda")
    ref = fn(x)                                   # cusadi_eval (also loads the kernels)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        y = torch.full_like(ref, float("nan"))
        L.cusadi_eval_noalloc(fn.handle, x.data_ptr(), x.stride(0), y.data_ptr(), y.stride(0), N,
                              stream)
        torch.cuda.synchronize()
        r, a = ref.cpu().numpy(), y.cpu().numpy()
        tol = 1e-12 * np.max(np.abs(r), axis=1, keepdims=True)
        assert np.all(np.abs(a - r) <= tol), f"call {call}"


def test_noalloc_rejects_batches_beyond_the_scratch_size():
    fn = Function(programs.random_program(3000, seed=43), dtype="f64", segment_ops=600)
    per_instance = L.cusadi_workspace_bytes(fn.handle, 32, False) / 32
    N = int(L.CUSADI_NOALLOC_SCRATCH_BYTES / per_instance) + 4096
    assert L.cusadi_workspace_bytes(fn.handle, N, False) > L.CUSADI_NOALLOC_SCRATCH_BYTES
    # real buffers of the full size: the call must be refused on the host
    x = torch.zeros((64, N), dtype=torch.float64, device="cuda")
    y = torch.zeros((32, N), dtype=torch.float64, device="cuda")
    fn(x[:, :1].contiguous())                     # loads the kernels on this device
    with pytest.raises(L.CusadiError) as e:
        L.cusadi_eval_noalloc(fn.handle, x.data_ptr(), N, y.data_ptr(), N, N,
                              torch.cuda.current_stream().cuda_stream)
    assert e.value.status == L.CUSADI_E_INVALID_ARG and "scratch" in str(e.value)


def test_noalloc_interpreter_with_work_slots_in_the_scratch():
    from paper_2408_09662_gb300.experiments import _spd
    fn = Function(programs.ldlt_spd_solve(47), dtype="f64", path="interp")
    assert not fn.compiled and fn.info.n_slots > 1000   # far more slots than shared memory holds
    N = 4099
    assert 0 < L.cusadi_workspace_bytes(fn.handle, N, False) <= L.CUSADI_NOALLOC_SCRATCH_BYTES
    x = torch.tensor(_spd(47, N, seed=47), device="cuda")
    ref = fn(x)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        y = torch.full_like(ref, float("nan"))
        L.cusadi_eval_noalloc(fn.handle, x.data_ptr(), x.stride(0), y.data_ptr(), y.stride(0), N,
                              stream)
        torch.cuda.synchronize()
        r, a = ref.cpu().numpy(), y.cpu().numpy()
        tol = 1e-12 * np.max(np.abs(r), axis=1, keepdims=True)
        assert np.all(np.abs(a - r) <= tol), f"call {call}"
