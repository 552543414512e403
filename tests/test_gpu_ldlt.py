"""GPU parity of the §IV LDL^T benchmark family (FP64).  The largest member
(~363k ops) exceeds the default compile limit, so AUTO evaluates it with the
interpreter kernel; the one-launch-per-op comparator must agree too."""
import numpy as np
import pytest
import torch

from oracle import Oracle, tolerance
from paper_2408_09662_gb300 import programs
from paper_2408_09662_gb300.api import Function
from paper_2408_09662_gb300.experiments import _spd
from paper_2408_09662_gb300.vectorized import VectorizedProgram

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", programs.LDLT_SIZES)
def test_ldlt_family_parity(n):
    ir = programs.ldlt_spd_solve(n)
    irb = ir.to_bytes()
    N = 2048 if n < 100 else 256
    X = _spd(n, N, seed=n)
    fn = Function(irb, dtype="f64")
    assert fn.compiled == (n < 100)
    y = fn(torch.tensor(X, device="cuda")).cpu().numpy()
    orc = Oracle(irb)
    idx = np.arange(0, N, max(1, N // 32))
    ref = orc.eval(X[:, idx])
    tol = tolerance(orc, X[:, idx], ref, 1e-12, kind=0)
    assert np.all(np.abs(y[:, idx] - ref) <= tol)
    if n <= 22:
        v = VectorizedProgram(ir)(torch.tensor(X, device="cuda")).cpu().numpy()
        np.testing.assert_allclose(v, y, rtol=1e-9, atol=1e-12)
