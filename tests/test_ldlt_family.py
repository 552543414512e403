"""The §IV benchmark family: LDL^T solutions of SPD systems of growing size
(about ten times more operations each), pinned against LAPACK."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2408_09662_gb300 import programs
from paper_2408_09662_gb300.ir import ProgramIR


def spd_inputs(n, N, seed=0):
    """Random SPD matrices A = M M' / n + I (lower triangles, row-major) and b."""
    rng = np.random.default_rng(seed)
    Ms = rng.standard_normal((N, n, n))
    A = Ms @ Ms.transpose(0, 2, 1) / n + np.eye(n)
    il = np.tril_indices(n)
    low = A[:, il[0], il[1]].T
    b = rng.standard_normal((n, N))
    return np.vstack([low, b]), A, b


@pytest.mark.parametrize("n", programs.LDLT_SIZES[:4])
def test_ldlt_solution_matches_lapack(n):
    ir = programs.ldlt_spd_solve(n)
    assert ir.inputs[0].nrow == n and ir.inputs[0].nnz == n * (n + 1) // 2   # lower-triangular pattern
    X, A, b = spd_inputs(n, 6, seed=n)
    x = Oracle(ir.to_bytes()).eval(X)
    for i in range(6):
        ref = np.linalg.solve(A[i], b[:, i])
        np.testing.assert_allclose(x[:, i], ref, rtol=1e-11, atol=1e-12)


def test_family_grows_about_tenfold():
    ops = [programs.ldlt_spd_solve(n).count_ops() for n in programs.LDLT_SIZES[:4]]
    ratios = [b / a for a, b in zip(ops, ops[1:])]
    assert all(5 < r < 12 for r in ratios), ops
