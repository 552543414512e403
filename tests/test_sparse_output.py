"""Sparse outputs (§II-A): the quadrotor step's Jacobian stored as its
structural non-zeros.  The pattern the library reports is the tracer's, bit
for bit; the oracle's non-zeros, scattered by that pattern, equal the
hand-derived dense Jacobian, and the entries left out are exactly the ones
that vanish identically."""
import numpy as np

from oracle import Oracle
from oracle import models as M
from paper_2408_09662_gb300 import _lib as L
from paper_2408_09662_gb300 import programs


def scatter(sp, nz):
    """Dense [nrow, ncol, N] from CSR non-zeros [nnz, N] (test-side helper)."""
    d = np.zeros((sp.nrow, sp.ncol, nz.shape[1]))
    for r in range(sp.nrow):
        for p in range(sp.rowptr[r], sp.rowptr[r + 1]):
            d[r, sp.col[p]] = nz[p]
    return d


def test_library_reports_the_tracers_pattern():
    ir = programs.quadrotor_step_sparse_jacobian()
    fn = L.cusadi_load(ir.to_bytes())
    try:
        for j, sp in enumerate(ir.outputs):
            a = L.cusadi_arg_info(fn, True, j)
            assert (a.nrow, a.ncol, a.nnz) == (sp.nrow, sp.ncol, sp.nnz)
            assert [a.rowptr[k] for k in range(sp.nrow + 1)] == list(sp.rowptr)
            assert [a.col[k] for k in range(sp.nnz)] == list(sp.col)
        assert L.cusadi_arg_info(fn, True, 1).row_offset == 6
    finally:
        L.cusadi_free(fn)


def test_sparse_jacobian_equals_hand_derived_dense():
    ir = programs.quadrotor_step_sparse_jacobian()
    p = M.QUAD
    rng = np.random.default_rng(31)
    N = 12
    X = np.vstack([rng.uniform(-1, 1, (6, N)), rng.uniform(0, 10, (2, N))])
    y = Oracle(ir.to_bytes()).eval(X)
    sp = ir.outputs[1]
    assert sp.nnz == 25                       # of 48 entries
    J = scatter(sp, y[6:])
    for i in range(N):
        A, B = M.quad_step_jac(X[:6, i], X[6:, i], p)
        dense = np.hstack([A, B])
        np.testing.assert_allclose(J[:, :, i], dense, rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(y[:6, i], M.quad_step(X[:6, i], X[6:, i], p), rtol=1e-14, atol=1e-15)
    # left-out entries vanish identically; kept ones are non-zero at a generic point
    A, B = M.quad_step_jac(X[:6, 0], X[6:, 0], p)
    mask = np.zeros((6, 8), bool)
    for r in range(6):
        mask[r, sp.col[sp.rowptr[r]:sp.rowptr[r + 1]]] = True
    assert np.array_equal(mask, np.hstack([A, B]) != 0)
