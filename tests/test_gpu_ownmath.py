"""Accuracy of the engine's own FP32 sin, cos and exp (compiled path,
own_math = 1) against the FP64 oracle on float inputs: at most 2 ulp, the
bound the tolerance tables assume for these ops, with IEEE special values
(NaN, +-inf, signed zero, overflow, underflow) handled like libm."""
import numpy as np
import pytest
import torch

from oracle import Oracle
from paper_2408_09662_gb300 import programs
from paper_2408_09662_gb300.api import Function
from paper_2408_09662_gb300.ir import Op

pytestmark = pytest.mark.gpu


def ulp_error(y, ref):
    ref32 = ref.astype(np.float32)
    e = np.floor(np.log2(np.maximum(np.abs(ref32.astype(np.float64)), np.finfo(np.float32).tiny)))
    ulp = np.ldexp(1.0, (e - 23).astype(int))
    return np.abs(y - ref) / ulp


def sweep(op):
    rng = np.random.default_rng(int(op))
    if op == Op.EXP:
        dense = np.linspace(-110, 95, 1 << 21)
        special = [0.0, -0.0, 1e-30, -1e-30, 88.72, 88.73, -87.3, -103.9, -104.5, np.inf, -np.inf, np.nan]
    else:
        dense = np.concatenate([np.linspace(-260, 260, 1 << 21), rng.uniform(-1e5, 1e5, 1 << 16)])
        k = np.arange(-128, 129)
        near = (k * np.pi / 2)[:, None] + np.array([-1e-6, 0.0, 1e-6])[None, :]
        special = list(near.ravel()) + [0.0, -0.0, 1e-30, 201.0, -201.0, 201.1, np.inf, -np.inf, np.nan]
    x = np.concatenate([dense, np.array(special)]).astype(np.float32).astype(np.float64)
    return x[None, :]


@pytest.mark.parametrize("op", [Op.SIN, Op.COS, Op.EXP], ids=lambda o: o.name)
def test_own_fp32_math_within_two_ulp(op):
    ir = programs.single_op(op).to_bytes()
    fn = Function(ir, dtype="f32", own_math=1)
    assert "cs_own_" in fn.source()
    x = sweep(op)
    y = fn(torch.tensor(x, dtype=torch.float32, device="cuda")).double().cpu().numpy()[0]
    ref = Oracle(ir).eval(x)[0]
    fin = np.isfinite(ref) & (np.abs(ref) < np.finfo(np.float32).max)
    nz = fin & (np.abs(ref) >= np.finfo(np.float32).tiny)
    err = ulp_error(y[nz], ref[nz])
    assert err.max() <= 2.0, (float(err.max()), float(x[0, nz][np.argmax(err)]))
    # subnormal and zero results: absolute error within one subnormal step
    sub = fin & ~nz
    assert np.all(np.abs(y[sub] - ref[sub]) <= 2.0 ** -149)
    # specials behave like libm after rounding to float
    ref32 = ref.astype(np.float32).astype(np.float64)
    spec = ~fin
    np.testing.assert_array_equal(np.isnan(y[spec]), np.isnan(ref32[spec]))
    np.testing.assert_array_equal(y[spec & ~np.isnan(ref)], ref32[spec & ~np.isnan(ref)])
