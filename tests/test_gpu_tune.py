"""The launch-configuration autotuner: it keeps the fastest candidate it timed,
the kernel it returns computes what the default kernel computes (bit for bit
with contraction off), and a second call with the same program, GPU, dtype and
batch size takes the choice from the on-disk cache without timing anything."""
import json
import os

import numpy as np
import pytest
import torch

from oracle import Oracle, tolerance
from paper_2408_09662_gb300 import inputs, programs
from paper_2408_09662_gb300.api import Function
from paper_2408_09662_gb300.tune import autotune

pytestmark = pytest.mark.gpu


def test_autotune_keeps_the_fastest_and_caches_it(tmp_path):
    ir = programs.cartpole_rk4().to_bytes()
    N = 4099
    xn = inputs.cartpole(N, seed=71)
    x = torch.tensor(xn, device="cuda")
    fn = autotune(ir, x, "f64", ways=(0, 4), cache_dir=str(tmp_path), reps=3, fmad=0)
    rec = fn.tune_record
    assert not rec["from_cache"]
    times = [ms for _, ms in rec["candidates"]]
    assert rec["ms"] == min(times) and len(times) >= 3        # both shapes, then refinements
    assert rec["candidates"][0][0] == rec["options"]
    y = fn(x)
    ref = Function(ir, dtype="f64", fmad=0)(x)
    torch.cuda.synchronize()
    assert torch.equal(y, ref)
    orc = Oracle(ir)
    r = orc.eval(xn)
    assert np.all(np.abs(y.cpu().numpy() - r) <= tolerance(orc, xn, r, 1e-12, kind=0))
    # the record is on disk, keyed by program, GPU, dtype, batch size and fixed options
    db = json.load(open(os.path.join(str(tmp_path), "tuning.json")))
    assert len(db) == 1 and next(iter(db.values()))["options"] == rec["options"]
    again = autotune(ir, x, "f64", ways=(0, 4), cache_dir=str(tmp_path), fmad=0)
    assert again.tune_record["from_cache"] and again.tune_record["options"] == rec["options"]
    assert torch.equal(again(x), ref)
    # another batch size bucket or fixed option is another entry
    autotune(ir, x[:, :1000].contiguous(), "f64", ways=(0,), refine=False, cache_dir=str(tmp_path), fmad=0)
    assert len(json.load(open(os.path.join(str(tmp_path), "tuning.json")))) == 2


def test_autotune_on_the_reverse_sweep(tmp_path):
    """With ybar the candidates are timed on the adjoint; the chosen Function's
    reverse sweep matches the oracle's, and the record is kept apart from the
    forward choice of the same program."""
    ir = programs.srb_step().to_bytes()
    rng = np.random.default_rng(73)
    N = 2051
    X = np.vstack([np.tile(rng.normal(0, 0.1, (144, 1)), (1, N)), rng.uniform(-0.1, 0.1, (12, N)),
                   np.zeros((1, N))])
    ybar = rng.standard_normal((13, N))
    x, yb = torch.tensor(X, device="cuda"), torch.tensor(ybar, device="cuda")
    fn = autotune(ir, x, "f64", ways=(0, 4), cache_dir=str(tmp_path), reps=3, ybar=yb,
                  adjoint_kw=dict(reduce_broadcast=True))
    rec = fn.tune_record
    assert rec["target"] == "adjoint(reduce_broadcast=True)" and rec["ms"] == min(t for _, t in rec["candidates"])
    got = fn.adjoint(x, yb, reduce_broadcast=True).cpu().numpy()
    ref = Oracle(ir).adjoint(X, ybar)
    np.testing.assert_allclose(got[144:], ref[144:], rtol=0, atol=1e-12 * np.max(np.abs(ref[144:])))
    red = ref[:144].sum(axis=1)
    np.testing.assert_allclose(got[:144, 0], red, rtol=1e-11, atol=1e-12 * np.max(np.abs(red)))
    fwd = autotune(ir, x, "f64", ways=(0,), refine=False, cache_dir=str(tmp_path), reps=3)
    assert fwd.tune_record["target"] == "eval"
    assert len(json.load(open(os.path.join(str(tmp_path), "tuning.json")))) == 2
