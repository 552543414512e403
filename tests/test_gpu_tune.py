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
