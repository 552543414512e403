"""Batched launch: several random programs of uneven length and instance count
in one persistent, graph-replayed kernel.

Checks: persistent == plain launches bit for bit (same per-instance code);
every program against the FP64 oracle under the FP32 rule
max(2e-4 * s_k, 2 * B32_k,i); every tile size; ragged instance counts.
"""
import numpy as np
import pytest
import torch

from oracle import Oracle, tolerance
from paper_2408_09662_gb300 import inputs, programs
from paper_2408_09662_gb300.api import Batch, Function

pytestmark = pytest.mark.gpu

SIZES = [(300, 3000), (2500, 1000), (6000, 70), (1200, 33)]


@pytest.fixture(scope="module")
def batch():
    irs = [programs.random_program(n, seed=100 + j).to_bytes() for j, (n, _) in enumerate(SIZES)]
    b = Batch(irs, [N for _, N in SIZES], dtype="f32", segment_ops=2000)
    return irs, b


def _buffers(irs):
    xs, outs, xn = [], [], []
    for j, (n, N) in enumerate(SIZES):
        x = inputs.normal(64, N, seed=200 + j).astype(np.float32).astype(np.float64)
        xn.append(x)
        xs.append(torch.tensor(x, dtype=torch.float32, device="cuda"))
        outs.append(torch.full((32, N), float("nan"), dtype=torch.float32, device="cuda"))
    return xs, outs, xn


def test_persistent_equals_plain_and_oracle(batch):
    irs, b = batch
    xs, outs, xn = _buffers(irs)
    for block in (32, 64, 128):
        b.set_block(block)
        b(xs, outs, mode="persistent")
        torch.cuda.synchronize()
        pers = [o.double().cpu().numpy() for o in outs]
        for o in outs:
            o.fill_(float("nan"))
        b(xs, outs, mode="plain")
        torch.cuda.synchronize()
        plain = [o.double().cpu().numpy() for o in outs]
        for j in range(len(SIZES)):
            np.testing.assert_array_equal(pers[j], plain[j], err_msg=f"program {j} block {block}")
    for j in range(len(SIZES)):
        orc = Oracle(irs[j])
        ref = orc.eval(xn[j])
        tol = tolerance(orc, xn[j], ref, 2e-4, kind=1)
        bad = ~(np.abs(pers[j] - ref) <= tol)
        assert not np.any(bad), (j, int(bad.sum()))


def test_repeated_launches_and_buffer_changes(batch):
    irs, b = batch
    xs, outs, _ = _buffers(irs)
    b(xs, outs)
    torch.cuda.synchronize()
    first = [o.clone() for o in outs]
    for _ in range(3):                       # graph replay with the same buffers
        b(xs, outs)
    torch.cuda.synchronize()
    for a, c in zip(first, outs):
        assert torch.equal(a, c)
    outs2 = [torch.zeros_like(o) for o in outs]   # new buffers: table re-uploaded
    b(xs, outs2)
    torch.cuda.synchronize()
    for a, c in zip(first, outs2):
        assert torch.equal(a, c)


def test_tune_picks_a_tile_size(batch):
    irs, b = batch
    xs, outs, _ = _buffers(irs)
    blk = b.tune(xs, outs, reps=2)
    assert blk in (32, 64, 128) and b.info()["block"] == blk and b.info()["grid"] > 0


COOP_SIZES = [(70000, 200), (3000, 2000), (500, 5000)]


def test_cooperative_tiles_equal_plain_launches():
    """ways=4: the 70k-op program (few instances, many ops) runs as cooperative
    tiles: the 128-thread scheduler's 4 warps split one group of 32 instances,
    and its per-program launch runs the same cooperative code.  With FMA
    contraction off every op rounds once in any layout, so the persistent
    launch, the plain launches and the standalone one-thread-per-instance
    kernel agree bit for bit; 32- and 64-thread tiles are refused.  The 70k-op
    random program is too deep to compare with the oracle (two correct FP64
    evaluations of it drift apart by O(1) in its last outputs); the regular
    programs meet the FP64 rule against the oracle."""
    irs = [programs.random_program(n, seed=300 + j).to_bytes() for j, (n, _) in enumerate(COOP_SIZES)]
    b = Batch(irs, [N for _, N in COOP_SIZES], dtype="f64", ways=4, fmad=0)
    xn = [inputs.normal(64, N, seed=400 + j) for j, (_, N) in enumerate(COOP_SIZES)]
    xs = [torch.tensor(x, dtype=torch.float64, device="cuda") for x in xn]
    outs = [torch.full((32, N), float("nan"), dtype=torch.float64, device="cuda") for _, N in COOP_SIZES]
    b(xs, outs, mode="plain")
    torch.cuda.synchronize()
    plain = [o.cpu().numpy() for o in outs]
    with pytest.raises(Exception):
        b.set_block(32)
    for _ in range(2):
        for o in outs:
            o.fill_(float("nan"))
        b(xs, outs, mode="persistent")
        torch.cuda.synchronize()
        for j in range(len(COOP_SIZES)):
            np.testing.assert_array_equal(outs[j].cpu().numpy(), plain[j], err_msg=f"program {j}")
    alone = Function(irs[0], dtype="f64", fmad=0)(xs[0])
    torch.cuda.synchronize()
    np.testing.assert_array_equal(plain[0], alone.cpu().numpy())
    for j in (1, 2):
        orc = Oracle(irs[j])
        idx = np.random.default_rng(j).choice(COOP_SIZES[j][1], 40, replace=False)
        ref = orc.eval(xn[j][:, idx])
        tol = tolerance(orc, xn[j][:, idx], ref, 1e-12, kind=0)
        assert np.all(np.abs(plain[j][:, idx] - ref) <= tol)


# the uneven batch as the benchmark states it: 8 random programs of the 20k-op
# generator, program seeds 100..107, input seeds 200..207
C5_SIZES = [(1000, 65536), (5000, 32768), (10000, 32768), (20000, 16384), (50000, 8192),
            (100000, 4096), (150000, 2048), (200000, 512)]


def test_uneven_batch_at_stated_sizes_against_the_oracle():
    """FP32, one persistent launch with cooperative tiles for the longest
    programs (ways = 4), every program at its stated instance count.  Sampled
    instances (64 per program plus the last, ragged, one) against the FP64
    oracle under the FP32 rule max(2e-4 s_k, 2 B32_k,i, 4 S_k): B32 is the
    first-order rounding bound, S_k the largest deviation of 8 Monte Carlo
    arithmetic runs at FP32 sizes on output row k.  Past ~20k ops most outputs
    keep no correct float digit (S_k reaches s_k), so only S_k can judge them;
    the fraction of outputs within the plain 2e-4 s_k is recorded and must
    fall with depth as the oracle says it does."""
    irs = [programs.random_program(n, seed=100 + j).to_bytes() for j, (n, _) in enumerate(C5_SIZES)]
    b = Batch(irs, [N for _, N in C5_SIZES], dtype="f32", ways=4)
    xn = [inputs.normal(64, N, seed=200 + j).astype(np.float32).astype(np.float64)
          for j, (_, N) in enumerate(C5_SIZES)]
    xs = [torch.tensor(x, dtype=torch.float32, device="cuda") for x in xn]
    outs = [torch.full((32, N), float("nan"), dtype=torch.float32, device="cuda") for _, N in C5_SIZES]
    b(xs, outs, mode="persistent")
    torch.cuda.synchronize()
    frac_tau = []
    for j, (n, N) in enumerate(C5_SIZES):
        idx = np.unique(np.r_[np.random.default_rng(j).choice(N, 64, replace=False), N - 1])
        got = outs[j][:, idx].double().cpu().numpy()
        assert np.all(np.isfinite(got)), j
        orc = Oracle(irs[j])
        ref = orc.eval(xn[j][:, idx])
        tol = tolerance(orc, xn[j][:, idx], ref, 2e-4, kind=1, mca_runs=8)
        err = np.abs(got - ref)
        bad = err > tol
        assert not np.any(bad), (n, int(bad.sum()), float(np.max(err / tol)))
        s = np.max(np.abs(ref), axis=1, keepdims=True)
        frac_tau.append(float(np.mean(err <= 2e-4 * s)))
    # shallow programs meet the plain tolerance everywhere, the deepest almost nowhere
    assert frac_tau[0] == 1.0 and frac_tau[1] == 1.0, frac_tau
    assert frac_tau[-1] < 0.2, frac_tau
