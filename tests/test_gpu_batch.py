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


COOP_SIZES = [(70000, 200), (3000, 2000), (500, 5000), (45000, 4099)]


@pytest.mark.parametrize("ways", [4, 8])
def test_satellites_equal_plain_launches(ways):
    """ways = W: the 70k- and 45k-op programs (few instances, many ops) run as
    satellite kernels, W warps splitting each group of 32 instances, beside
    the persistent kernel of the others; the plain mode launches the same
    kernels.  With FMA contraction off every op rounds once in any layout, so
    the persistent launch, the plain launches and the standalone
    one-thread-per-instance kernel agree bit for bit, for every tile size and
    after the buffers change (the satellites' graph branches are captured
    again).  The 70k-op random program is too deep for the FP64 parity rule
    (two correct FP64 evaluations of it drift apart by O(1) in its last
    outputs); the others meet it against the oracle."""
    irs = [programs.random_program(n, seed=300 + j).to_bytes() for j, (n, _) in enumerate(COOP_SIZES)]
    b = Batch(irs, [N for _, N in COOP_SIZES], dtype="f64", ways=ways, fmad=0)
    xn = [inputs.normal(64, N, seed=400 + j) for j, (_, N) in enumerate(COOP_SIZES)]
    xs = [torch.tensor(x, dtype=torch.float64, device="cuda") for x in xn]
    outs = [torch.full((32, N), float("nan"), dtype=torch.float64, device="cuda") for _, N in COOP_SIZES]
    b(xs, outs, mode="plain")
    torch.cuda.synchronize()
    plain = [o.cpu().numpy() for o in outs]
    for block in (32, 64, 128):
        b.set_block(block)
        for _ in range(2):
            for o in outs:
                o.fill_(float("nan"))
            b(xs, outs, mode="persistent")
            torch.cuda.synchronize()
            for j in range(len(COOP_SIZES)):
                np.testing.assert_array_equal(outs[j].cpu().numpy(), plain[j], err_msg=f"program {j}")
    outs2 = [torch.zeros_like(o) for o in outs]          # new buffers: graph captured again
    b(xs, outs2)
    torch.cuda.synchronize()
    for j in range(len(COOP_SIZES)):
        np.testing.assert_array_equal(outs2[j].cpu().numpy(), plain[j], err_msg=f"program {j}")
    for j in (0, 3):
        alone = Function(irs[j], dtype="f64", fmad=0)(xs[j])
        torch.cuda.synchronize()
        np.testing.assert_array_equal(plain[j], alone.cpu().numpy())
    for j in (1, 2, 3):
        orc = Oracle(irs[j])
        idx = np.unique(np.r_[np.random.default_rng(j).choice(COOP_SIZES[j][1], 40, replace=False),
                              COOP_SIZES[j][1] - 1])
        ref = orc.eval(xn[j][:, idx])
        tol = tolerance(orc, xn[j][:, idx], ref, 1e-12, kind=0)
        assert np.all(np.abs(plain[j][:, idx] - ref) <= tol)


# the uneven batch as the benchmark states it: 8 random programs of the 20k-op
# generator, program seeds 100..107, input seeds 200..207
C5_SIZES = [(1000, 65536), (5000, 32768), (10000, 32768), (20000, 16384), (50000, 8192),
            (100000, 4096), (150000, 2048), (200000, 512)]


def test_uneven_batch_at_stated_sizes_against_the_oracle():
    """FP32, one persistent launch with the 50k- to 200k-op programs as
    satellite kernels (8 warps per group), every program at its stated
    instance count.  Sampled
    instances (64 per program plus the last, ragged, one) against the FP64
    oracle under the FP32 rule max(2e-4 s_k, 2 B32_k,i, 4 S_k): B32 is the
    first-order rounding bound, S_k the largest deviation of 8 Monte Carlo
    arithmetic runs at FP32 sizes on output row k.  Past ~20k ops most outputs
    keep no correct float digit (S_k reaches s_k), so only S_k can bound their error;
    the fraction of outputs within the plain 2e-4 s_k is recorded and must
    fall with depth as the oracle says it does."""
    irs = [programs.random_program(n, seed=100 + j).to_bytes() for j, (n, _) in enumerate(C5_SIZES)]
    b = Batch(irs, [N for _, N in C5_SIZES], dtype="f32", ways=8)
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
