"""Multi-rank data parallelism on CPU ranks (gloo, world size 2): sharded
evaluation equals unsharded evaluation, and the shared-gain gradient summed
over ranks equals the single-process sum.  The per-rank work is done by the
oracle, so this runs without a GPU."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2408_09662_gb300.shard import instance_range


def test_instance_ranges_partition_the_batch():
    for N in (0, 1, 7, 65536, 65537):
        for world in (1, 2, 3, 8):
            got = [instance_range(N, r, world) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == N
            assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
            sizes = [b - a for a, b in got]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    from oracle import Oracle
    from paper_2408_09662_gb300 import inputs, programs
    from paper_2408_09662_gb300.shard import allreduce_shared_grad, instance_range
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # sharded evaluation of the random program
        ir = programs.random_program(1500, seed=5).to_bytes()
        N = 1001
        x = inputs.normal(64, N, seed=1)
        a, b = instance_range(N, rank, world)
        y = torch.tensor(Oracle(ir).eval(x[:, a:b]))
        parts = [None] * world
        dist.all_gather_object(parts, (a, b, y.numpy()))
        # shared gain gradient: per-rank in-shard sum, then all-reduce
        step = programs.srb_step().to_bytes()
        M = 257
        rng = np.random.default_rng(3)
        K = rng.normal(0, 0.1, 144)
        X = np.vstack([np.tile(K[:, None], (1, M)), rng.uniform(-0.1, 0.1, (12, M)), np.zeros((1, M))])
        ybar = rng.standard_normal((13, M))
        c, d = instance_range(M, rank, world)
        xb = Oracle(step).adjoint(X[:, c:d], ybar[:, c:d])
        g = torch.tensor(xb[:144].sum(axis=1))
        allreduce_shared_grad(g)
        if rank == 0:
            out.put((parts, g.numpy()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_match_single_process():
    from oracle import Oracle
    from paper_2408_09662_gb300 import inputs, programs
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    parts, g = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ir = programs.random_program(1500, seed=5).to_bytes()
    x = inputs.normal(64, 1001, seed=1)
    full = Oracle(ir).eval(x)
    for a, b, y in parts:
        np.testing.assert_array_equal(y, full[:, a:b])
    assert sum(b - a for a, b, _ in parts) == 1001
    rng = np.random.default_rng(3)
    K = rng.normal(0, 0.1, 144)
    X = np.vstack([np.tile(K[:, None], (1, 257)), rng.uniform(-0.1, 0.1, (12, 257)), np.zeros((1, 257))])
    ybar = rng.standard_normal((13, 257))
    ref = Oracle(programs.srb_step().to_bytes()).adjoint(X, ybar)[:144].sum(axis=1)
    np.testing.assert_allclose(g, ref, rtol=1e-12, atol=1e-12)


def _rollout_worker(rank, world, port, out):
    """Each rank rolls out its own instances through the rollout's autograd
    function with a CPU step program (the oracle stands in for the library's
    kernels); the shared gain's gradient must come back summed over ranks."""
    import torch
    import torch.distributed as dist

    from oracle import Oracle
    from paper_2408_09662_gb300 import programs
    from paper_2408_09662_gb300.rollout import StepProgram, rollout
    from paper_2408_09662_gb300.shard import instance_range

    class OracleStep(StepProgram):
        def __init__(self):
            self.orc = Oracle(programs.srb_step().to_bytes())
            self.P, self.n = 144, 12

        @property
        def dtype(self):
            return torch.float64

        def step(self, src, dst):
            dst[self.P:] = torch.from_numpy(self.orc.eval(src.numpy()))

        def adjoint_step(self, state, src_bar, dst_bar, shared_bar):
            xb = self.orc.adjoint(state.numpy(), src_bar[self.P:].numpy())
            dst_bar[self.P:] = torch.from_numpy(xb[self.P:])
            shared_bar[:self.P] += torch.from_numpy(xb[:self.P].sum(axis=1))

        def loss_sum(self, buf, out=None):
            return buf[self.P + self.n].sum()

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(7)
        N = 37
        x0 = rng.uniform(-0.1, 0.1, (12, N))
        K = rng.normal(0.0, 0.1, 144)
        a, b = instance_range(N, rank, world)
        xt = torch.tensor(x0[:, a:b], requires_grad=True)
        kt = torch.tensor(K, requires_grad=True)
        L, _ = rollout(OracleStep(), xt, kt, 6, checkpoint_every=4)
        L.backward()
        out.put((rank, a, b, float(L), xt.grad.numpy(), kt.grad.numpy()))
    finally:
        dist.destroy_process_group()


def test_rollout_gradient_of_the_shared_gain_is_summed_over_ranks():
    from oracle import Oracle
    from paper_2408_09662_gb300 import programs
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rollout_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # single process, whole batch: the oracle's forward steps and reverse sweeps
    rng = np.random.default_rng(7)
    N = 37
    x0 = rng.uniform(-0.1, 0.1, (12, N))
    K = rng.normal(0.0, 0.1, 144)
    orc = Oracle(programs.srb_step().to_bytes())
    X = np.vstack([np.tile(K[:, None], (1, N)), x0, np.zeros((1, N))])
    states = []
    for _ in range(6):
        states.append(X.copy())
        X[144:] = orc.eval(X)
    ybar = np.zeros((13, N))
    ybar[12] = 1.0
    gK = np.zeros(144)
    for S in reversed(states):
        xb = orc.adjoint(S, ybar)
        gK += xb[:144].sum(axis=1)
        ybar = xb[144:]
    for rank, a, b, L, gx, gk in res:
        np.testing.assert_allclose(gk, gK, rtol=1e-12, atol=1e-14)      # summed over both ranks
        np.testing.assert_allclose(gx, ybar[:12, a:b], rtol=1e-12, atol=1e-14)
        assert abs(L - X[156, a:b].sum()) <= 1e-12 * abs(L)
