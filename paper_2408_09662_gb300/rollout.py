"""Differentiable batched rollouts of a one-step program (torch.autograd).

A step program maps [P (broadcast parameters), x (state), L (running loss)]
to [x+, L+] with its outputs lined up with input rows P..P+n+1, so a rollout
ping-pongs two [P + n + 1, N] buffers with no copies: step t reads buffer
t % 2 and writes the state rows of the other.

Backward pass (reverse mode through the library's adjoint kernels): states are
kept every ``checkpoint_every`` steps; each segment is recomputed forward from
its checkpoint, then the adjoint kernel runs once per step in reverse.  The
parameter gradient is reduced over instances by the library (per-instance
terms in the workspace, summed in a fixed order) and accumulated over steps
into one vector, and the loss is summed over instances by the library in a
fixed order, so both have the same bits on every run; this module only moves
buffers.  Under torch.distributed with more than one rank, each rank rolls out
its own instances and the parameter gradient is summed over ranks.
"""
from __future__ import annotations

import torch

from .api import Function, sum_instances
from .shard import allreduce_shared_grad


class StepProgram:
    """One step of a rollout: the library calls a rollout makes on a step
    program (forward step, reverse step, loss sum over instances)."""

    def __init__(self, fn: Function, n_param: int, n_state: int):
        if fn.nnz_in != n_param + n_state + 1 or fn.nnz_out != n_state + 1:
            raise ValueError("step program must map [P, x, L] -> [x+, L+]")
        self.fn, self.P, self.n = fn, n_param, n_state

    @property
    def dtype(self):
        return self.fn.torch_dtype

    def buffers(self, K: torch.Tensor, N: int, count: int):
        rows = self.P + self.n + 1
        b = torch.zeros((count, rows, N), dtype=self.dtype, device=K.device)
        b[:, :self.P, 0] = K.reshape(1, self.P)
        return b

    def step(self, src: torch.Tensor, dst: torch.Tensor):
        """dst[x, L] = step(src[P, x, L])."""
        self.fn(src, out=dst[self.P:])

    def adjoint_step(self, state: torch.Tensor, src_bar: torch.Tensor, dst_bar: torch.Tensor,
                     shared_bar: torch.Tensor):
        """dst_bar[x, L] = J^T src_bar[x, L] at `state`; the parameters' adjoint,
        summed over instances, is added to shared_bar[:P]."""
        self.fn.adjoint(state, src_bar[self.P:], out=dst_bar, accumulate_broadcast=True,
                        shared_out=shared_bar)

    def loss_sum(self, buf: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """Sum over instances of the running-loss row of `buf`, a 0-d tensor."""
        row = self.P + self.n
        s = sum_instances(buf[row:row + 1], out=None if out is None else out.reshape(1))
        return s.reshape(()) if out is None else out


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, K, prog: StepProgram, steps: int, checkpoint_every: int):
        N = x0.shape[1]
        P, n = prog.P, prog.n
        buf = prog.buffers(K, N, 2)
        buf[0, P:P + n] = x0
        ckpts = {}
        for t in range(steps):
            if t % checkpoint_every == 0:
                ckpts[t] = buf[t % 2, P:P + n].clone()
            prog.step(buf[t % 2], buf[(t + 1) % 2])
        final = buf[steps % 2]
        ctx.prog, ctx.steps, ctx.ce, ctx.ckpts = prog, steps, checkpoint_every, ckpts
        ctx.save_for_backward(K)
        return prog.loss_sum(final), final[P:P + n].clone()

    @staticmethod
    def backward(ctx, gL, gx):
        prog, steps, ce = ctx.prog, ctx.steps, ctx.ce
        (K,) = ctx.saved_tensors
        P, n = prog.P, prog.n
        N = next(iter(ctx.ckpts.values())).shape[1]
        bar = prog.buffers(torch.zeros_like(K), N, 2)        # ping-pong adjoint buffers
        shared = torch.zeros(P + n + 1, dtype=prog.dtype, device=K.device)
        if gx is not None:
            bar[steps % 2, P:P + n] = gx
        bar[steps % 2, P + n] = gL
        states = prog.buffers(K, N, ce)
        for start in sorted(ctx.ckpts, reverse=True):
            seg = min(ce, steps - start)
            states[0, P:P + n] = ctx.ckpts[start]
            for j in range(seg - 1):
                prog.step(states[j], states[j + 1])
            for j in reversed(range(seg)):
                t = start + j
                prog.adjoint_step(states[j], bar[(t + 1) % 2], bar[t % 2], shared)
        xbar = bar[0, P:P + n].clone()
        Kbar = allreduce_shared_grad(shared[:P].clone()).reshape(K.shape)
        return xbar, Kbar, None, None, None


def rollout(prog: StepProgram, x0: torch.Tensor, K: torch.Tensor, steps: int,
            checkpoint_every: int = 10):
    """(sum over instances of the running loss after `steps` steps, final states).
    Differentiable with respect to x0 [n, N] and the shared parameters K."""
    return _Rollout.apply(x0, K, prog, steps, checkpoint_every)


class GraphRollout:
    """The same rollout and its gradient replayed from two CUDA graphs (one for
    the forward pass, one for the checkpointed reverse pass), so the host issues
    one launch per pass instead of one per step and kernel.  Inputs are copied
    into static buffers; every call returns (L, x_T, dL/dx0, dL/dK) computed on
    the device.  The step program's kernels must already be loaded (the
    constructor runs one eager pass first).  One process only: the gradient is
    not summed over ranks."""

    def __init__(self, prog: StepProgram, N: int, steps: int, checkpoint_every: int = 10,
                 device="cuda"):
        self.prog, self.steps, self.ce = prog, steps, checkpoint_every
        dt = prog.dtype
        P, n = prog.P, prog.n
        self.x0 = torch.zeros((n, N), dtype=dt, device=device)
        self.K = torch.zeros(P, dtype=dt, device=device)
        self.gL = torch.ones((), dtype=dt, device=device)
        self.L = torch.zeros((), dtype=dt, device=device)
        self.shared = torch.zeros(P + n + 1, dtype=dt, device=device)
        self._eager()                                   # loads forward + adjoint kernels
        torch.cuda.synchronize()
        s = torch.cuda.Stream(device)
        s.wait_stream(torch.cuda.current_stream(device))
        with torch.cuda.stream(s):
            self._eager()                               # warm the graph pool
        torch.cuda.current_stream(device).wait_stream(s)
        torch.cuda.synchronize()
        self.g_fwd, self.g_bwd = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.g_fwd):
            self._forward()
        with torch.cuda.graph(self.g_bwd):
            self._backward()

    def _forward(self):
        prog, P, n = self.prog, self.prog.P, self.prog.n
        N = self.x0.shape[1]
        buf = prog.buffers(self.K, N, 2)
        buf[0, P:P + n] = self.x0
        self.ckpt = {}
        for t in range(self.steps):
            if t % self.ce == 0:
                self.ckpt[t] = buf[t % 2, P:P + n].clone()
            prog.step(buf[t % 2], buf[(t + 1) % 2])
        final = buf[self.steps % 2]
        prog.loss_sum(final, out=self.L)
        self.xT = final[P:P + n]

    def _backward(self):
        prog, P, n, steps, ce = self.prog, self.prog.P, self.prog.n, self.steps, self.ce
        N = self.x0.shape[1]
        bar = prog.buffers(torch.zeros_like(self.K), N, 2)
        bar[steps % 2, P + n] = self.gL
        self.shared.zero_()
        states = prog.buffers(self.K, N, ce)
        for start in sorted(self.ckpt, reverse=True):
            seg = min(ce, steps - start)
            states[0, P:P + n] = self.ckpt[start]
            for j in range(seg - 1):
                prog.step(states[j], states[j + 1])
            for j in reversed(range(seg)):
                t = start + j
                prog.adjoint_step(states[j], bar[(t + 1) % 2], bar[t % 2], self.shared)
        self.gx = bar[0, P:P + n]
        self.gK = self.shared[:P]

    def _eager(self):
        self._forward()
        self._backward()

    def forward(self, x0: torch.Tensor, K: torch.Tensor):
        self.x0.copy_(x0)
        self.K.copy_(K.reshape(-1))
        self.g_fwd.replay()
        return self.L, self.xT

    def backward(self):
        """dL/dx0, dL/dK of the last forward()."""
        self.g_bwd.replay()
        return self.gx, self.gK
