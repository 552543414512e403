"""Differentiable batched rollouts of a one-step program (torch.autograd).

A step program maps [P (broadcast parameters), x (state), L (running loss)]
to [x+, L+] with its outputs lined up with input rows P..P+n+1, so a rollout
ping-pongs two [P + n + 1, N] buffers with no copies: step t reads buffer
t % 2 and writes the state rows of the other.

Backward pass (reverse mode through the library's adjoint kernels): states are
kept every ``checkpoint_every`` steps; each segment is recomputed forward from
its checkpoint, then the adjoint kernel runs once per step in reverse.  The
parameter gradient is reduced over instances by the adjoint (per-instance
terms in the workspace, summed in a fixed order) and accumulated over
steps in place, so it has the same bits on every run.
"""
from __future__ import annotations

import torch

from .api import Function


class StepProgram:
    def __init__(self, fn: Function, n_param: int, n_state: int):
        if fn.nnz_in != n_param + n_state + 1 or fn.nnz_out != n_state + 1:
            raise ValueError("step program must map [P, x, L] -> [x+, L+]")
        self.fn, self.P, self.n = fn, n_param, n_state

    def buffers(self, K: torch.Tensor, N: int, count: int):
        rows = self.P + self.n + 1
        b = torch.zeros((count, rows, N), dtype=self.fn.torch_dtype, device=K.device)
        b[:, :self.P, 0] = K.reshape(1, self.P)
        return b

    def step(self, src: torch.Tensor, dst: torch.Tensor):
        self.fn(src, out=dst[self.P:])


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
        return final[P + n].sum(), final[P:P + n].clone()

    @staticmethod
    def backward(ctx, gL, gx):
        prog, steps, ce = ctx.prog, ctx.steps, ctx.ce
        (K,) = ctx.saved_tensors
        P, n = prog.P, prog.n
        N = next(iter(ctx.ckpts.values())).shape[1]
        bar = prog.buffers(torch.zeros_like(K), N, 2)        # ping-pong adjoint buffers
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
                src, dst = bar[(t + 1) % 2], bar[t % 2]
                prog.fn.adjoint(states[j], src[P:], out=dst, reduce_broadcast=True,
                                accumulate_broadcast=True)
        xbar = bar[0, P:P + n].clone()
        Kbar = (bar[0, :P, 0] + bar[1, :P, 0]).reshape(K.shape)
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
    constructor runs one eager pass first)."""

    def __init__(self, prog: StepProgram, N: int, steps: int, checkpoint_every: int = 10,
                 device="cuda"):
        self.prog, self.steps, self.ce = prog, steps, checkpoint_every
        dt = prog.fn.torch_dtype
        P, n = prog.P, prog.n
        self.x0 = torch.zeros((n, N), dtype=dt, device=device)
        self.K = torch.zeros(P, dtype=dt, device=device)
        self.gL = torch.ones((), dtype=dt, device=device)
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
        self.L = final[P + n].sum()
        self.xT = final[P:P + n]

    def _backward(self):
        prog, P, n, steps, ce = self.prog, self.prog.P, self.prog.n, self.steps, self.ce
        N = self.x0.shape[1]
        bar = prog.buffers(torch.zeros_like(self.K), N, 2)
        bar[steps % 2, P + n] = self.gL
        states = prog.buffers(self.K, N, ce)
        for start in sorted(self.ckpt, reverse=True):
            seg = min(ce, steps - start)
            states[0, P:P + n] = self.ckpt[start]
            for j in range(seg - 1):
                prog.step(states[j], states[j + 1])
            for j in reversed(range(seg)):
                t = start + j
                prog.fn.adjoint(states[j], bar[(t + 1) % 2][P:], out=bar[t % 2],
                                reduce_broadcast=True, accumulate_broadcast=True)
        self.gx = bar[0, P:P + n]
        self.gK = bar[0, :P, 0] + bar[1, :P, 0]

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
