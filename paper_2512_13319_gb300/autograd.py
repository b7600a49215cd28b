"""torch.autograd wrappers of the MAP solve and its hand-written adjoint.

Marshalling only: forward runs map_smoother_update + map_smoother_solve,
backward runs map_smoother_grad (the implicit-function adjoint in the CUDA
library).  Parameters theta = (F, log q, log r) with Q = e^log_q L W L^T and
R = e^log_r R of the model the smoother was created with.
"""
from __future__ import annotations

import torch


def _set_params(smoother, F, log_q, log_r):
    smoother.update(F.detach().to("cpu", torch.float64).numpy(), float(log_q), float(log_r))


class MapSolve(torch.autograd.Function):
    """x* = argmin_x M(x; F, log q, log r) for observations y."""

    @staticmethod
    def forward(ctx, F, log_q, log_r, y, smoother):
        _set_params(smoother, F, log_q, log_r)
        x = smoother.solve(y)
        ctx.smoother = smoother
        ctx.save_for_backward(y, x)
        ctx.dtypes = (F.dtype, log_q.dtype, log_r.dtype)
        return x

    @staticmethod
    def backward(ctx, gx):
        y, x = ctx.saved_tensors
        sm = ctx.smoother
        g = sm.grad(y, x, gx.contiguous().to(x.dtype))
        n = sm.nx
        dF = torch.tensor(g[: n * n].reshape(n, n), dtype=ctx.dtypes[0])
        dq = torch.tensor(g[n * n], dtype=ctx.dtypes[1])
        dr = torch.tensor(g[n * n + 1], dtype=ctx.dtypes[2])
        return dF, dq, dr, None, None


class MapCost(torch.autograd.Function):
    """min_x M(x; F, log q, log r): the MAP cost (Eq. 2, discrete), optionally
    with the Gaussian log-normalisers; gradient by the envelope theorem."""

    @staticmethod
    def forward(ctx, F, log_q, log_r, y, smoother, logdet):
        _set_params(smoother, F, log_q, log_r)
        x, _, cost = smoother.solve(y, cost=True)
        if logdet:
            cost += smoother.log_normaliser()
        ctx.smoother = smoother
        ctx.logdet = logdet
        ctx.save_for_backward(y, x)
        ctx.dtypes = (F.dtype, log_q.dtype, log_r.dtype)
        return torch.tensor(cost, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gc):
        y, x = ctx.saved_tensors
        sm = ctx.smoother
        g = sm.grad(y, x, None, logdet=ctx.logdet) * float(gc)
        n = sm.nx
        dF = torch.tensor(g[: n * n].reshape(n, n), dtype=ctx.dtypes[0])
        dq = torch.tensor(g[n * n], dtype=ctx.dtypes[1])
        dr = torch.tensor(g[n * n + 1], dtype=ctx.dtypes[2])
        return dF, dq, dr, None, None, None


def map_solve(smoother, y, F, log_q, log_r):
    return MapSolve.apply(F, log_q, log_r, y, smoother)


def map_cost(smoother, y, F, log_q, log_r, logdet=False):
    return MapCost.apply(F, log_q, log_r, y, smoother, logdet)
