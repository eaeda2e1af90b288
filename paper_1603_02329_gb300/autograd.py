"""torch.autograd binding of the forward operator: data = H p0, and its backward H^T.

H is linear in p0 (Sec. III), so the vector-Jacobian product of ``PATFunction`` is exactly the
adjoint solve pat_adjoint applied to the incoming gradient, with no stored forward fields.  The
batched form applies one plan per instance (instances may have different grids).
"""
from __future__ import annotations

from typing import Optional, Sequence

import torch

from .api import PATBatch, PATOperator


class PATFunction(torch.autograd.Function):
    """data[Nt][Ns] = H p0 with grad_p0 = H^T grad_data (pat_forward_plan / pat_adjoint)."""

    @staticmethod
    def forward(ctx, p0: torch.Tensor, op: PATOperator) -> torch.Tensor:
        ctx.op = op
        return op.forward(p0.contiguous())

    @staticmethod
    def backward(ctx, grad_data: torch.Tensor):
        return ctx.op.adjoint(grad_data.contiguous()), None


class PATBatchFunction(torch.autograd.Function):
    """A batch of independent instances: out[i] = H_i p0[i] (one plan per instance); with a
    ``PATBatch`` every direction is one graph launch over all instances."""

    @staticmethod
    def forward(ctx, *args):
        ops, batch = args[-2], args[-1]
        p0s = [p.contiguous() for p in args[:-2]]
        ctx.ops, ctx.batch = ops, batch
        if batch is not None:
            return tuple(batch.forward(p0s))
        return tuple(op.forward(p) for p, op in zip(p0s, ops))

    @staticmethod
    def backward(ctx, *grads):
        grads = [g.contiguous() for g in grads]
        if ctx.batch is not None:
            outs = tuple(ctx.batch.adjoint(grads))
        else:
            outs = tuple(op.adjoint(g) for g, op in zip(grads, ctx.ops))
        return outs + (None, None)


def pat_apply(op: PATOperator, p0: torch.Tensor) -> torch.Tensor:
    """Differentiable H p0."""
    return PATFunction.apply(p0, op)


def pat_apply_batch(ops: Sequence[PATOperator], p0s: Sequence[torch.Tensor], batch: Optional[PATBatch] = None):
    """Differentiable [H_i p0_i] for a batch of instances (one launch per direction when ``batch``
    is given)."""
    return PATBatchFunction.apply(*p0s, list(ops), batch)
