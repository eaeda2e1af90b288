"""torch.autograd binding of the forward operator: data = H p0, and its backward H^T.

H is linear in p0 (Sec. III), so the vector-Jacobian product of ``PATFunction`` is exactly the
adjoint solve pat_adjoint applied to the incoming gradient, with no stored forward fields.  The
batched form applies one plan per instance (instances may have different grids).
"""
from __future__ import annotations

from typing import Sequence

import torch

from .api import PATOperator


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
    """A batch of independent instances: out[i] = H_i p0[i] (one plan per instance)."""

    @staticmethod
    def forward(ctx, *args):
        ops = args[-1]
        p0s = args[:-1]
        ctx.ops = ops
        return tuple(op.forward(p.contiguous()) for p, op in zip(p0s, ops))

    @staticmethod
    def backward(ctx, *grads):
        outs = tuple(op.adjoint(g.contiguous()) for g, op in zip(grads, ctx.ops))
        return outs + (None,)


def pat_apply(op: PATOperator, p0: torch.Tensor) -> torch.Tensor:
    """Differentiable H p0."""
    return PATFunction.apply(p0, op)


def pat_apply_batch(ops: Sequence[PATOperator], p0s: Sequence[torch.Tensor]):
    """Differentiable [H_i p0_i] for a batch of instances."""
    return PATBatchFunction.apply(*p0s, list(ops))
