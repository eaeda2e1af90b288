"""torch.autograd binding of the forward operator: data = H p0, and its backward H^T.

H is linear in p0 (Sec. III), so the vector-Jacobian product of ``PATFunction`` is exactly the
adjoint solve pat_adjoint applied to the incoming gradient, with no stored forward fields.  The
batched form applies one plan per instance (instances may have different grids).

``PATMediumFunction`` makes the medium differentiable as well: data = H(c0^2, rho0) p0, whose
vector-Jacobian product with respect to (p0, c0^2, rho0) is one checkpointed reverse sweep
(pat_gradient_medium: forward states every K time levels, each segment recomputed once), for the
joint reconstruction of the medium that Sec. VII motivates.
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np
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


class PATMediumFunction(torch.autograd.Function):
    """data[Nt][Ns] = H(c0^2, rho0) p0 on the plan ``op`` built for this c0^2 and rho0 (the medium
    tensors name the plan's medium for autograd; they are not read).  Backward: the products with
    grad_data of the derivatives with respect to p0 (H^T grad_data), c0^2 (readings M1-M3: alpha0,
    y, rho0 and the plan's reference speed, dt, kappa and PML held fixed) and rho0 (readings D1-D3),
    from one sweep that stores forward checkpoints every K time levels; only the requested ones
    are formed, and without a medium gradient it is the plain adjoint solve."""

    @staticmethod
    def forward(ctx, p0: torch.Tensor, c2: torch.Tensor, rho0: torch.Tensor, op: PATOperator, K: int):
        ctx.op, ctx.K = op, int(K)
        ctx.save_for_backward(p0)
        return op.forward(p0.contiguous())

    @staticmethod
    def backward(ctx, grad_data: torch.Tensor):
        (p0,) = ctx.saved_tensors
        need = ctx.needs_input_grad[:3]
        want = tuple(k for k, n in zip(("p0", "c2", "rho"), need) if n)
        if not want:
            return None, None, None, None, None
        g = grad_data.contiguous()
        if want == ("p0",):
            return ctx.op.adjoint(g), None, None, None, None
        gr, gc, gp = ctx.op.gradient_medium(p0.contiguous(), g, ctx.K, want=want)
        return gp, gc, gr, None, None


def checkpoint_bytes(op: PATOperator, K: int, c2: bool = True, rho: bool = True) -> int:
    """Device memory the checkpointed sweep allocates for one call (pat_gradient_medium with interval
    K): the ceil((Nt - 1) / K) checkpoints of (u_xi, rho_xi, spectrum of p), K fields q^n for the
    c0^2 gradient, K + 1 steps of (D+ p, D- u) and d accumulators for the rho0 gradient, and a copy
    of the forward state."""
    d = len(op.shape)
    w = 4 if op.dtype == torch.float32 else 8
    N = op.N
    nh = int(np.prod(op.shape[:-1])) * ((op.shape[-1] // 2 + 1 + 7) // 8 * 8)
    nseg = (op.Nt - 2) // K + 1 if op.Nt > 1 else 0
    b = max(nseg, 1) * (2 * d * N + 2 * nh) * w            # checkpoints
    b += (2 * d + (1 if op.lossy else 0) + 1) * N * w + max(d, 2) * nh * 2 * w   # forward state, p0 copy
    if c2:
        b += (1 + max(1, min(K, op.Nt))) * N * w
    if rho:
        b += (1 + d + (min(K, max(op.Nt - 1, 1)) + 1) * 2 * d) * N * w
    return int(b)


def pat_apply_medium(op: PATOperator, p0: torch.Tensor, c2: torch.Tensor, rho0: torch.Tensor,
                     checkpoint_every: int = 50) -> torch.Tensor:
    """Differentiable H(c0^2, rho0) p0 (gradients in p0, c0^2 and rho0)."""
    return PATMediumFunction.apply(p0, c2, rho0, op, checkpoint_every)


def pat_apply(op: PATOperator, p0: torch.Tensor) -> torch.Tensor:
    """Differentiable H p0."""
    return PATFunction.apply(p0, op)


def pat_apply_batch(ops: Sequence[PATOperator], p0s: Sequence[torch.Tensor], batch: Optional[PATBatch] = None):
    """Differentiable [H_i p0_i] for a batch of instances (one launch per direction when ``batch``
    is given)."""
    return PATBatchFunction.apply(*p0s, list(ops), batch)
