"""Differentiable compressed encoding operator and unrolled CG.

`Ec` wraps gpjc_apply_E as a torch.autograd.Function whose backward is the
hand-written adjoint kernel gpjc_apply_EH (and `EcH` the reverse).  With
PyTorch's convention for complex tensors (the gradient of a real loss is
dL/dRe + i dL/dIm), the vector-Jacobian product of the linear map
y = E_c x is E_c^H applied to the incoming gradient.

`unrolled_cg` runs K iterations of CG on E_c^H E_c x = E_c^H S' (Sec. 3.4,
Eq. 16) as differentiable torch code around those two functions, with each
iteration under activation checkpointing so that memory stays at one
iteration's state while the backward pass recomputes the forward one
iteration at a time.  The operator applications run in the library's
kernels; the few scalar and vector updates of CG are plain torch ops here
because they must carry gradients.
"""
from __future__ import annotations

from typing import Optional

import torch
from torch.utils.checkpoint import checkpoint

from .gpjc import Operator


class Ec(torch.autograd.Function):
    """y = E_c x; backward: grad_x = E_c^H grad_y."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, op: Operator) -> torch.Tensor:
        ctx.op = op
        return op.E(x.contiguous())

    @staticmethod
    def backward(ctx, gy: torch.Tensor):
        return ctx.op.EH(gy.contiguous()), None


class EcH(torch.autograd.Function):
    """x = E_c^H y; backward: grad_y = E_c grad_x."""

    @staticmethod
    def forward(ctx, y: torch.Tensor, op: Operator) -> torch.Tensor:
        ctx.op = op
        return op.EH(y.contiguous())

    @staticmethod
    def backward(ctx, gx: torch.Tensor):
        return ctx.op.E(gx.contiguous()), None


def _dot(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """Re <a, b> accumulated in double precision."""
    return torch.sum(a.real.double() * b.real.double() + a.imag.double() * b.imag.double())


def _cg_step(op: Operator, x, r, p, rr):
    q = Ec.apply(p, op)
    Ap = EcH.apply(q, op)
    qq = _dot(q, q)
    alpha = torch.where(rr > 0, rr / qq, torch.zeros_like(rr)).to(torch.float32)
    x = x + alpha * p
    r = r - alpha * Ap
    rr_new = _dot(r, r)
    beta = torch.where(rr > 0, rr_new / rr, torch.zeros_like(rr)).to(torch.float32)
    p = r + beta * p
    return x, r, p, rr_new


def unrolled_cg(op: Operator, Sc: torch.Tensor, iters: int, x0: Optional[torch.Tensor] = None,
                use_checkpoint: bool = True) -> torch.Tensor:
    """K CG iterations (alpha = ||r||^2 / ||E_c p||^2, beta = ||r_new||^2 / ||r||^2),
    differentiable with respect to Sc (and x0)."""
    b = EcH.apply(Sc, op)
    if x0 is None:
        x = torch.zeros_like(b)
        r = b
    else:
        x = x0
        r = b - EcH.apply(Ec.apply(x0, op), op)
    p = r
    rr = _dot(r, r)
    for _ in range(iters):
        if use_checkpoint:
            x, r, p, rr = checkpoint(_cg_step, op, x, r, p, rr, use_reentrant=False)
        else:
            x, r, p, rr = _cg_step(op, x, r, p, rr)
    return x
