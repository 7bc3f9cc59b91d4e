"""torch.autograd wrappers: y = D H_m x with its adjoint as the backward pass.

H_m is orthogonal (eq. (1)), so the gradient of a loss L(y) with respect to x is
H_m^T D dL/dy, computed by chw_adjoint (the reversed cascade, see chw.h) with D applied
to the incoming gradient before the transform.
"""

import torch

from . import chw_adjoint, chw_forward, chw_plan


class CHWFunction(torch.autograd.Function):
    """y = D H_m x for a (batch, 2^m) fp32 CUDA tensor; D is an int8 +-1 vector or None."""

    @staticmethod
    def forward(ctx, x, plan, diag):
        x = x.contiguous()
        y = torch.empty_like(x)
        chw_forward(plan, x, y, diag=diag)
        ctx.plan = plan
        ctx.diag = diag
        return y

    @staticmethod
    def backward(ctx, g):
        g = g.contiguous()
        gx = torch.empty_like(g)
        chw_adjoint(ctx.plan, g, gx, diag=ctx.diag)
        return gx, None, None


class DHLayer(torch.nn.Module):
    """The fixed layer y = D H_m x (D a +-1 diagonal), one plan per batch size."""

    def __init__(self, m, diag, norm="end"):
        super().__init__()
        self.m = int(m)
        self.norm = norm
        self.register_buffer("diag", diag.to(torch.int8).contiguous())
        self._plans = {}

    def plan_for(self, batch):
        p = self._plans.get(batch)
        if p is None:
            p = chw_plan(self.m, batch, "f32", self.norm)
            self._plans[batch] = p
        return p

    def forward(self, x):
        if x.dim() != 2 or x.shape[1] != (1 << self.m):
            raise ValueError(f"expected (batch, 2^{self.m}) input")
        return CHWFunction.apply(x, self.plan_for(x.shape[0]), self.diag)
