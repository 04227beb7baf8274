"""torch.autograd wrappers: R with backward R#, and R# with backward R.

With torch's plain sums, <R f, g> = sum_ak (R f)_ak g_ak approximates (1 / (dtheta ds)) times
the continuous inner product, and <f, R# g> = sum_p f_p (R# g)_p approximates (1 / dx^2) times
its continuous counterpart.  So the gradient of sum (R f) * G with respect to f is
(dx^2 / (dtheta ds)) R# G, and that of sum (R# g) * F with respect to g is (dtheta ds / dx^2) R F.
Here dx = 2/N, dtheta = pi/n_angles and ds = 2 sqrt(2)/n_det.

R# is the discretised adjoint of the continuous R (Algorithm 2), not the transpose of the discrete
Algorithm 1. The two agree to about 1e-5 relative on smooth inputs and differ more on rough
ones, and that difference is what a finite-difference check of these gradients measures.

``radon(image, plan, exact=True)`` takes the backward from radon_transpose instead: the exact
transpose of the discrete forward map, so its gradients pass a finite-difference check to FP32
rounding (no scale factor: it is the transpose for torch's plain sums).

R is linear, so nothing is saved for backward.  Inputs of shape [N, N] / [n_angles, n_det] or
batches [B, ...] of them.  A batch runs through the batched C ABI entry points in chunks of the
plan's reserved capacity (radon_plan_reserve_batch; one slice per call when nothing is reserved),
on the current stream.
"""

from __future__ import annotations

import math

import torch

from . import binding


def adjoint_scales(plan: binding.RadonPlan):
    """(c_R, c_B): grad of R is c_R * R#, grad of R# is c_B * R."""
    info = plan.info
    dx2 = (2.0 / info["N"]) ** 2
    dsino = (math.pi / info["n_angles"]) * (2.0 * math.sqrt(2.0) / info["n_det"])
    return dx2 / dsino, dsino / dx2


def _apply(fn, fn_batch, plan, x, out_shape):
    x = x.contiguous()
    if x.dim() == 2:
        out = torch.empty(out_shape, dtype=torch.float32, device=x.device)
        fn(plan, x, out)
        return out
    out = torch.empty((x.shape[0],) + tuple(out_shape), dtype=torch.float32, device=x.device)
    cap = max(1, getattr(plan, "max_batch", 1))
    for b0 in range(0, x.shape[0], cap):
        b1 = min(x.shape[0], b0 + cap)
        if b1 - b0 == 1:
            fn(plan, x[b0], out[b0])
        else:
            fn_batch(plan, x[b0:b1], out[b0:b1])
    return out


class RadonFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, image, plan):
        ctx.plan = plan
        return _apply(binding.radon_forward, binding.radon_forward_batch, plan, image, plan.sino_shape)

    @staticmethod
    def backward(ctx, grad):
        plan = ctx.plan
        c_r, _ = adjoint_scales(plan)
        return _apply(binding.radon_backproject, binding.radon_backproject_batch, plan, grad, plan.image_shape) * c_r, None


class RadonExactFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, image, plan):
        ctx.plan = plan
        return _apply(binding.radon_forward, binding.radon_forward_batch, plan, image, plan.sino_shape)

    @staticmethod
    def backward(ctx, grad):
        plan = ctx.plan
        return _apply(binding.radon_transpose, binding.radon_transpose_batch, plan, grad, plan.image_shape), None


class BackprojectFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sino, plan):
        ctx.plan = plan
        return _apply(binding.radon_backproject, binding.radon_backproject_batch, plan, sino, plan.image_shape)

    @staticmethod
    def backward(ctx, grad):
        plan = ctx.plan
        _, c_b = adjoint_scales(plan)
        return _apply(binding.radon_forward, binding.radon_forward_batch, plan, grad, plan.sino_shape) * c_b, None


def radon(image: torch.Tensor, plan: binding.RadonPlan, exact: bool = False) -> torch.Tensor:
    """R f for [N, N] or [B, N, N] float32 CUDA tensors (differentiable).  The backward is the
    scaled R# (exact=False) or the exact transpose R^T (exact=True)."""
    return (RadonExactFunction if exact else RadonFunction).apply(image, plan)


def backproject(sino: torch.Tensor, plan: binding.RadonPlan) -> torch.Tensor:
    """R# g for [n_angles, n_det] or [B, n_angles, n_det] float32 CUDA tensors (differentiable)."""
    return BackprojectFunction.apply(sino, plan)
