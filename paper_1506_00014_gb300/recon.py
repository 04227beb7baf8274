"""Iterative reconstructions on top of R and R# (Section 8 of the paper): everything stays on
the GPU between the initial upload and the final result.

least_squares: gradient descent on ||R f - g||^2 with the gradient 2 c_R R#(R f - g) (the
    autograd.RadonFunction backward).  The step is 1 / L, with L estimated by power iteration on
    the normal operator c_R R# R.  Optionally one iteration is captured in a CUDA graph and
    replayed.
em: f <- f * R#(g / R f) / R# chi_C (Section 8), chi_C the indicator of the lines that meet the
    unit disc (bins with |s| < 1).
"""

from __future__ import annotations

import torch

from . import binding
from .autograd import adjoint_scales


def _fwd(plan, f, out):
    binding.radon_forward(plan, f, out)
    return out


def _bp(plan, g, out):
    binding.radon_backproject(plan, g, out)
    return out


def normal_operator_norm(plan: binding.RadonPlan, iters: int = 20, seed: int = 0) -> float:
    """Largest eigenvalue of c_R R# R by power iteration (R# R is close to self-adjoint)."""
    c_r, _ = adjoint_scales(plan)
    gen = torch.Generator(device="cuda").manual_seed(seed)
    x = torch.randn(plan.image_shape, device="cuda", generator=gen)
    s = torch.empty(plan.sino_shape, device="cuda")
    y = torch.empty(plan.image_shape, device="cuda")
    lam = 0.0
    for _ in range(iters):
        x = x / x.norm()
        _bp(plan, _fwd(plan, x, s), y)
        y.mul_(c_r)
        lam = float(torch.dot(x.flatten(), y.flatten()))
        x = y.clone()
    return lam


class LeastSquares:
    """Gradient descent x <- x - step * 2 c_R R#(R x - g), optionally replayed from a CUDA graph."""

    def __init__(self, plan: binding.RadonPlan, g: torch.Tensor, step: float | None = None, f0=None,
                 use_graph: bool = False):
        self.plan = plan
        self.g = g.contiguous()
        self.c_r, _ = adjoint_scales(plan)
        if step is None:
            step = 1.0 / (2.0 * normal_operator_norm(plan))
        self.step = float(step)
        self.f = torch.zeros(plan.image_shape, device="cuda") if f0 is None else f0.clone().contiguous()
        self.r = torch.empty(plan.sino_shape, device="cuda")
        self.grad = torch.empty(plan.image_shape, device="cuda")
        self.graph = None
        if use_graph:
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                for _ in range(2):  # warm up outside the capture
                    self._iterate(dry=True)
            torch.cuda.current_stream().wait_stream(side)
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph):
                self._iterate()

    def _iterate(self, dry: bool = False):
        _fwd(self.plan, self.f, self.r)
        self.r.sub_(self.g)
        _bp(self.plan, self.r, self.grad)
        if not dry:
            self.f.add_(self.grad, alpha=-2.0 * self.c_r * self.step)

    def run(self, steps: int):
        for _ in range(steps):
            if self.graph is not None:
                self.graph.replay()
            else:
                self._iterate()
        return self.f

    def loss(self) -> float:
        _fwd(self.plan, self.f, self.r)
        return float(((self.r - self.g) ** 2).sum())


def em(plan: binding.RadonPlan, g: torch.Tensor, iters: int, f0=None, eps: float = 1e-12) -> torch.Tensor:
    """Expectation-maximisation for non-negative f and data g >= 0 (Section 8)."""
    info = plan.info
    nd = info["n_det"]
    k = torch.arange(nd, device="cuda")
    live = (2 * (2 * k - nd) ** 2 < nd * nd).to(torch.float32)
    chi = live.expand(info["n_angles"], nd).contiguous()
    norm = torch.empty(plan.image_shape, device="cuda")
    _bp(plan, chi, norm)
    disc = norm > eps
    f = torch.where(disc, torch.ones(plan.image_shape, device="cuda"), torch.zeros(plan.image_shape, device="cuda")) \
        if f0 is None else f0.clone().contiguous()
    r = torch.empty(plan.sino_shape, device="cuda")
    back = torch.empty(plan.image_shape, device="cuda")
    for _ in range(iters):
        _fwd(plan, f, r)
        ratio = torch.where(r > eps, g / r.clamp_min(eps), torch.zeros_like(r)) * chi
        _bp(plan, ratio.contiguous(), back)
        f = torch.where(disc, f * back / norm.clamp_min(eps), torch.zeros_like(f))
    return f


class BatchedLeastSquares:
    """Gradient descent for B slices of one plan at once, through autograd: the loss
    sum_b ||R f_b - g_b||^2 is differentiated by RadonFunction, whose backward is the scaled R#
    (batched C ABI calls in chunks of the plan's reserved capacity), then f <- f - step * grad.
    With use_graph, one whole iteration (forward, backward, update) is captured in a CUDA graph
    and replayed; reserve the plan's batch capacity before constructing it."""

    def __init__(self, plan: binding.RadonPlan, g: torch.Tensor, step: float, f0=None, use_graph: bool = False):
        from .autograd import radon

        self._radon = radon
        self.plan = plan
        self.g = g.contiguous()
        self.step = float(step)
        shape = (g.shape[0],) + plan.image_shape
        self.f = (torch.zeros(shape, device="cuda") if f0 is None else f0.clone().contiguous()).requires_grad_(True)
        self.graph = None
        if use_graph:
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                f_save = self.f.detach().clone()
                for _ in range(2):  # warm up outside the capture (autograd and allocator state)
                    self._iterate()
                with torch.no_grad():
                    self.f.copy_(f_save)
            torch.cuda.current_stream().wait_stream(side)
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph):
                self._iterate()

    def _iterate(self):
        self.f.grad = None
        loss = ((self._radon(self.f, self.plan) - self.g) ** 2).sum()
        loss.backward()
        with torch.no_grad():
            self.f.sub_(self.f.grad, alpha=self.step)

    def run(self, steps: int):
        for _ in range(steps):
            if self.graph is not None:
                self.graph.replay()
            else:
                self._iterate()
        return self.f.detach()

    def losses(self) -> torch.Tensor:
        """Per-slice ||R f_b - g_b||^2."""
        with torch.no_grad():
            r = self._radon(self.f.detach(), self.plan) - self.g
            return (r * r).sum(dim=(1, 2))


def em_batched(plan: binding.RadonPlan, g: torch.Tensor, iters: int, eps: float = 1e-12) -> torch.Tensor:
    """em() for a stack of slices g [B, n_angles, n_det] (a volume): every R and R# goes through
    the batched C ABI in chunks of the plan's reserved capacity, and everything stays on the GPU
    between the upload of g and the returned stack f [B, N, N]."""
    info = plan.info
    nd, na = info["n_det"], info["n_angles"]
    B = g.shape[0]
    cap = max(1, getattr(plan, "max_batch", 1))
    k = torch.arange(nd, device="cuda")
    chi = (2 * (2 * k - nd) ** 2 < nd * nd).to(torch.float32).expand(na, nd).contiguous()
    norm = torch.empty(plan.image_shape, device="cuda")
    _bp(plan, chi, norm)
    disc = norm > eps
    f = torch.where(disc, 1.0, 0.0).to(torch.float32).expand(B, *plan.image_shape).contiguous()
    r = torch.empty((B,) + plan.sino_shape, device="cuda")
    back = torch.empty_like(f)
    g = g.contiguous()
    for _ in range(iters):
        for b0 in range(0, B, cap):
            b1 = min(B, b0 + cap)
            binding.radon_forward_batch(plan, f[b0:b1], r[b0:b1])
        ratio = torch.where(r > eps, g / r.clamp_min(eps), torch.zeros_like(r)) * chi
        for b0 in range(0, B, cap):
            b1 = min(B, b0 + cap)
            binding.radon_backproject_batch(plan, ratio[b0:b1].contiguous(), back[b0:b1])
        f = torch.where(disc, f * back / norm.clamp_min(eps), torch.zeros_like(f))
    return f
