"""Least-squares fit of volumes to target planes transforms by gradient descent.

The planes transform A (all 12 dodecants) is linear; its gradient is the
hand-written adjoint (backprojection of Section 5.1).  ``LeastSquaresLoss``
computes the residual A x - b inside the transform's last pass and
backprojects it; ``fit`` minimises 0.5 * ||A x - b||^2 from x = 0 with
the fixed step 1 / L, L = sigma_max(A)^2 estimated by power iteration on
A^T A (the step that makes plain gradient descent monotone on this convex
quadratic).
"""
from __future__ import annotations

import torch

from . import ALL, _mask, get_plan, planes_adjoint, planes_forward, planes_forward_residual_loss


class LeastSquaresLoss(torch.autograd.Function):
    """0.5 ||A x - b||^2 over a batch, with A the planes transform.

    Forward computes the residual r = A x - b in the transform's own store
    (one pass over b, none over A x) and the loss as r is stored (no pass
    over r); backward is the hand-written adjoint (backprojection) of r,
    scaled by the incoming gradient.  r is kept between the two (the one
    tensor of the size of b).
    """

    @staticmethod
    def forward(ctx, x: torch.Tensor, b: torch.Tensor, dodecants: int = ALL):
        if x.dtype != torch.float32 or x.dim() != 4:
            raise TypeError("expected (B, N, N, N) float32 volumes")
        x = x.contiguous()
        B, N = int(x.shape[0]), int(x.shape[1])
        m = _mask(dodecants)
        r = torch.empty_like(b)
        losses = torch.empty((B,), dtype=torch.float64, device=x.device)
        ws = get_plan(N, torch.float32).workspace("planes_residual_loss")
        for i in range(B):
            planes_forward_residual_loss(x[i], b[i], m, out=r[i], loss=losses[i], workspace=ws)
        ctx.save_for_backward(r)
        ctx.mask = m
        return losses.sum()

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        (r,) = ctx.saved_tensors
        B, N = int(r.shape[0]), int(r.shape[2])
        grad = torch.empty((B, N, N, N), dtype=torch.float32, device=r.device)
        ws = get_plan(N, torch.float32).workspace("planes_adjoint")
        for i in range(B):
            planes_adjoint(r[i], ctx.mask, out=grad[i], workspace=ws)
        grad.mul_(g.to(grad.dtype))  # the incoming gradient (1 for loss.backward())
        return grad, None, None


def least_squares_loss(x: torch.Tensor, b: torch.Tensor, dodecants=ALL) -> torch.Tensor:
    """0.5 ||A x - b||^2 (float64 scalar; squares of the float32 residual
    added per lane in float32, then in float64) for (B, N, N, N) float32 x and
    (B, k, N, N, 3N) float32 targets; differentiable in x."""
    return LeastSquaresLoss.apply(x, b, _mask(dodecants))


def operator_norm_sq(N: int, iters: int = 20, seed: int = 0, device=None) -> float:
    """sigma_max(A)^2 by ``iters`` power iterations on A^T A (float32 volumes)."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    v = torch.randn((N, N, N), generator=g, dtype=torch.float32).to(device or "cuda")
    v /= v.norm()
    lam = 0.0
    for _ in range(iters):
        w = planes_adjoint(planes_forward(v, ALL), ALL)
        lam = float(torch.dot(v.flatten().double(), w.flatten().double()))
        v = w / w.norm()
    return lam


def fit(b: torch.Tensor, steps: int = 50, L: float | None = None, dodecants: int = ALL):
    """Gradient descent on 0.5 ||A x - b||^2, batch over the leading dim.

    ``b``: (B, k, N, N, 3N) float32 targets.  Returns (x, losses) with
    losses[t] the loss before step t (float64 host values).
    """
    B, N = int(b.shape[0]), int(b.shape[2])
    if L is None:
        L = operator_norm_sq(N, device=b.device)
    x = torch.zeros((B, N, N, N), dtype=torch.float32, device=b.device)
    losses = []
    for _ in range(steps):
        xr = x.detach().requires_grad_(True)
        loss = least_squares_loss(xr, b, dodecants)
        loss.backward()
        losses.append(float(loss.detach()))
        x = (xr - xr.grad / L).detach()
    return x, losses
