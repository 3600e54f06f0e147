"""Least-squares fit of volumes to target planes transforms by gradient descent.

The planes transform A (all 12 dodecants) is linear; its gradient is the
hand-written adjoint (backprojection of Section 5.1) through
``PlanesTransform``.  ``fit`` minimises 0.5 * ||A x - b||^2 from x = 0 with
the fixed step 1 / L, L = sigma_max(A)^2 estimated by power iteration on
A^T A (the step that makes plain gradient descent monotone on this convex
quadratic).
"""
from __future__ import annotations

import torch

from . import ALL, planes, planes_adjoint, planes_forward


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
        r = planes(xr, dodecants) - b
        loss = 0.5 * (r.double() ** 2).sum()
        loss.backward()
        losses.append(float(loss.detach()))
        x = (xr - xr.grad / L).detach()
    return x, losses
