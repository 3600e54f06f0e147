"""Iterative inverse of the 3D DRT of planes (Section 5.2), float64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): only ``tests/``, the
smoke check and the benchmark's CPU legs may use this module.

Section 5.2 inverts the planes transform the way Press did in 2D: the adjoint
(backprojection, eq.(invmap3Dsummation)) followed by the high-pass filter h is
an approximate inverse, used for iterative improvement of a solution of
A f = R, and a multigrid scheme with the prolongation P (image domain) and the
restriction S (transform domain, each dodecant) makes it fast.  The paper
prints h, P and S and otherwise defers to Press; the steps below are this
oracle's reading of that scheme, in the paper's order:

* approximate inverse at size N:  B_N r = c_N * h (*) A_N^T r, with h applied
  with mirrored borders (a voxel outside the cube takes the value of the
  nearest voxel inside), and c_N = factor / lambda_N, lambda_N the spectral
  radius of h (*) A_N^T A_N (estimated by power iteration);
* one multigrid sweep M_N(r): restrict r down to N = 1 (r_{N/2} = S r_N);
  at N = 1 solve exactly (the one voxel's twelve dodecant values, averaged);
  then for N' = 2, 4, ..., N: x = P x_{N'/2} followed by ``smooth`` steps
  x <- x + B_{N'} (r_{N'} - A_{N'} x);
* outer iteration (iterative improvement): f_0 = 0,
  f_{k+1} = f_k + M_N(R - A_N f_k).

The transform R is the twelve dodecants of Algorithm 2 (order k = 0..11,
storage index d in [0, 3N)).  The oracle's convergence claims are pinned by
its own tests; the paper's "N = 64, ten iterations almost exact" is not
reproduced here (parity of the rate with the paper is unpinned).
"""
from __future__ import annotations

import numpy as np

from . import planes_adjoint, planes_forward

# The high-pass filter h of Section 5.2: slices h(0,:,:) = h(2,:,:) and
# h(1,:,:), as printed.
_H_OUTER = np.array([[-1 / 64, -1 / 32, -1 / 64],
                     [-1 / 32, -1 / 16, -1 / 32],
                     [-1 / 64, -1 / 32, -1 / 64]])
_H_CENTRE = np.array([[-1 / 32, -1 / 16, -1 / 32],
                      [-1 / 16, 7 / 8, -1 / 16],
                      [-1 / 32, -1 / 16, -1 / 32]])
H = np.stack([_H_OUTER, _H_CENTRE, _H_OUTER])

DODECANTS = range(12)


def A(f: np.ndarray) -> np.ndarray:
    """All twelve dodecants of the planes transform, float64 (12, N, N, 3N)."""
    return planes_forward(np.asarray(f, dtype=np.float64), DODECANTS)


def AT(R: np.ndarray) -> np.ndarray:
    """Backprojection summed over the twelve dodecants, float64 (N, N, N)."""
    return planes_adjoint(np.asarray(R, dtype=np.float64), DODECANTS)


def hfilter(x: np.ndarray) -> np.ndarray:
    """h (*) x with mirrored borders: 27 shifted copies, weights H."""
    N = x.shape[0]
    p = np.pad(np.asarray(x, dtype=np.float64), 1, mode="edge")
    out = np.zeros((N, N, N), dtype=np.float64)
    for a in range(3):
        for b in range(3):
            for c in range(3):
                out += H[a, b, c] * p[a:a + N, b:b + N, c:c + N]
    return out


def prolong(g: np.ndarray) -> np.ndarray:
    """P: voxel (i, j, k) of the N-cube takes voxel (i//2, j//2, k//2) of the
    N/2-cube."""
    return g.repeat(2, axis=0).repeat(2, axis=1).repeat(2, axis=2)


def restrict(R: np.ndarray) -> np.ndarray:
    """S, per dodecant: R'(s1, s2, d) = (R(2s1, 2s2, 2d) + R(2s1, 2s2, 2d+1)) / 8,
    d in [0, 3N/2)."""
    return (R[:, 0::2, 0::2, 0::2] + R[:, 0::2, 0::2, 1::2]) / 8.0


def coarsest(R1: np.ndarray) -> np.ndarray:
    """Exact least-squares solve at N = 1: the lone voxel sits at d = 2 of each
    dodecant's column; average the twelve values."""
    return np.full((1, 1, 1), R1[:, 0, 0, 2].mean())


def spectral_radius(N: int, start: np.ndarray, iterations: int = 30) -> float:
    """Power iteration on h (*) A^T A at size N from ``start``: the norm ratio
    ||y|| / ||x|| of the last step."""
    x = np.asarray(start, dtype=np.float64).reshape(N, N, N)
    x = x / np.linalg.norm(x)
    lam = 0.0
    for _ in range(iterations):
        y = hfilter(AT(A(x)))
        lam = float(np.linalg.norm(y))
        x = y / lam
    return lam


def step_sizes(N: int, starts: dict, iterations: int = 30, factor: float = 1.5) -> dict:
    """c_{N'} = factor / lambda_{N'} for N' = 2, 4, ..., N (``starts[N']`` is
    the power iteration's start vector at that size)."""
    out = {}
    L = 2
    while L <= N:
        out[L] = factor / spectral_radius(L, starts[L], iterations)
        L *= 2
    return out


def multigrid(r: np.ndarray, steps: dict, smooth: int = 2) -> np.ndarray:
    """One sweep M_N(r) of the reading above."""
    levels = [np.asarray(r, dtype=np.float64)]
    while levels[-1].shape[1] > 1:
        levels.append(restrict(levels[-1]))
    x = coarsest(levels[-1])
    for rl in reversed(levels[:-1]):
        L = rl.shape[1]
        x = prolong(x)
        for _ in range(smooth):
            x = x + steps[L] * hfilter(AT(rl - A(x)))
    return x


def press_inverse(R: np.ndarray, iterations: int, steps: dict, smooth: int = 2, history: bool = False):
    """f_{k+1} = f_k + M_N(R - A f_k) from f_0 = 0, ``iterations`` times.
    With ``history`` the list of all iterates f_1 .. f_K is returned."""
    R = np.asarray(R, dtype=np.float64)
    N = R.shape[1]
    f = np.zeros((N, N, N))
    hist = []
    for k in range(iterations):
        r = R if k == 0 else R - A(f)
        f = f + multigrid(r, steps, smooth)
        hist.append(f.copy())
    return hist if history else f


def nrmsd(x: np.ndarray, f: np.ndarray) -> float:
    """Normalised root-mean-square deviation (range-normalised), the error
    measure of the paper's inversion figures."""
    rng = float(f.max() - f.min())
    return float(np.sqrt(np.mean((np.asarray(x) - f) ** 2)) / (rng if rng else 1.0))
