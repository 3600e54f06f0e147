"""Ray in noise (Section 4.1, the DJT example): a digital line buried in white
noise of larger amplitude still stands out in the John domain; keeping only
the largest coefficients and backprojecting them brings the line back.

The volume, the transform, the thresholding and the backprojection all stay
on the GPU; the line is drawn with eq.(digitalLine) in the sector's frame.
"""
from __future__ import annotations

import torch

from . import lines_adjoint, lines_forward


def _lline(n: int, s: int, u: int) -> int:
    """l^n_s(u) of eq.(digitalLine)."""
    return sum(((u >> (n - 1 - i)) & 1) * (((s >> i) + 1) >> 1) for i in range(n))


def ray_in_noise(N: int = 128, amplitude: int = 16, noise: int = 32, top: int = 16, seed: int = 9,
                 line=(37, 90, 150, 140), sector: int = 0, device="cuda") -> dict:
    """Embed the line (s1, s2, d1, d2) of ``sector`` (driving axis x, no flips
    for sector 0) with value ``amplitude`` into integer noise uniform in
    [-noise, noise], take the DJT of that sector, keep the ``top`` largest
    coefficients and backproject them.

    Returns the volume, the line's voxel mask, the position of the largest
    coefficient, the line's own coefficient, the largest coefficient off the
    line's cell, and the backprojection."""
    n = N.bit_length() - 1
    s1, s2, d1, d2 = line
    g = torch.Generator(device=device).manual_seed(seed)
    f = torch.randint(-noise, noise + 1, (N, N, N), generator=g, device=device, dtype=torch.int32)
    mask = torch.zeros((N, N, N), dtype=torch.bool, device=device)
    for x in range(N):
        y, z = _lline(n, s1, x) + d1 - N, _lline(n, s2, x) + d2 - N
        if 0 <= y < N and 0 <= z < N:
            mask[x, y, z] = True
    f = f + amplitude * mask.to(torch.int32)
    J = lines_forward(f, [sector])
    flat = J.reshape(-1)
    vals, idx = torch.topk(flat, top)
    peak = [int(v) for v in torch.unravel_index(idx[0], J.shape[1:])]
    own = int(J[0, s1, s2, d1, d2])
    J.zero_()
    J.view(-1)[idx] = vals
    back = lines_adjoint(J, [sector])
    others = vals[1:] if peak == [s1, s2, d1, d2] else vals
    return {"volume": f, "line_mask": mask, "peak": tuple(peak), "line_coefficient": own,
            "largest_other": int(others.max()) if others.numel() else None, "backprojection": back,
            "line_voxels": int(mask.sum())}


def recovered_fraction(result: dict) -> float:
    """Share of the line's voxels among the same number of largest
    backprojected voxels."""
    back, mask = result["backprojection"], result["line_mask"]
    k = int(mask.sum())
    _, idx = torch.topk(back.reshape(-1), k)
    return float(mask.reshape(-1)[idx].float().mean())
