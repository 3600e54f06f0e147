"""Ray in noise (Section 4.1, the DJT example): a digital line buried in white
noise of larger amplitude still stands out in the John domain; keeping only
the largest coefficients and backprojecting them brings the line back.

The volume, the transform, the thresholding and the backprojection all stay
on the GPU.  The caller supplies the line's voxels (a boolean N^3 mask in the
sector's frame) and its cell (s1, s2, d1, d2) of the transform.
"""
from __future__ import annotations

import torch

from . import lines_adjoint, lines_forward


def ray_in_noise(line_mask: torch.Tensor, line, amplitude: int = 16, noise: int = 32, top: int = 16, seed: int = 9,
                 sector: int = 0) -> dict:
    """Add ``amplitude`` on the voxels of ``line_mask`` (a line of ``sector``,
    whose transform cell is ``line`` = (s1, s2, d1, d2)) to integer noise
    uniform in [-noise, noise], take the DJT of that sector, keep the ``top``
    largest coefficients and backproject them.

    Returns the volume, the line's voxel mask, the position of the largest
    coefficient, the line's own coefficient, the largest coefficient off the
    line's cell, and the backprojection."""
    N = int(line_mask.shape[0])
    device = line_mask.device
    s1, s2, d1, d2 = line
    g = torch.Generator(device=device).manual_seed(seed)
    f = torch.randint(-noise, noise + 1, (N, N, N), generator=g, device=device, dtype=torch.int32)
    mask = line_mask.to(torch.bool)
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
