"""Seeded synthetic input volumes for the 3D DRT/DJT workloads.

This module is shared by the tests, the benchmark and the smoke check.  It holds
none of the transform's arithmetic: no digital lines, no dodecant or sector
maps, no stage maps.  Embedded planes and lines are rasterised with a plain
floor-of-product rule of this module's own, in the volume's own axes, so that
the generator cannot agree with either implementation by construction.

Workloads (numpy ``default_rng(seed)`` throughout):

* ``c1_volume``   -- 32^3 int32, uniform integers 0..255 (seed 1).
* ``c2_volume``   -- N^3 uint8 (N=256 by default): zeros, 1 % of voxels at
                     uniform positions set to uniform 1..255, then 8 digital
                     planes of value 255 at random axis, slopes and intercept
                     (seed 2).  Stands in for the paper's 128^3 voxelised depth
                     map and its 512^3 timing cube (sparse occupancy + planes).
* ``c3_volume``   -- N^3 int16 (N=128), uniform 0..1023 plus 32 digital lines
                     of value 1023 (seed 3); stands in for the paper's
                     ray-in-noise example.
* ``c4_batch``    -- 96 uint8 volumes, sizes 16:30, 32:30, 64:20, 128:10,
                     256:6 shuffled (seed 4), each drawn like ``c2_volume``
                     with seed 4 + i.
* ``c5_batch``    -- 8 x 128^3 float32, standard normal (seed 5).
* ``images_2d``   -- B x N x N uint8 images (B=512, N=256 by default): zeros,
                     5 % of pixels at uniform positions set to uniform 1..255,
                     then 4 straight lines of value 255 per image at random
                     slope and intercept (seed 6); the by-product 2D DRT's
                     batch (the paper gives no 2D workload of its own).
* ``phantom``     -- N^3 float32 (N=128): a sum of 6 solid ellipsoids of
                     random centre, semi-axes N/10..N/3 and intensity 0.2..1
                     (seed 7); stands in for the paper's 128^3 head and spine
                     MRI inversions (the scans themselves are not available).
* ``dense_u8``    -- N^3 uint8 uniform 0..255, drawn directly as bytes (the
                     maximum-size tests, N up to 1024).
* ``raw_int32``   -- full-range uniform int32 from the generator's raw bits
                     (multi-GB lines cotangents at N = 128).
"""
from __future__ import annotations

import numpy as np

C4_COUNTS = {16: 30, 32: 30, 64: 20, 128: 10, 256: 6}


def _raster(u: np.ndarray, slope: int, N: int) -> np.ndarray:
    """floor(slope * u / (N - 1)) for integer slope in [-(N-1), N-1]."""
    if N == 1:
        return np.zeros_like(u)
    return np.floor_divide(slope * u, N - 1)


def _embed_planes(f: np.ndarray, rng: np.random.Generator, count: int, value: int) -> list:
    """Set voxels of ``count`` random digital planes to ``value``.

    A plane is driven by axis a: for every (u, v) on the two other axes the
    voxel at a = floor(p u/(N-1)) + floor(q v/(N-1)) + c is set, with p, q
    uniform in [-(N-1), N-1] and c chosen so the plane crosses the cube.
    Returns the drawn parameters.
    """
    N = f.shape[0]
    params = []
    u, v = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    for _ in range(count):
        a = int(rng.integers(0, 3))
        p = int(rng.integers(-(N - 1), N))
        q = int(rng.integers(-(N - 1), N))
        base = _raster(u, p, N) + _raster(v, q, N)
        lo, hi = int(base.min()), int(base.max())
        c = int(rng.integers(-hi, N - lo))  # some voxel of the plane lands inside
        w = base + c
        ok = (w >= 0) & (w < N)
        uu, vv, ww = u[ok], v[ok], w[ok]
        if a == 0:
            f[ww, uu, vv] = value
        elif a == 1:
            f[uu, ww, vv] = value
        else:
            f[uu, vv, ww] = value
        params.append((a, p, q, c))
    return params


def _embed_lines(f: np.ndarray, rng: np.random.Generator, count: int, value: int) -> list:
    """Set voxels of ``count`` random digital lines to ``value``.

    A line is driven by axis a: for t in [0, N) the two other coordinates are
    floor(p t/(N-1)) + c1 and floor(q t/(N-1)) + c2.
    """
    N = f.shape[0]
    t = np.arange(N)
    params = []
    for _ in range(count):
        a = int(rng.integers(0, 3))
        p = int(rng.integers(-(N - 1), N))
        q = int(rng.integers(-(N - 1), N))
        rb, rc = _raster(t, p, N), _raster(t, q, N)
        c1 = int(rng.integers(-int(rb.max()), N - int(rb.min())))
        c2 = int(rng.integers(-int(rc.max()), N - int(rc.min())))
        b, c = rb + c1, rc + c2
        ok = (b >= 0) & (b < N) & (c >= 0) & (c < N)
        tt, bb, cc = t[ok], b[ok], c[ok]
        if a == 0:
            f[tt, bb, cc] = value
        elif a == 1:
            f[cc, tt, bb] = value
        else:
            f[bb, cc, tt] = value
        params.append((a, p, q, c1, c2))
    return params


def c1_volume(N: int = 32, seed: int = 1) -> np.ndarray:
    """Dense int32 volume, uniform integers 0..255."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, size=(N, N, N), dtype=np.int64).astype(np.int32)


def c2_volume(N: int = 256, seed: int = 2, planes: int = 8) -> np.ndarray:
    """Sparse uint8 volume: 1 % occupancy at 1..255 plus ``planes`` planes of 255."""
    rng = np.random.default_rng(seed)
    f = np.zeros(N * N * N, dtype=np.uint8)
    k = max(1, (N * N * N) // 100)
    pos = rng.choice(N * N * N, size=k, replace=False)
    f[pos] = rng.integers(1, 256, size=k, dtype=np.int64).astype(np.uint8)
    f = f.reshape(N, N, N)
    _embed_planes(f, rng, planes, 255)
    return f


def c3_volume(N: int = 128, seed: int = 3, lines: int = 32) -> np.ndarray:
    """Dense int16 volume, uniform 0..1023, plus ``lines`` lines of 1023."""
    rng = np.random.default_rng(seed)
    f = rng.integers(0, 1024, size=(N, N, N), dtype=np.int64).astype(np.int16)
    _embed_lines(f, rng, lines, 1023)
    return f


def c4_sizes(seed: int = 4) -> list:
    """The 96 volume sizes of the ragged batch, shuffled."""
    rng = np.random.default_rng(seed)
    sizes = [N for N, c in C4_COUNTS.items() for _ in range(c)]
    rng.shuffle(sizes)
    return [int(s) for s in sizes]


def c4_batch(seed: int = 4, sizes=None) -> list:
    """96 uint8 volumes of ragged size, each drawn like ``c2_volume``."""
    sizes = c4_sizes(seed) if sizes is None else sizes
    return [c2_volume(N, seed + i) for i, N in enumerate(sizes)]


def c5_batch(N: int = 128, batch: int = 8, seed: int = 5) -> np.ndarray:
    """``batch`` float32 volumes of standard normal values."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(size=(batch, N, N, N), dtype=np.float32)


def random_int32(shape, seed: int, lo: int = -(2 ** 31), hi: int = 2 ** 31) -> np.ndarray:
    """Uniform int32 over [lo, hi) (full range by default, exercises wrapping)."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi, size=shape, dtype=np.int64).astype(np.int32)


def raw_int32(shape, seed: int) -> np.ndarray:
    """Uniform int32 over the full range, taken straight from the generator's
    raw 64-bit output (fast enough for multi-GB cotangents)."""
    n = int(np.prod(shape))
    rng = np.random.default_rng(seed)
    raw = rng.bit_generator.random_raw((n + 1) // 2)
    return raw.view(np.int32)[:n].reshape(shape)


def random_float(shape, seed: int) -> np.ndarray:
    """Standard normal float32."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(size=shape, dtype=np.float32)


def images_2d(N: int = 256, batch: int = 512, seed: int = 6, lines: int = 4) -> np.ndarray:
    """``batch`` sparse uint8 images with ``lines`` straight lines of 255 each."""
    rng = np.random.default_rng(seed)
    f = np.zeros((batch, N * N), dtype=np.uint8)
    k = max(1, (N * N) // 20)
    for b in range(batch):
        pos = rng.choice(N * N, size=k, replace=False)
        f[b, pos] = rng.integers(1, 256, size=k, dtype=np.int64).astype(np.uint8)
    f = f.reshape(batch, N, N)
    u = np.arange(N)
    for b in range(batch):
        for _ in range(lines):
            slope = int(rng.integers(-(N - 1), N))
            icpt = int(rng.integers(0, N))
            v = icpt + _raster(u, slope, N)
            ok = (v >= 0) & (v < N)
            if rng.integers(0, 2):
                f[b, u[ok], v[ok]] = 255
            else:
                f[b, v[ok], u[ok]] = 255
    return f


def phantom(N: int = 128, seed: int = 7, blobs: int = 6) -> np.ndarray:
    """Sum of ``blobs`` solid ellipsoids, float32."""
    rng = np.random.default_rng(seed)
    x = (np.arange(N, dtype=np.float64) + 0.5) / N
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    f = np.zeros((N, N, N), dtype=np.float64)
    for _ in range(blobs):
        c = rng.uniform(0.3, 0.7, size=3)
        a = rng.uniform(0.1, 1 / 3, size=3)
        v = rng.uniform(0.2, 1.0)
        f += v * ((((X - c[0]) / a[0]) ** 2 + ((Y - c[1]) / a[1]) ** 2 + ((Z - c[2]) / a[2]) ** 2) <= 1.0)
    return f.astype(np.float32)


def dense_u8(N: int, seed: int) -> np.ndarray:
    """Uniform uint8 volume, generated without a wider intermediate."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, size=(N, N, N), dtype=np.uint8)
