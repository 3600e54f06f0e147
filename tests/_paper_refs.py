"""Small, independent restatements used to pin the oracle (CPU only).

Nothing here is imported by the library or by the oracle.  Each helper
restates a different printed form than the one the oracle implements, so a
mistake in either shows up as a mismatch:

* ``lline_rec``  -- the *recursive* form of eq.(digitalLine)
                    (the oracle uses the summation form).
* ``drt2d_map``  -- the 2D partial-transform recursion eq.(map2D) of Section 2.1
                    (the oracle implements the 3D map eq.(map3D)).
* ``drt2d_def``  -- the 2D definition eq.(GotzfDRT) as a direct sum.
"""
from functools import lru_cache

import numpy as np


@lru_cache(maxsize=None)
def lline_rec(n: int, s: int, u: int) -> int:
    """l^n_s(u) = l^{n-1}_{floor(s/2)}(u_0..u_{n-2}) + u_{n-1} * floor((s+1)/2)."""
    if n == 0:
        return 0
    top = (u >> (n - 1)) & 1
    return lline_rec(n - 1, s // 2, u & ((1 << (n - 1)) - 1)) + top * ((s + 1) // 2)


def lline_rec_table(N: int) -> np.ndarray:
    n = N.bit_length() - 1
    return np.array([[lline_rec(n, s, u) for u in range(N)] for s in range(N)], dtype=np.int64)


def drt2d_map(h: np.ndarray) -> np.ndarray:
    """2D DRT of an N x N image h[x][z] by eq.(map2D); output D[s][e], e in [0, 3N).

    The image is embedded at e in [2N, 3N) (as Algorithm 1 does for planes),
    rows at stage m are sigma + (v << m) with the new slope lsb + 2 sigma, and
    reads past 3N are zero.
    """
    N = h.shape[0]
    n = N.bit_length() - 1
    W = 3 * N
    f = np.zeros((N, W), dtype=np.int64)
    f[:, 2 * N:] = h
    for m in range(n):
        g = np.zeros_like(f)
        for v in range(1 << (n - m - 1)):
            for sg in range(1 << m):
                lo = f[sg + (v << (m + 1))]
                hi = f[sg + (1 << m) + (v << (m + 1))]
                for lsb in range(2):
                    sh = sg + lsb
                    row = lo.copy()
                    row[: W - sh] += hi[sh:]
                    g[lsb + 2 * sg + (v << (m + 1))] = row
        f = g
    return f


def drt2d_def(h: np.ndarray) -> np.ndarray:
    """eq.(GotzfDRT) directly: D[s][e] = sum_u h(u, l_s(u) + e - 2N)."""
    N = h.shape[0]
    n = N.bit_length() - 1
    D = np.zeros((N, 3 * N), dtype=np.int64)
    for s in range(N):
        for e in range(3 * N):
            acc = 0
            for u in range(N):
                z = lline_rec(n, s, u) + e - 2 * N
                if 0 <= z < N:
                    acc += int(h[u, z])
            D[s, e] = acc
    return D
