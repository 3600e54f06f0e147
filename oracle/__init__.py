"""Plain CPU oracle for the 3D multiscale DRT of planes and DJT of lines.

TEST INFRASTRUCTURE ONLY.  This package is the independent reference that the
GPU library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with
the CUDA library (``paper_2501_13664_gb300``) and never imports it.

The arithmetic lives in ``drt3d_oracle.c`` (plain C, compiled with gcc on first
use); this module only marshals numpy arrays.  Paper references are to
Marichal-Hernandez et al., "Three-dimensional multiscale discrete Radon and
John transforms" (arXiv 2501.13664):

* ``lline``                 -- eq.(digitalLine), Section 2.1
* ``planes_brute``          -- eq.(3DfDRT), Section 3.1 (definition, scatter)
* ``planes_alg1``           -- Algorithm 1 with eq.(map3D)
* ``planes_forward``        -- Algorithm 2's twelve dodecants (input remap)
* ``planes_adjoint``        -- Section 5.1, eq.(invmap3Dsummation)
* ``planes_inverse``        -- exact integer stage inverse derived from
                               eq.(map2D)/eq.(map3D) and Algorithm 1's zero
                               embedding (the paper's own inverse is the
                               iterative scheme of Section 5.2)
* ``lines_brute``           -- eq.(3DfDJT), Section 4.1
* ``lines_alg3``            -- Algorithm 3 with eq.(map3DJ)
* ``lines_forward``         -- the twelve line sectors of Section 4.1
* ``drt2d_brute``           -- the 2D DRT of lines by its definition
                               (stage n of eq.(our2Dfm)), Section 2.1
* ``drt2d_map2d``           -- the 2D stage recursion eq.(map2D)
* ``drt2d_forward``         -- the four quadrants of Section 2.2 (axes
                               swapped and/or flipped), batched
* ``press`` (submodule)     -- Section 5.2's iterative inverse: adjoint +
                               high-pass filter h, multigrid with P and S

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
invariants and brute force; ``cond_number`` (Table "condNumber") is the one
quantity whose paper values are not reproduced ("parity unpinned").
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "drt3d_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle_drt3d.so")
_lock = threading.Lock()
_lib = None

N_DODECANTS = 12
N_SECTORS = 12


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc into ``oracle/_build`` and return its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I = ctypes.c_int
        I64 = ctypes.c_int64
        sig = {
            "drto_lline": (I64, [I, I64, I64]),
            "drto_dodecant_src": (I64, [I, I, I, I, I]),
            "drto_sector_src": (I64, [I, I, I, I, I]),
            "drto_gather_dodecant_4": (None, [I, I, P, P]),
            "drto_gather_dodecant_8": (None, [I, I, P, P]),
            "drto_scatter_add_dodecant_f64": (None, [I, I, P, P]),
            "drto_scatter_add_dodecant_i32": (None, [I, I, P, P]),
            "drto_gather_sector_4": (None, [I, I, P, P]),
            "drto_dodecant_index_table": (None, [I, I, P]),
            "drto_sector_index_table": (None, [I, I, P]),
            "drto_planes_brute_i64": (None, [I, P, P]),
            "drto_planes_brute_f64": (None, [I, P, P]),
            "drto_planes_cell_i64": (I64, [I, P, I, I, I]),
            "drto_planes_adjoint_brute_f64": (None, [I, P, P]),
            "drto_planes_alg1_i32": (I, [I, P, P]),
            "drto_planes_alg1_f64": (I, [I, P, P]),
            "drto_planes_adjoint_i32": (I, [I, P, P]),
            "drto_planes_adjoint_f64": (I, [I, P, P]),
            "drto_planes_inverse_i32": (I, [I, P, P]),
            "drto_lines_brute_i64": (None, [I, P, P]),
            "drto_lines_cell_i64": (I64, [I, P, I, I, I, I]),
            "drto_lines_alg3_i32": (I, [I, P, P]),
            "drto_lines_adjoint_brute_i64": (None, [I, P, P]),
            "drto_lines_adjoint_i32": (I, [I, P, P]),
            "drto_drt2d_brute_i64": (None, [I, P, P]),
            "drto_drt2d_map2d_i32": (I, [I, P, P]),
            "drto_drt2d_map2d_f64": (I, [I, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _check_N(N: int) -> int:
    if N < 2 or N > 1024 or (N & (N - 1)):
        raise ValueError(f"N must be a power of two in [2, 1024], got {N}")
    return N.bit_length() - 1


def _cube(f: np.ndarray) -> int:
    if f.ndim != 3 or not (f.shape[0] == f.shape[1] == f.shape[2]):
        raise ValueError(f"expected an N x N x N volume, got shape {f.shape}")
    N = f.shape[0]
    _check_N(N)
    return N


# --------------------------------------------------------------------------
# Geometry
# --------------------------------------------------------------------------
def lline(n: int, s: int, u: int) -> int:
    """l^n_s(u) of eq.(digitalLine)."""
    return int(_load().drto_lline(n, s, u))


def lline_table(N: int) -> np.ndarray:
    """Table T[s][u] = l^n_s(u) for s, u in [0, N)."""
    n = _check_N(N)
    lib = _load()
    return np.array([[lib.drto_lline(n, s, u) for u in range(N)] for s in range(N)], dtype=np.int64)


def dodecant_src_index(N: int, k: int) -> np.ndarray:
    """Flat index into f of g_k(x', y', z') for every (x', y', z'), shape N^3."""
    idx = np.empty((N, N, N), dtype=np.int64)
    _load().drto_dodecant_index_table(N, k, _ptr(idx))
    return idx


def sector_src_index(N: int, k: int) -> np.ndarray:
    """Flat index into f of sector k's frame volume at every (x', y', z')."""
    idx = np.empty((N, N, N), dtype=np.int64)
    _load().drto_sector_index_table(N, k, _ptr(idx))
    return idx


def dodecant_volume(f: np.ndarray, k: int) -> np.ndarray:
    """g_k = f seen in dodecant k's frame (Algorithm 2 input permute/flip)."""
    N = _cube(f)
    f = np.ascontiguousarray(f)
    if f.dtype.itemsize == 4:
        g = np.empty_like(f)
        _load().drto_gather_dodecant_4(N, k, _ptr(f), _ptr(g))
    elif f.dtype.itemsize == 8:
        g = np.empty_like(f)
        _load().drto_gather_dodecant_8(N, k, _ptr(f), _ptr(g))
    else:
        g = dodecant_volume(f.astype(np.int32), k).astype(f.dtype)
    return g


def sector_volume(f: np.ndarray, k: int) -> np.ndarray:
    """f seen in DJT sector k's frame (x' along the driving axis)."""
    N = _cube(f)
    f = np.ascontiguousarray(f)
    if f.dtype.itemsize != 4:
        return sector_volume(f.astype(np.int32), k).astype(f.dtype)
    g = np.empty_like(f)
    _load().drto_gather_sector_4(N, k, _ptr(f), _ptr(g))
    return g


# --------------------------------------------------------------------------
# Planes
# --------------------------------------------------------------------------
def planes_brute(g: np.ndarray) -> np.ndarray:
    """eq.(3DfDRT) by scatter, one dodecant frame.  int64 or float64 output."""
    N = _cube(g)
    R = None
    if np.issubdtype(g.dtype, np.floating):
        gg = np.ascontiguousarray(g, dtype=np.float64)
        R = np.empty((N, N, 3 * N), dtype=np.float64)
        _load().drto_planes_brute_f64(N, _ptr(gg), _ptr(R))
    else:
        gg = np.ascontiguousarray(g, dtype=np.int64)
        R = np.empty((N, N, 3 * N), dtype=np.int64)
        _load().drto_planes_brute_i64(N, _ptr(gg), _ptr(R))
    return R


def planes_cell(g: np.ndarray, s1: int, s2: int, d: int) -> int:
    """One output cell of eq.(3DfDRT), exact int64, one dodecant frame."""
    N = _cube(g)
    gg = np.ascontiguousarray(g, dtype=np.int32)
    return int(_load().drto_planes_cell_i64(N, _ptr(gg), s1, s2, d))


def planes_alg1(g: np.ndarray) -> np.ndarray:
    """Algorithm 1 for one dodecant frame: int32 (wrapping) or float64."""
    N = _cube(g)
    lib = _load()
    if np.issubdtype(g.dtype, np.floating):
        gg = np.ascontiguousarray(g, dtype=np.float64)
        R = np.empty((N, N, 3 * N), dtype=np.float64)
        rc = lib.drto_planes_alg1_f64(N, _ptr(gg), _ptr(R))
    else:
        gg = np.ascontiguousarray(g.astype(np.int32, copy=False))
        R = np.empty((N, N, 3 * N), dtype=np.int32)
        rc = lib.drto_planes_alg1_i32(N, _ptr(gg), _ptr(R))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return R


def planes_forward(f: np.ndarray, dodecants=range(N_DODECANTS), exact: str = "alg1") -> np.ndarray:
    """All requested dodecants: out[i] is dodecant ``dodecants[i]``.

    Integer inputs give int32 (wrapping) results, floating inputs float64.
    ``exact='brute'`` uses the eq.(3DfDRT) scatter instead of Algorithm 1.
    """
    N = _cube(f)
    ks = list(dodecants)
    is_float = np.issubdtype(f.dtype, np.floating)
    base = f.astype(np.float64) if is_float else f.astype(np.int32)
    outs = []
    for k in ks:
        g = dodecant_volume(base, k)
        if exact == "brute":
            R = planes_brute(g)
            outs.append(R if is_float else R.astype(np.int64).astype(np.int32, casting="unsafe"))
        else:
            outs.append(planes_alg1(g))
    return np.stack(outs) if outs else np.empty((0, N, N, 3 * N))


def planes_adjoint(Rbar: np.ndarray, dodecants=range(N_DODECANTS)) -> np.ndarray:
    """Backprojection summed over dodecants: sum_k g_k^T(A_k^T Rbar[i]).

    ``Rbar`` has shape (len(dodecants), N, N, 3N); int32 (wrapping) or float64.
    Dodecants are accumulated in the given order.
    """
    ks = list(dodecants)
    N = Rbar.shape[1]
    _check_N(N)
    lib = _load()
    is_float = np.issubdtype(Rbar.dtype, np.floating)
    if is_float:
        acc = np.zeros((N, N, N), dtype=np.float64)
        for i, k in enumerate(ks):
            rb = np.ascontiguousarray(Rbar[i], dtype=np.float64)
            gb = np.empty((N, N, N), dtype=np.float64)
            if lib.drto_planes_adjoint_f64(N, _ptr(rb), _ptr(gb)) != 0:
                raise MemoryError
            lib.drto_scatter_add_dodecant_f64(N, k, _ptr(gb), _ptr(acc))
    else:
        acc = np.zeros((N, N, N), dtype=np.int32)
        for i, k in enumerate(ks):
            rb = np.ascontiguousarray(Rbar[i], dtype=np.int32)
            gb = np.empty((N, N, N), dtype=np.int32)
            if lib.drto_planes_adjoint_i32(N, _ptr(rb), _ptr(gb)) != 0:
                raise MemoryError
            lib.drto_scatter_add_dodecant_i32(N, k, _ptr(gb), _ptr(acc))
    return acc


def planes_adjoint_frame(Rbar_k: np.ndarray) -> np.ndarray:
    """Adjoint of Algorithm 1 alone (one dodecant frame, no remap)."""
    N = Rbar_k.shape[0]
    lib = _load()
    if np.issubdtype(Rbar_k.dtype, np.floating):
        rb = np.ascontiguousarray(Rbar_k, dtype=np.float64)
        gb = np.empty((N, N, N), dtype=np.float64)
        rc = lib.drto_planes_adjoint_f64(N, _ptr(rb), _ptr(gb))
    else:
        rb = np.ascontiguousarray(Rbar_k, dtype=np.int32)
        gb = np.empty((N, N, N), dtype=np.int32)
        rc = lib.drto_planes_adjoint_i32(N, _ptr(rb), _ptr(gb))
    if rc != 0:
        raise MemoryError
    return gb


def planes_adjoint_brute_frame(Rbar_k: np.ndarray) -> np.ndarray:
    """Transpose of the eq.(3DfDRT) scatter, one dodecant frame, float64."""
    N = Rbar_k.shape[0]
    rb = np.ascontiguousarray(Rbar_k, dtype=np.float64)
    gb = np.empty((N, N, N), dtype=np.float64)
    _load().drto_planes_adjoint_brute_f64(N, _ptr(rb), _ptr(gb))
    return gb


def planes_inverse(R_k: np.ndarray, k: int = 0):
    """Exact integer inverse of dodecant k's transform.

    Returns ``(f, in_range)``: the volume in the original frame (int32) and
    whether ``R_k`` lies in the range of the forward map.
    """
    N = R_k.shape[0]
    _check_N(N)
    rr = np.ascontiguousarray(R_k, dtype=np.int32)
    g = np.empty((N, N, N), dtype=np.int32)
    rc = _load().drto_planes_inverse_i32(N, _ptr(rr), _ptr(g))
    if rc < 0:
        raise MemoryError
    # back to the original frame: f[src(x',y',z')] = g[x',y',z']
    f = np.empty(N * N * N, dtype=np.int32)
    f[dodecant_src_index(N, k).ravel()] = g.ravel()
    return f.reshape(N, N, N), rc == 0


# --------------------------------------------------------------------------
# Lines
# --------------------------------------------------------------------------
def lines_brute(g: np.ndarray) -> np.ndarray:
    """eq.(3DfDJT) by scatter, one sector frame, int64, shape (N,N,2N,2N)."""
    N = _cube(g)
    gg = np.ascontiguousarray(g, dtype=np.int64)
    J = np.empty((N, N, 2 * N, 2 * N), dtype=np.int64)
    _load().drto_lines_brute_i64(N, _ptr(gg), _ptr(J))
    return J


def lines_cell(g: np.ndarray, s1: int, s2: int, d1: int, d2: int) -> int:
    """One output cell of eq.(3DfDJT), exact int64, one sector frame."""
    N = _cube(g)
    gg = np.ascontiguousarray(g, dtype=np.int32)
    return int(_load().drto_lines_cell_i64(N, _ptr(gg), s1, s2, d1, d2))


def lines_alg3(g: np.ndarray) -> np.ndarray:
    """Algorithm 3 for one sector frame, int32 wrapping, shape (N,N,2N,2N)."""
    N = _cube(g)
    gg = np.ascontiguousarray(g.astype(np.int32, copy=False))
    J = np.empty((N, N, 2 * N, 2 * N), dtype=np.int32)
    if _load().drto_lines_alg3_i32(N, _ptr(gg), _ptr(J)) != 0:
        raise MemoryError("oracle allocation failed")
    return J


def lines_forward(f: np.ndarray, sectors=range(N_SECTORS), exact: str = "alg3") -> np.ndarray:
    """Requested sectors of the DJT: out[i] is sector ``sectors[i]`` (int32)."""
    _cube(f)
    base = f.astype(np.int32)
    outs = []
    for k in sectors:
        g = sector_volume(base, k)
        if exact == "brute":
            outs.append(lines_brute(g).astype(np.int32, casting="unsafe"))
        else:
            outs.append(lines_alg3(g))
    return np.stack(outs)


def lines_adjoint_brute_frame(Jbar_k: np.ndarray) -> np.ndarray:
    """Transposed scatter of eq.(3DfDJT) for one sector frame, int64, (N,N,N)."""
    N = Jbar_k.shape[0]
    _check_N(N)
    jb = np.ascontiguousarray(Jbar_k, dtype=np.int64)
    g = np.empty((N, N, N), dtype=np.int64)
    _load().drto_lines_adjoint_brute_i64(N, _ptr(jb), _ptr(g))
    return g


def lines_adjoint_frame(Jbar_k: np.ndarray) -> np.ndarray:
    """Algorithm 3 reversed with eq.(invmap3DJsummation), one sector frame, int32 wrapping."""
    N = Jbar_k.shape[0]
    _check_N(N)
    jb = np.ascontiguousarray(Jbar_k, dtype=np.int32)
    g = np.empty((N, N, N), dtype=np.int32)
    if _load().drto_lines_adjoint_i32(N, _ptr(jb), _ptr(g)) != 0:
        raise MemoryError("oracle allocation failed")
    return g


def lines_adjoint(Jbar: np.ndarray, sectors=range(N_SECTORS)) -> np.ndarray:
    """Backprojection of lines summed over sectors (int32 wrapping):
    f_bar = sum_k (sector k's frame map)^T (J_k^T Jbar[i]), in the given order.
    ``Jbar`` has shape (len(sectors), N, N, 2N, 2N)."""
    ks = list(sectors)
    N = Jbar.shape[1]
    _check_N(N)
    acc = np.zeros(N * N * N, dtype=np.int64)
    for i, k in enumerate(ks):
        g = lines_adjoint_frame(Jbar[i]).astype(np.int64).ravel()
        np.add.at(acc, sector_src_index(N, k).ravel(), g)
    return (acc & 0xFFFFFFFF).astype(np.uint32).view(np.int32).reshape(N, N, N)


def lines_cell_global(f: np.ndarray, k: int, s1: int, s2: int, d1: int, d2: int) -> int:
    """One DJT cell of sector k, computed from the original-frame volume."""
    N = _cube(f)
    lib = _load()
    n = N.bit_length() - 1
    acc = 0
    ff = f.reshape(-1)
    for x in range(N):
        y = lib.drto_lline(n, s1, x) + d1 - N
        z = lib.drto_lline(n, s2, x) + d2 - N
        if 0 <= y < N and 0 <= z < N:
            acc += int(ff[lib.drto_sector_src(N, k, x, y, z)])
    return acc


def planes_cell_global(f: np.ndarray, k: int, s1: int, s2: int, d: int) -> int:
    """One planes cell of dodecant k, computed from the original-frame volume."""
    N = _cube(f)
    g = dodecant_volume(f.astype(np.int32), k)
    return planes_cell(g, s1, s2, d)


# --------------------------------------------------------------------------
# Global 4N x 4N x (3N-2) layout (Algorithm 2: OutOrder, DodecantCoords).
# --------------------------------------------------------------------------
# Algorithm 2's output tables as printed (1-based dimension numbers; a
# negative entry flips that output dimension after the permutation).
OUT_ORDER = [(-2, -1, 3), (-1, 2, 3), (2, 1, 3), (1, -2, 3),
             (2, 1, 3), (1, -2, 3), (-1, 2, 3), (-2, -1, 3),
             (2, 1, 3), (-1, 2, 3), (1, -2, 3), (-2, -1, 3)]
DODECANT_COORDS = [(1, 1), (1, 2), (2, 2), (2, 1),
                   (0, 2), (0, 1), (3, 2), (3, 1),
                   (2, 0), (1, 0), (2, 3), (1, 3)]


def place_global(R: np.ndarray) -> np.ndarray:
    """Algorithm 2's merge of the 12 dodecant outputs R[k][s1][s2][d]
    (d in [0, 3N)) into one 4N x 4N x (3N-2) array: drop displacements 0 and 1
    (always zero; the global array keeps 3N-2), permute the dodecant's
    dimensions as abs(OutOrder[k]) (output dimension i takes input dimension
    |OutOrder[k][i]|), flip the output dimensions with negative entries, and
    store the block at (DodecantCoords[k][0] N, DodecantCoords[k][1] N).
    The four unused blocks stay zero."""
    N = R.shape[1]
    G = np.zeros((4 * N, 4 * N, 3 * N - 2), dtype=R.dtype)
    for k in range(12):
        A = R[k][:, :, 2:]
        order = OUT_ORDER[k]
        A = np.transpose(A, [abs(o) - 1 for o in order])
        for dim, o in enumerate(order):
            if o < 0:
                A = np.flip(A, axis=dim)
        b0, b1 = DODECANT_COORDS[k]
        G[b0 * N:(b0 + 1) * N, b1 * N:(b1 + 1) * N, :] = A
    return G


def planes_global(f: np.ndarray) -> np.ndarray:
    """The 3D DRT of a cube in Algorithm 2's global layout (int32)."""
    return place_global(planes_forward(f))


def dodecant_frame_axes(N: int, k: int) -> list:
    """For frame axes x', y', z' of dodecant k: (original axis, +1 or -1)."""
    lib = _load()
    o = lib.drto_dodecant_src(N, k, 0, 0, 0)
    strides = {N * N: 0, N: 1, 1: 2}
    out = []
    for v in [(1, 0, 0), (0, 1, 0), (0, 0, 1)]:
        d = lib.drto_dodecant_src(N, k, *v) - o
        out.append((strides[abs(d)], 1 if d > 0 else -1))
    return out


# --------------------------------------------------------------------------
# Dense operator (tiny N) for condition numbers (Table "condNumber").
# --------------------------------------------------------------------------
def planes_matrix(N: int) -> np.ndarray:
    """Dense matrix of the 12-dodecant forward operator, rows = output cells."""
    cols = []
    for i in range(N ** 3):
        e = np.zeros(N ** 3, dtype=np.int32)
        e[i] = 1
        cols.append(planes_forward(e.reshape(N, N, N)).reshape(-1).astype(np.float64))
    return np.stack(cols, axis=1)


def cond_number(N: int) -> float:
    """sigma_max / sigma_min of the 12-dodecant operator.  Parity unpinned:
    the paper's printed values are not reproduced by this operator."""
    s = np.linalg.svd(planes_matrix(N), compute_uv=False)
    return float(s[0] / s[-1])


# --------------------------------------------------------------------------
# 2D DRT of lines (Section 2.1, eq.(map2D)) and its four quadrants.
# --------------------------------------------------------------------------
N_QUADRANTS = 4


def _square(f: np.ndarray) -> int:
    if f.ndim != 2 or f.shape[0] != f.shape[1]:
        raise ValueError("expected an N x N image")
    _check_N(f.shape[0])
    return f.shape[0]


def drt2d_brute(f: np.ndarray) -> np.ndarray:
    """R[s][d] = sum_u f(u, l_s(u) + d - N) by scatter, int64 or float64, (N, 2N)."""
    N = _square(f)
    if np.issubdtype(f.dtype, np.floating):
        # exact enough in float64 for the sizes tested: evaluate the same
        # scatter with numpy on the lline table
        L = lline_table(N)
        R = np.zeros((N, 2 * N), dtype=np.float64)
        y = np.arange(N)
        for s in range(N):
            for u in range(N):
                np.add.at(R[s], y - L[s, u] + N, f[u].astype(np.float64))
        return R
    ff = np.ascontiguousarray(f, dtype=np.int64)
    R = np.empty((N, 2 * N), dtype=np.int64)
    _load().drto_drt2d_brute_i64(N, _ptr(ff), _ptr(R))
    return R


def drt2d_map2d(f: np.ndarray) -> np.ndarray:
    """The n stages of eq.(map2D) on one image: int32 wrapping for integer
    input, float64 for floating input, shape (N, 2N)."""
    N = _square(f)
    lib = _load()
    if np.issubdtype(f.dtype, np.floating):
        ff = np.ascontiguousarray(f, dtype=np.float64)
        R = np.empty((N, 2 * N), dtype=np.float64)
        rc = lib.drto_drt2d_map2d_f64(N, _ptr(ff), _ptr(R))
    else:
        ff = np.ascontiguousarray(f.astype(np.int32, copy=False))
        R = np.empty((N, 2 * N), dtype=np.int32)
        rc = lib.drto_drt2d_map2d_i32(N, _ptr(ff), _ptr(R))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return R


def quadrant_image(f: np.ndarray, q: int) -> np.ndarray:
    """Image seen by quadrant q (Section 2.2: the basic quadrant reused on
    swapped and/or flipped copies of the input).  Bit 1 of q swaps the axes
    (lines driven by y instead of x), bit 0 reverses the other axis:
    f_q(u, y) = f(u, y), f(u, N-1-y), f(y, u), f(N-1-y, u) for q = 0..3."""
    if not 0 <= q < N_QUADRANTS:
        raise ValueError("quadrant out of range")
    g = f.T if q & 2 else f
    return g[:, ::-1] if q & 1 else g


def drt2d_forward(imgs: np.ndarray, quadrants=range(N_QUADRANTS), exact: str = "map2d") -> np.ndarray:
    """2D DRT of a batch of images (B, N, N) for the given quadrants:
    out[b][i] is quadrant ``quadrants[i]`` of image b, shape (B, nq, N, 2N)
    (int32 wrapping for integer input, float64 for floating input)."""
    if imgs.ndim != 3:
        raise ValueError("expected (B, N, N) images")
    qs = list(quadrants)
    fn = drt2d_brute if exact == "brute" else drt2d_map2d
    out = [[fn(np.ascontiguousarray(quadrant_image(im, q))) for q in qs] for im in imgs]
    res = np.array(out)
    if exact == "brute" and not np.issubdtype(imgs.dtype, np.floating):
        res = res.astype(np.int32, casting="unsafe")
    return res
