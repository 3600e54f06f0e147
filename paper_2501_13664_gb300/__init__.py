"""GB300-native 3D multiscale discrete Radon transform of planes and discrete
John transform of lines (Marichal-Hernandez et al., arXiv 2501.13664).

This is the thin PyTorch-facing layer over the C-ABI library ``libdrt3d``
(``include/drt3d.h``).  PyTorch provides device memory and streams; every
arithmetic step runs in the library's sm_103a kernels.  There is no CPU
fallback: if the library cannot be built or loaded, these functions raise.

Public functions (device tensors in, device tensors out; a CPU input tensor is
copied to the current CUDA device and the result copied back):

* ``planes_forward(vol, dodecants)``   -> (k, N, N, 3N) int32 / float32
* ``planes_adjoint(cot, dodecants)``   -> (N, N, N)
* ``planes_inverse(R_k, dodecant)``    -> (N, N, N) int32
* ``lines_forward(vol, sectors)``      -> (k, N, N, 2N, 2N) int32
* ``lines_adjoint(cot, sectors)``      -> (N, N, N) int32
* ``drt2d_forward(imgs, quadrants)``   -> (B, q, N, 2N) int32 / float32
* ``planes_press_inverse(R, iters)``   -> (N, N, N) float32, Section 5.2's
                                          iterative (multigrid) inverse
* ``PlanesTransform``                  -- torch.autograd.Function (float32)
"""
from __future__ import annotations

import ctypes
import threading

import torch

from . import _abi
from ._abi import DRT3DError

ALL = 0xFFF

_TORCH_DTYPES = {torch.uint8: "u8", torch.int16: "i16", torch.int32: "i32", torch.float32: "f32"}


def _mask(sel) -> int:
    if isinstance(sel, int):
        m = sel
    else:
        m = 0
        for k in sel:
            if not 0 <= int(k) < 12:
                raise ValueError(f"dodecant/sector index out of range: {k}")
            m |= 1 << int(k)
    if m <= 0 or m > ALL:
        raise ValueError(f"bad dodecant/sector mask {m:#x}")
    return m


def _count(m: int) -> int:
    return bin(m).count("1")


class Plan:
    """A libdrt3d plan for N^3 volumes of one dtype on the current device."""

    def __init__(self, N: int, dtype: torch.dtype):
        if dtype not in _TORCH_DTYPES:
            raise TypeError(f"unsupported dtype {dtype}")
        self.N = int(N)
        self.dtype = dtype
        self._lib = _abi.lib()
        h = ctypes.c_void_p()
        _abi.check(self._lib.drt3d_plan_create(ctypes.byref(h), self.N, _abi.DTYPES[_TORCH_DTYPES[dtype]], 0),
                   "drt3d_plan_create")
        self.handle = h
        self.device = torch.cuda.current_device()

    def workspace_bytes(self, op: str) -> int:
        v = ctypes.c_size_t()
        _abi.check(self._lib.drt3d_workspace_bytes(self.handle, _abi.OPS[op], ctypes.byref(v)),
                   "drt3d_workspace_bytes")
        return int(v.value)

    def workspace(self, op: str) -> torch.Tensor:
        return torch.empty(max(16, self.workspace_bytes(op)), dtype=torch.uint8, device=f"cuda:{self.device}")

    def device_error(self, stream=None) -> int:
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        return int(self._lib.drt3d_get_device_error(self.handle, ctypes.c_void_p(s)))

    def set_profiling(self, on: bool) -> None:
        """Record per-launch CUDA-event times of this plan's calls (diagnostic)."""
        _abi.check(self._lib.drt3d_set_profiling(self.handle, 1 if on else 0), "drt3d_set_profiling")

    def profiled_launches(self) -> list:
        """[(name, ms, algorithmic_bytes)] of every launch recorded since enabling."""
        cnt = ctypes.c_int()
        _abi.check(self._lib.drt3d_profiled_launches(self.handle, None, None, 0, ctypes.byref(cnt)),
                   "drt3d_profiled_launches")
        n = cnt.value
        ms = (ctypes.c_float * max(1, n))()
        by = (ctypes.c_double * max(1, n))()
        _abi.check(self._lib.drt3d_profiled_launches(self.handle, ms, by, n, ctypes.byref(cnt)),
                   "drt3d_profiled_launches")
        return [(self._lib.drt3d_profiled_launch_name(self.handle, i).decode(), float(ms[i]), float(by[i]))
                for i in range(n)]

    def set_schedule(self, groups) -> None:
        """Stage-fusion split of the planes forward (e.g. (4, 4) or (3, 3, 2))."""
        arr = (ctypes.c_int * len(groups))(*[int(g) for g in groups])
        _abi.check(self._lib.drt3d_plan_set_schedule(self.handle, len(groups), arr), "drt3d_plan_set_schedule")

    def schedule(self) -> tuple:
        ng = ctypes.c_int()
        arr = (ctypes.c_int * 8)()
        _abi.check(self._lib.drt3d_plan_get_schedule(self.handle, ctypes.byref(ng), arr), "drt3d_plan_get_schedule")
        return tuple(arr[i] for i in range(ng.value))

    def set_adjoint_schedule(self, groups) -> None:
        """Stage-fusion split of the planes adjoint; None or () follows the
        forward's schedule (see drt3d_plan_set_adjoint_schedule)."""
        groups = tuple(groups or ())
        arr = (ctypes.c_int * max(1, len(groups)))(*[int(g) for g in groups])
        _abi.check(self._lib.drt3d_plan_set_adjoint_schedule(self.handle, len(groups), arr),
                   "drt3d_plan_set_adjoint_schedule")

    def adjoint_schedule(self) -> tuple:
        ng = ctypes.c_int()
        arr = (ctypes.c_int * 8)()
        _abi.check(self._lib.drt3d_plan_get_adjoint_schedule(self.handle, ctypes.byref(ng), arr),
                   "drt3d_plan_get_adjoint_schedule")
        return tuple(arr[i] for i in range(ng.value))

    def __del__(self):
        try:
            if getattr(self, "handle", None):
                self._lib.drt3d_plan_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


class _VolDesc(ctypes.Structure):
    _fields_ = [("d_in", ctypes.c_void_p), ("d_out", ctypes.c_void_p)]


class BatchPlan:
    """Planes forward of many uint8 volumes (N in 16..256) in one persistent launch.

    ``bind`` fixes the device buffers; ``run`` enqueues one memset and one
    kernel on the current stream (capturable in a CUDA graph), or with
    ``set_mode(1)`` the volumes' per-pass launches over internal streams.
    """

    def __init__(self, Ns, dtype: torch.dtype = torch.uint8, schedules: dict | None = None,
                 item_tiles: dict | None = None):
        if dtype != torch.uint8:
            raise TypeError("the batched forward takes uint8 volumes")
        self.Ns = [int(n) for n in Ns]
        self._lib = _abi.lib()
        h = ctypes.c_void_p()
        arr = (ctypes.c_int * len(self.Ns))(*self.Ns)
        _abi.check(self._lib.drt3d_batch_plan_create(ctypes.byref(h), len(self.Ns), arr, _abi.DTYPES["u8"], 0),
                   "drt3d_batch_plan_create")
        self.handle = h
        for N, groups in (schedules or {}).items():
            g = (ctypes.c_int * len(groups))(*[int(x) for x in groups])
            _abi.check(self._lib.drt3d_batch_set_schedule(self.handle, int(N), len(groups), g),
                       "drt3d_batch_set_schedule")
        for N, tiles in (item_tiles or {}).items():
            self.set_item_tiles(N, tiles)
        self._keep = None

    def set_item_tiles(self, N: int, tiles) -> None:
        """Unit-tiles per work item of each pass of the persistent launch for
        the volumes of size N (0 = default); see drt3d_batch_set_item_tiles.
        Rebind afterwards."""
        t = (ctypes.c_int * len(tiles))(*[int(x) for x in tiles])
        _abi.check(self._lib.drt3d_batch_set_item_tiles(self.handle, int(N), len(tiles), t),
                   "drt3d_batch_set_item_tiles")

    def workspace_bytes(self) -> int:
        v = ctypes.c_size_t()
        _abi.check(self._lib.drt3d_batch_workspace_bytes(self.handle, ctypes.byref(v)), "drt3d_batch_workspace_bytes")
        return int(v.value)

    def bind(self, vols, outs=None, workspace: torch.Tensor | None = None):
        """Bind device volumes (and outputs, allocated if omitted); returns outs."""
        if len(vols) != len(self.Ns):
            raise ValueError("one volume per size")
        if outs is None:
            outs = [torch.empty((12, N, N, 3 * N), dtype=torch.int32, device=v.device) for v, N in zip(vols, self.Ns)]
        for v, o, N in zip(vols, outs, self.Ns):
            if tuple(v.shape) != (N, N, N) or v.dtype != torch.uint8 or not v.is_cuda or not v.is_contiguous():
                raise ValueError("volumes must be contiguous cuda uint8 N^3 tensors matching the plan")
            if tuple(o.shape) != (12, N, N, 3 * N) or o.dtype != torch.int32 or not o.is_contiguous():
                raise ValueError("outputs must be contiguous (12, N, N, 3N) int32 tensors")
        nb = self.workspace_bytes()
        ws = workspace if workspace is not None else torch.empty(max(16, nb), dtype=torch.uint8, device=vols[0].device)
        descs = (_VolDesc * len(vols))(*[_VolDesc(v.data_ptr(), o.data_ptr()) for v, o in zip(vols, outs)])
        _abi.check(self._lib.drt3d_batch_bind(self.handle, descs, ws.data_ptr(), ws.numel()), "drt3d_batch_bind")
        self._keep = (list(vols), list(outs), ws)
        return outs

    def set_mode(self, mode: int, streams: int = 4) -> None:
        """0: one persistent kernel (default); 1: per-volume launches spread
        over ``streams`` internal streams (see drt3d_batch_set_mode)."""
        _abi.check(self._lib.drt3d_batch_set_mode(self.handle, int(mode), int(streams)), "drt3d_batch_set_mode")

    def run(self) -> None:
        _abi.check(self._lib.drt3d_planes_forward_batched(self.handle, _stream()), "drt3d_planes_forward_batched")

    def device_error(self) -> int:
        return int(self._lib.drt3d_batch_get_device_error(self.handle, _stream()))

    def set_wait_limit(self, ns: int, withhold_vol: int = -1, withhold_dodecant: int = -1) -> None:
        _abi.check(self._lib.drt3d_batch_set_wait_limit(self.handle, int(ns), int(withhold_vol),
                                                        int(withhold_dodecant)), "drt3d_batch_set_wait_limit")

    def __del__(self):
        try:
            if getattr(self, "handle", None):
                self._lib.drt3d_batch_plan_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


_plan_cache: dict = {}
_plan_lock = threading.Lock()  # host threads may ask for the same plan at once


def get_plan(N: int, dtype: torch.dtype) -> Plan:
    key = (torch.cuda.current_device(), int(N), dtype)
    with _plan_lock:
        p = _plan_cache.get(key)
        if p is None:
            p = Plan(N, dtype)
            _plan_cache[key] = p
    return p


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _vol_check(vol: torch.Tensor) -> int:
    if vol.dim() != 3 or not (vol.shape[0] == vol.shape[1] == vol.shape[2]):
        raise ValueError(f"expected an N x N x N volume, got {tuple(vol.shape)}")
    return int(vol.shape[0])


def _to_device(t: torch.Tensor):
    """(device tensor, came_from_host)."""
    if t.is_cuda:
        return t.contiguous(), False
    return t.contiguous().pin_memory().to("cuda", non_blocking=True), True


def planes_forward(vol: torch.Tensor, dodecants=ALL, out: torch.Tensor | None = None,
                   workspace: torch.Tensor | None = None) -> torch.Tensor:
    """Forward 3D DRT of planes over the selected dodecants (Algorithms 1-2)."""
    vol_d, host = _to_device(vol)
    N = _vol_check(vol_d)
    m = _mask(dodecants)
    plan = get_plan(N, vol_d.dtype)
    odt = torch.float32 if vol_d.dtype == torch.float32 else torch.int32
    if out is None:
        out = torch.empty((_count(m), N, N, 3 * N), dtype=odt, device=vol_d.device)
    ws = workspace if workspace is not None else plan.workspace("planes_forward")
    _abi.check(plan._lib.drt3d_planes_forward(plan.handle, vol_d.data_ptr(), out.data_ptr(), m,
                                              ws.data_ptr(), ws.numel(), _stream()),
               "drt3d_planes_forward")
    if host:
        return out.to("cpu")
    return out


def planes_forward_residual(vol: torch.Tensor, target: torch.Tensor, dodecants=ALL,
                            out: torch.Tensor | None = None, workspace: torch.Tensor | None = None) -> torch.Tensor:
    """A vol - target over the selected dodecants, the subtraction done as the
    transform's last pass stores each cell (``target`` in the output layout;
    ``out`` may be ``target`` itself)."""
    vol_d, host = _to_device(vol)
    N = _vol_check(vol_d)
    m = _mask(dodecants)
    plan = get_plan(N, vol_d.dtype)
    odt = torch.float32 if vol_d.dtype == torch.float32 else torch.int32
    shape = (_count(m), N, N, 3 * N)
    if tuple(target.shape) != shape or target.dtype != odt or not target.is_cuda or not target.is_contiguous():
        raise ValueError(f"target must be a contiguous cuda {odt} tensor of shape {shape}")
    if out is None:
        out = torch.empty(shape, dtype=odt, device=vol_d.device)
    ws = workspace if workspace is not None else plan.workspace("planes_forward")
    _abi.check(plan._lib.drt3d_planes_forward_residual(plan.handle, vol_d.data_ptr(), target.data_ptr(),
                                                       out.data_ptr(), m, ws.data_ptr(), ws.numel(), _stream()),
               "drt3d_planes_forward_residual")
    return out.to("cpu") if host else out


def planes_forward_residual_loss(vol: torch.Tensor, target: torch.Tensor, dodecants=ALL,
                                 out: torch.Tensor | None = None, loss: torch.Tensor | None = None,
                                 workspace: torch.Tensor | None = None):
    """(r, loss): r = A vol - target as ``planes_forward_residual`` (float32
    volumes) and loss = 0.5 ||r||^2, a float64 cuda scalar summed as the
    transform stores r (see drt3d_planes_forward_residual_loss)."""
    vol_d, host = _to_device(vol)
    N = _vol_check(vol_d)
    if vol_d.dtype != torch.float32:
        raise TypeError("the residual loss takes float32 volumes")
    m = _mask(dodecants)
    plan = get_plan(N, vol_d.dtype)
    shape = (_count(m), N, N, 3 * N)
    if (tuple(target.shape) != shape or target.dtype != torch.float32 or not target.is_cuda
            or not target.is_contiguous()):
        raise ValueError(f"target must be a contiguous cuda float32 tensor of shape {shape}")
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device=vol_d.device)
    if loss is None:
        loss = torch.empty((), dtype=torch.float64, device=vol_d.device)
    ws = workspace if workspace is not None else plan.workspace("planes_residual_loss")
    _abi.check(plan._lib.drt3d_planes_forward_residual_loss(plan.handle, vol_d.data_ptr(), target.data_ptr(),
                                                            out.data_ptr(), m, loss.data_ptr(), ws.data_ptr(),
                                                            ws.numel(), _stream()),
               "drt3d_planes_forward_residual_loss")
    return (out.to("cpu"), loss.to("cpu")) if host else (out, loss)


def planes_forward_global(vol: torch.Tensor, out: torch.Tensor | None = None,
                          workspace: torch.Tensor | None = None) -> torch.Tensor:
    """All 12 dodecants in Algorithm 2's global 4N x 4N x (3N-2) layout."""
    vol_d, host = _to_device(vol)
    N = _vol_check(vol_d)
    plan = get_plan(N, vol_d.dtype)
    if out is None:
        odt = torch.float32 if vol_d.dtype == torch.float32 else torch.int32
        out = torch.empty((4 * N, 4 * N, 3 * N - 2), dtype=odt, device=vol_d.device)
    ws = workspace if workspace is not None else plan.workspace("planes_forward")
    _abi.check(plan._lib.drt3d_planes_forward_global(plan.handle, vol_d.data_ptr(), out.data_ptr(),
                                                     ws.data_ptr(), ws.numel(), _stream()),
               "drt3d_planes_forward_global")
    return out.to("cpu") if host else out


def planes_adjoint(cot: torch.Tensor, dodecants=ALL, out: torch.Tensor | None = None,
                   workspace: torch.Tensor | None = None) -> torch.Tensor:
    """Backprojection (Section 5.1), summed over the selected dodecants."""
    cot_d, host = _to_device(cot)
    m = _mask(dodecants)
    if cot_d.dim() != 4 or cot_d.shape[0] != _count(m) or cot_d.shape[3] != 3 * cot_d.shape[1]:
        raise ValueError(f"cotangent shape {tuple(cot_d.shape)} does not match the mask")
    N = int(cot_d.shape[1])
    plan = get_plan(N, cot_d.dtype)
    if out is None:
        out = torch.empty((N, N, N), dtype=cot_d.dtype, device=cot_d.device)
    ws = workspace if workspace is not None else plan.workspace("planes_adjoint")
    _abi.check(plan._lib.drt3d_planes_adjoint(plan.handle, cot_d.data_ptr(), out.data_ptr(), m,
                                              ws.data_ptr(), ws.numel(), _stream()),
               "drt3d_planes_adjoint")
    return out.to("cpu") if host else out


class NotInRangeError(DRT3DError):
    """The array handed to ``planes_inverse`` is not a forward transform."""


def planes_inverse(R_k: torch.Tensor, dodecant: int, out: torch.Tensor | None = None,
                   workspace: torch.Tensor | None = None, check: bool = True) -> torch.Tensor:
    """Exact integer inverse of one dodecant's transform -> (N, N, N) int32.

    With ``check`` the call synchronises and raises ``NotInRangeError`` when
    ``R_k`` is not in the range of the forward map; without it the status
    stays in the plan's device word (``get_plan(N, torch.int32).device_error()``).
    """
    R_d, host = _to_device(R_k)
    if R_d.dtype != torch.int32 or R_d.dim() != 3 or R_d.shape[2] != 3 * R_d.shape[0]:
        raise ValueError(f"expected an (N, N, 3N) int32 block, got {tuple(R_d.shape)} {R_d.dtype}")
    N = int(R_d.shape[0])
    if not 0 <= int(dodecant) < 12:
        raise ValueError(f"dodecant index out of range: {dodecant}")
    plan = get_plan(N, torch.int32)
    if out is None:
        out = torch.empty((N, N, N), dtype=torch.int32, device=R_d.device)
    ws = workspace if workspace is not None else plan.workspace("planes_inverse")
    _abi.check(plan._lib.drt3d_planes_inverse(plan.handle, R_d.data_ptr(), int(dodecant), out.data_ptr(),
                                              ws.data_ptr(), ws.numel(), _stream()),
               "drt3d_planes_inverse")
    if check:
        code = plan.device_error()
        if code == 6:
            raise NotInRangeError(code, "drt3d_planes_inverse")
        _abi.check(code, "drt3d_planes_inverse (device)")
    return out.to("cpu") if host else out


def lines_forward(vol: torch.Tensor, sectors=ALL, out: torch.Tensor | None = None,
                  workspace: torch.Tensor | None = None) -> torch.Tensor:
    """Forward 3D DJT of lines over the selected sectors (Algorithm 3)."""
    vol_d, host = _to_device(vol)
    N = _vol_check(vol_d)
    if vol_d.dtype == torch.float32:
        raise TypeError("the lines transform takes integer volumes")
    m = _mask(sectors)
    plan = get_plan(N, vol_d.dtype)
    if out is None:
        out = torch.empty((_count(m), N, N, 2 * N, 2 * N), dtype=torch.int32, device=vol_d.device)
    ws = workspace if workspace is not None else plan.workspace("lines_forward")
    _abi.check(plan._lib.djt3d_lines_forward(plan.handle, vol_d.data_ptr(), out.data_ptr(), m,
                                             ws.data_ptr(), ws.numel(), _stream()),
               "djt3d_lines_forward")
    return out.to("cpu") if host else out


def lines_adjoint(cot: torch.Tensor, sectors=ALL, out: torch.Tensor | None = None,
                  workspace: torch.Tensor | None = None) -> torch.Tensor:
    """Backprojection of lines (eq.(invmap3DJsummation)) summed over the sectors,
    int32: ``cot`` is (len(sectors), N, N, 2N, 2N)."""
    cot_d, host = _to_device(cot)
    if cot_d.dtype != torch.int32:
        raise TypeError("the lines adjoint takes int32 cotangents")
    m = _mask(sectors)
    N = int(cot_d.shape[1])
    if cot_d.dim() != 5 or cot_d.shape[0] != _count(m) or tuple(cot_d.shape[2:]) != (N, 2 * N, 2 * N):
        raise ValueError(f"cotangent shape {tuple(cot_d.shape)} does not match {_count(m)} sectors")
    cot_d = cot_d.contiguous()
    plan = get_plan(N, torch.int32)
    if out is None:
        out = torch.empty((N, N, N), dtype=torch.int32, device=cot_d.device)
    ws = workspace if workspace is not None else plan.workspace("lines_adjoint")
    _abi.check(plan._lib.djt3d_lines_adjoint(plan.handle, cot_d.data_ptr(), out.data_ptr(), m,
                                             ws.data_ptr(), ws.numel(), _stream()),
               "djt3d_lines_adjoint")
    return out.to("cpu") if host else out


def _quad_mask(sel) -> int:
    if isinstance(sel, int):
        m = sel
    else:
        m = 0
        for q in sel:
            if not 0 <= int(q) < 4:
                raise ValueError(f"quadrant index out of range: {q}")
            m |= 1 << int(q)
    if m <= 0 or m > 0xF:
        raise ValueError(f"bad quadrant mask {m:#x}")
    return m


def drt2d_forward(imgs: torch.Tensor, quadrants=range(4), out: torch.Tensor | None = None,
                  workspace: torch.Tensor | None = None) -> torch.Tensor:
    """2D DRT of lines (eq.(map2D)) of a batch of N x N images (B, N, N) or
    one image (N, N), over the selected quadrants: (B, q, N, 2N)."""
    img_d, host = _to_device(imgs)
    single = img_d.dim() == 2
    if single:
        img_d = img_d.unsqueeze(0)
    if img_d.dim() != 3 or img_d.shape[1] != img_d.shape[2]:
        raise ValueError(f"expected (B, N, N) images, got {tuple(imgs.shape)}")
    B, N = int(img_d.shape[0]), int(img_d.shape[1])
    m = _quad_mask(quadrants)
    plan = get_plan(N, img_d.dtype)
    odt = torch.float32 if img_d.dtype == torch.float32 else torch.int32
    if out is None:
        out = torch.empty((B, _count(m), N, 2 * N), dtype=odt, device=img_d.device)
    if workspace is None:
        v = ctypes.c_size_t()
        _abi.check(plan._lib.drt2d_workspace_bytes(plan.handle, B, m, ctypes.byref(v)), "drt2d_workspace_bytes")
        workspace = torch.empty(max(16, int(v.value)), dtype=torch.uint8, device=img_d.device)
    _abi.check(plan._lib.drt2d_forward(plan.handle, img_d.data_ptr(), B, out.data_ptr(), m,
                                       workspace.data_ptr(), workspace.numel(), _stream()),
               "drt2d_forward")
    if single:
        out = out[0]
    return out.to("cpu") if host else out


_press_steps_cache: dict = {}


def press_step_sizes(N: int, factor: float = 1.5, iterations: int = 30, seed: int = 0) -> list:
    """Step sizes of the iterative inverse: [0, c_1, ..., c_n] with
    c_l = factor / (spectral radius of h * A^T A at size 2^l), each radius
    from ``iterations`` power-iteration steps on the GPU from a seeded
    normal start vector.  Cached per device and arguments."""
    dev = torch.cuda.current_device()
    key = (dev, int(N), float(factor), int(iterations), int(seed))
    if key in _press_steps_cache:
        return list(_press_steps_cache[key])
    plan = get_plan(N, torch.float32)
    ws = plan.workspace("planes_press")
    n = int(N).bit_length() - 1
    steps = [0.0]
    for level in range(1, n + 1):
        L = 1 << level
        g = torch.Generator(device=f"cuda:{dev}").manual_seed(seed + L)
        start = torch.randn((L, L, L), generator=g, device=f"cuda:{dev}", dtype=torch.float32)
        lam = ctypes.c_double()
        _abi.check(plan._lib.drt3d_press_spectral_radius(plan.handle, level, start.data_ptr(), iterations,
                                                          ctypes.byref(lam), ws.data_ptr(), ws.numel(), _stream()),
                   "drt3d_press_spectral_radius")
        steps.append(factor / lam.value)
    _press_steps_cache[key] = tuple(steps)
    return steps


def planes_press_inverse(R: torch.Tensor, iterations: int = 10, smooth: int = 2, steps=None,
                         out: torch.Tensor | None = None, workspace: torch.Tensor | None = None) -> torch.Tensor:
    """Iterative inverse of the twelve-dodecant planes transform (Section 5.2):
    ``R`` is (12, N, N, 3N) float32; returns the (N, N, N) float32 volume after
    ``iterations`` multigrid improvements with ``smooth`` smoothing steps per
    level.  ``steps`` defaults to ``press_step_sizes(N)``."""
    R_d, host = _to_device(R)
    if R_d.dtype != torch.float32 or R_d.dim() != 4 or R_d.shape[0] != 12:
        raise ValueError("expected a (12, N, N, 3N) float32 transform")
    N = int(R_d.shape[1])
    if tuple(R_d.shape) != (12, N, N, 3 * N):
        raise ValueError(f"expected (12, N, N, 3N), got {tuple(R_d.shape)}")
    plan = get_plan(N, torch.float32)
    if steps is None:
        steps = press_step_sizes(N)
    n = N.bit_length() - 1
    if len(steps) != n + 1:
        raise ValueError(f"need {n + 1} step sizes (entry 0 unused)")
    arr = (ctypes.c_float * (n + 1))(*[float(c) for c in steps])
    if out is None:
        out = torch.empty((N, N, N), dtype=torch.float32, device=R_d.device)
    ws = workspace if workspace is not None else plan.workspace("planes_press")
    _abi.check(plan._lib.drt3d_planes_press_inverse(plan.handle, R_d.data_ptr(), out.data_ptr(), int(iterations),
                                                    int(smooth), arr, ws.data_ptr(), ws.numel(), _stream()),
               "drt3d_planes_press_inverse")
    return out.to("cpu") if host else out


class PlanesTransform(torch.autograd.Function):
    """Differentiable 3D DRT of planes for float32 volumes.

    The operator is linear, so backward is the hand-written adjoint kernel
    applied to the cotangent; nothing from the forward is saved.
    """

    @staticmethod
    def forward(ctx, vol: torch.Tensor, dodecants: int = ALL):
        if vol.dtype != torch.float32:
            raise TypeError("PlanesTransform needs float32 volumes")
        ctx.mask = _mask(dodecants)
        return planes_forward(vol, ctx.mask)

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        return planes_adjoint(grad_out.contiguous(), ctx.mask), None


class PlanesTransformBatch(torch.autograd.Function):
    """``PlanesTransform`` over a leading batch dimension.

    Each volume's transform is written straight into its slice of one
    (B, k, N, N, 3N) output, and backward backprojects each cotangent slice
    into its slice of one (B, N, N, N) gradient: no stacking or splitting
    copies of the multi-GB transforms.
    """

    @staticmethod
    def forward(ctx, vols: torch.Tensor, dodecants: int = ALL):
        if vols.dtype != torch.float32:
            raise TypeError("PlanesTransformBatch needs float32 volumes")
        if vols.dim() != 4:
            raise ValueError(f"expected (B, N, N, N) volumes, got {tuple(vols.shape)}")
        vols = vols.contiguous()
        B, N = int(vols.shape[0]), int(vols.shape[1])
        m = _mask(dodecants)
        ctx.mask = m
        out = torch.empty((B, _count(m), N, N, 3 * N), dtype=torch.float32, device=vols.device)
        ws = get_plan(N, torch.float32).workspace("planes_forward")
        for b in range(B):
            planes_forward(vols[b], m, out=out[b], workspace=ws)
        return out

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        g = grad_out.contiguous()
        B, N = int(g.shape[0]), int(g.shape[2])
        grad = torch.empty((B, N, N, N), dtype=torch.float32, device=g.device)
        ws = get_plan(N, torch.float32).workspace("planes_adjoint")
        for b in range(B):
            planes_adjoint(g[b], ctx.mask, out=grad[b], workspace=ws)
        return grad, None


def planes(vol: torch.Tensor, dodecants=ALL) -> torch.Tensor:
    """Autograd-aware forward for float32 volumes (batched over a leading dim)."""
    m = _mask(dodecants)
    if vol.dim() == 4:
        return PlanesTransformBatch.apply(vol, m)
    return PlanesTransform.apply(vol, m)
