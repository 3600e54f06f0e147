"""GPU parity of Section 5.2's iterative inverse (adjoint + filter h,
multigrid with P and S) against the oracle.

The GPU computes in float32 and the oracle in float64; both run the same
steps with the same step sizes (the oracle's).  Each sweep is a contraction
applied to the data, so the float32 rounding of one sweep (sums of at most
12 N^2 terms, relative error a few 1e-7 per term after normalisation) does
not grow from sweep to sweep; the tests allow 1e-4 of the volume's range,
a wide margin over that and far below the error of the iterates
themselves."""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def drt():
    import paper_2501_13664_gb300 as drt3d

    return drt3d


@pytest.fixture(scope="module")
def press(oracle_mod):
    from oracle import press

    return press


def _starts(N):
    return {L: synth.random_float((L,) * 3, 100 + L).astype(np.float64) for L in (2 ** i for i in range(1, N.bit_length()))}


def _steps_list(steps, N):
    return [0.0] + [steps[2 ** l] for l in range(1, N.bit_length())]


def _corners_centre(N):
    f = np.zeros((N, N, N))
    for x in (0, N - 1):
        for y in (0, N - 1):
            for z in (0, N - 1):
                f[x, y, z] = 1.0
    f[N // 2, N // 2, N // 2] = 1.0
    return f


def test_spectral_radius_matches_oracle(drt, press):
    N = 8
    plan = drt.get_plan(N, torch.float32)
    ws = plan.workspace("planes_press")
    for level in (1, 2, 3):
        L = 1 << level
        start = synth.random_float((L, L, L), 40 + L)
        lam = ctypes.c_double()
        st = plan._lib.drt3d_press_spectral_radius(plan.handle, level, torch.from_numpy(start).cuda().data_ptr(), 30,
                                                   ctypes.byref(lam), ws.data_ptr(), ws.numel(),
                                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == 0
        want = press.spectral_radius(L, start.astype(np.float64), 30)
        assert abs(lam.value - want) <= 1e-4 * want


@pytest.mark.parametrize("N,iters,smooth", [(2, 1, 1), (4, 1, 2), (8, 2, 2), (16, 1, 2), (32, 2, 2)])
def test_iterates_match_oracle(drt, press, N, iters, smooth):
    f = synth.random_float((N, N, N), 50 + N).astype(np.float64)
    R = press.A(f)
    steps = press.step_sizes(N, _starts(N))
    want = press.press_inverse(R, iters, steps, smooth)
    got = drt.planes_press_inverse(torch.from_numpy(R.astype(np.float32)).cuda(), iters, smooth,
                                   _steps_list(steps, N)).cpu().numpy()
    tol = 1e-4 * (want.max() - want.min())
    assert np.abs(got - want).max() <= tol


def test_n64_corners_and_centre(drt, press, oracle_mod):
    """The paper's example at the size it quotes (N = 64): the GPU iterates
    follow the oracle's for two iterations, and the error keeps falling to
    ten iterations."""
    N = 64
    f = _corners_centre(N)
    R = press.A(f)
    steps = press.step_sizes(N, _starts(N), iterations=10)
    sl = _steps_list(steps, N)
    Rd = torch.from_numpy(R.astype(np.float32)).cuda()
    want = press.press_inverse(R, 2, steps)
    got2 = drt.planes_press_inverse(Rd, 2, 2, sl).cpu().numpy()
    assert np.abs(got2 - want).max() <= 1e-4
    errs = [press.nrmsd(drt.planes_press_inverse(Rd, k, 2, sl).cpu().numpy(), f) for k in (1, 2, 5, 10)]
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 2e-3


def test_zero_iterations_and_errors(drt):
    N = 8
    R = torch.zeros((12, N, N, 3 * N), dtype=torch.float32, device="cuda")
    out = torch.full((N, N, N), 7.0, device="cuda")
    steps = [0.0] + [1e-3] * 3
    drt.planes_press_inverse(R, 0, 2, steps, out=out)
    assert not out.any()
    plan = drt.get_plan(N, torch.float32)
    lib = plan._lib
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ws = plan.workspace("planes_press")
    arr = (ctypes.c_float * 4)(0.0, 1e-3, 1e-3, 1e-3)
    bad = (ctypes.c_float * 4)(0.0, 1e-3, 0.0, 1e-3)
    assert lib.drt3d_planes_press_inverse(plan.handle, R.data_ptr(), out.data_ptr(), 1, 2, bad, ws.data_ptr(),
                                          ws.numel(), s) == 1
    assert lib.drt3d_planes_press_inverse(plan.handle, R.data_ptr(), out.data_ptr(), 1, 0, arr, ws.data_ptr(),
                                          ws.numel(), s) == 1
    assert lib.drt3d_planes_press_inverse(plan.handle, R.data_ptr(), out.data_ptr(), 1, 2, arr, ws.data_ptr(),
                                          16, s) == 5
    iplan = drt.get_plan(N, torch.int32)
    assert lib.drt3d_planes_press_inverse(iplan.handle, R.data_ptr(), out.data_ptr(), 1, 2, arr, ws.data_ptr(),
                                          ws.numel(), s) == 3


def test_default_step_sizes_converge(drt, press):
    """press_step_sizes (GPU power iteration from its own seeded start) gives
    steps within 5 % of the oracle's (30 power steps from different starts
    approach the spectral radius from below at slightly different rates), and
    the default call recovers a smooth volume."""
    N = 16
    got = drt.press_step_sizes(N)
    want = press.step_sizes(N, _starts(N))
    for l in range(1, 5):
        assert abs(got[l] - want[2 ** l]) <= 0.05 * want[2 ** l]
    x = np.arange(N) / N
    f = np.sin(3 * x)[:, None, None] * np.cos(2 * x)[None, :, None] + x[None, None, :]
    R = torch.from_numpy(press.A(f).astype(np.float32)).cuda()
    rec = drt.planes_press_inverse(R, 10).cpu().numpy()
    assert press.nrmsd(rec, f) < 1e-3
