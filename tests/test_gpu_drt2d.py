"""GPU parity of the 2D DRT of lines (eq.(map2D), four quadrants) against the
oracle: bit-exact int32 (wrapping) for integer images; for float32 images
within the rounding bound of an n-level summation tree (below)."""
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


def _imgs(N, B, dt, seed):
    if dt == "u8":
        return synth.random_int32((B, N, N), seed, 0, 256).astype(np.uint8)
    if dt == "i16":
        return synth.random_int32((B, N, N), seed, -32768, 32768).astype(np.int16)
    if dt == "i32":
        return synth.random_int32((B, N, N), seed)  # full range: sums wrap
    return synth.random_float((B, N, N), seed)


def _run(drt, f, quadrants=range(4), workspace=None):
    t = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    return drt.drt2d_forward(t, quadrants, workspace=workspace).cpu().numpy()


@pytest.mark.parametrize("N", [2, 4, 8, 16, 32, 64])
@pytest.mark.parametrize("dt", ["u8", "i16", "i32"])
def test_integer_exact(drt, oracle_mod, N, dt):
    f = _imgs(N, 3, dt, 500 + N)
    np.testing.assert_array_equal(_run(drt, f), oracle_mod.drt2d_forward(f))


@pytest.mark.parametrize("N", [32, 64, 128, 256])
def test_uint8_single_cta_path(drt, oracle_mod, N):
    """uint8 images with 32 <= N <= 256 run one CTA per (image, quadrant)
    with 16-bit intermediates: full-range bytes (the largest sums) against
    the oracle, and against the same images widened to int16 (multi-pass)."""
    f = _imgs(N, 3, "u8", 800 + N)
    f[0] = 255
    got = _run(drt, f)
    np.testing.assert_array_equal(got, oracle_mod.drt2d_forward(f))
    np.testing.assert_array_equal(got, _run(drt, f.astype(np.int16)))
    for qs in ([3], [1, 2]):
        np.testing.assert_array_equal(_run(drt, f, qs), got[:, qs])


@pytest.mark.parametrize("N", [4, 32, 128])
def test_float_within_tree_rounding(drt, oracle_mod, N):
    """Each output is an n-level binary sum tree of N float32 terms, so its
    error is below (n + 1) * 2^-24 times the sum of the terms' magnitudes,
    which is the transform of |f| (computed in float64 by the oracle)."""
    n = N.bit_length() - 1
    f = _imgs(N, 2, "f32", 600 + N)
    got = _run(drt, f)
    want = oracle_mod.drt2d_forward(f.astype(np.float64))
    bound = (n + 1) * 2.0 ** -24 * oracle_mod.drt2d_forward(np.abs(f).astype(np.float64))
    assert (np.abs(got - want) <= bound + 1e-30).all()


def test_quadrant_subsets(drt, oracle_mod):
    N = 32
    f = _imgs(N, 2, "i16", 7)
    for qs in ([0], [3], [1, 2], [0, 2, 3]):
        np.testing.assert_array_equal(_run(drt, f, qs), oracle_mod.drt2d_forward(f, qs))


@pytest.mark.parametrize("N", [32, 256])
def test_chunked_batch(drt, oracle_mod, N):
    """A workspace that holds fewer images than the batch (a ragged last
    chunk) gives the same result as the default one (int16 images: the
    multi-pass path)."""
    B = 7
    f = synth.images_2d(N, B, seed=11).astype(np.int16)
    plan = drt.get_plan(N, torch.int16)
    per = ctypes.c_size_t()
    plan._lib.drt2d_workspace_bytes(plan.handle, 1, 0xF, ctypes.byref(per))
    assert per.value > 0
    ws = torch.empty(3 * per.value + 16, dtype=torch.uint8, device="cuda")  # 3 images per chunk
    got = _run(drt, f, workspace=ws)
    np.testing.assert_array_equal(got, oracle_mod.drt2d_forward(f))
    np.testing.assert_array_equal(got, _run(drt, f))


def test_single_image_and_empty_batch(drt, oracle_mod):
    N = 16
    f = _imgs(N, 1, "u8", 12)[0]
    got = drt.drt2d_forward(torch.from_numpy(f).cuda(), [0, 1]).cpu().numpy()
    np.testing.assert_array_equal(got, oracle_mod.drt2d_forward(f[None], [0, 1])[0])
    empty = torch.empty((0, N, N), dtype=torch.uint8, device="cuda")
    assert drt.drt2d_forward(empty).shape == (0, 4, N, 2 * N)


def test_n1024_exact(drt, oracle_mod):
    """Largest N (three passes, two ping-pong buffers)."""
    N = 1024
    f = _imgs(N, 1, "i32", 13)
    got = _run(drt, f, [1, 2])
    np.testing.assert_array_equal(got, oracle_mod.drt2d_forward(f, [1, 2]))


def test_full_batch_samples(drt, oracle_mod):
    """The benchmark's batch (512 images of 256^2 uint8, four quadrants):
    every output checked against the oracle for a sample of images, and the
    per-slope mass invariant for all of them."""
    f = synth.images_2d(256, 512, seed=6)
    t = torch.from_numpy(f).cuda()
    out = drt.drt2d_forward(t)
    for b in (0, 1, 255, 511):
        np.testing.assert_array_equal(out[b].cpu().numpy(), oracle_mod.drt2d_forward(f[b:b + 1])[0])
    mass = t.to(torch.int64).sum(dim=(1, 2))
    per_slope = out.to(torch.int64).sum(dim=3)  # (B, 4, N)
    assert torch.equal(per_slope, mass[:, None, None].expand_as(per_slope))
    assert not out[:, :, :, 0].any()


def test_errors(drt):
    import paper_2501_13664_gb300._abi as abi

    N = 16
    plan = drt.get_plan(N, torch.uint8)
    img = torch.zeros((2, N, N), dtype=torch.uint8, device="cuda")
    out = torch.zeros((2, 4, N, 2 * N), dtype=torch.int32, device="cuda")
    lib = plan._lib
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.drt2d_forward(plan.handle, img.data_ptr(), 2, out.data_ptr(), 0, None, 0, s) == 1
    assert lib.drt2d_forward(plan.handle, img.data_ptr(), 2, out.data_ptr(), 0x10, None, 0, s) == 1
    assert lib.drt2d_forward(plan.handle, img.data_ptr() + 4, 2, out.data_ptr(), 0xF, None, 0, s) == 4
    assert lib.drt2d_forward(plan.handle, img.data_ptr(), -1, out.data_ptr(), 0xF, None, 0, s) == 1
    # int16 images of N = 64 go through the multi-pass path, which needs a workspace
    big = drt.get_plan(64, torch.int16)
    img64 = torch.zeros((1, 64, 64), dtype=torch.int16, device="cuda")
    out64 = torch.zeros((1, 4, 64, 128), dtype=torch.int32, device="cuda")
    assert lib.drt2d_forward(big.handle, img64.data_ptr(), 1, out64.data_ptr(), 0xF, None, 0, s) == 5
    # uint8 images up to N = 256 need none (one CTA per image and quadrant)
    u8 = drt.get_plan(64, torch.uint8)
    assert lib.drt2d_forward(u8.handle, img64.data_ptr(), 1, out64.data_ptr(), 0xF, None, 0, s) == 0
    with pytest.raises(ValueError):
        drt.drt2d_forward(img, [4])
    assert abi.DRT3DError is not None
