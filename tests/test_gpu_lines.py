"""GPU parity of the 3D DJT of lines (Algorithm 3, twelve sectors) against the
oracle: bit-exact int32 (wrapping)."""
import numpy as np
import pytest
import torch

import synth

from _paper_refs import lline_rec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def drt():
    import paper_2501_13664_gb300 as drt3d

    return drt3d


def _fwd(drt, f, sectors=0xFFF):
    return drt.lines_forward(torch.from_numpy(np.ascontiguousarray(f)).cuda(), sectors).cpu().numpy()


@pytest.mark.parametrize("N", [2, 4, 8, 16, 32])
@pytest.mark.parametrize("dt", ["u8", "i16", "i32"])
def test_lines_integer_exact(drt, oracle_mod, N, dt):
    if dt == "u8":
        f = synth.random_int32((N, N, N), 200 + N, 0, 256).astype(np.uint8)
    elif dt == "i16":
        f = synth.random_int32((N, N, N), 300 + N, -32768, 32768).astype(np.int16)
    else:
        f = synth.random_int32((N, N, N), 400 + N)  # full range: sums wrap
    np.testing.assert_array_equal(_fwd(drt, f), oracle_mod.lines_forward(f))


@pytest.mark.parametrize("dt", ["u8", "i32"])
def test_lines_n64_frame_copies(drt, oracle_mod, dt):
    """N = 64: the y- and z-driven sectors read transposed copies of the
    volume (the 64 x 64-tile byte transpose for uint8, the element transpose
    otherwise); bit-exact against the oracle."""
    N = 64
    if dt == "u8":
        f = synth.random_int32((N, N, N), 90, 0, 256).astype(np.uint8)
    else:
        f = synth.random_int32((N, N, N), 91)
    ks = [5, 10]
    np.testing.assert_array_equal(_fwd(drt, f, ks), oracle_mod.lines_forward(f, ks))


def test_lines_sector_subsets(drt, oracle_mod):
    N = 16
    f = synth.c3_volume(N, seed=7)
    for mask in (0x001, 0x820, 0x555):
        ks = [k for k in range(12) if (mask >> k) & 1]
        np.testing.assert_array_equal(_fwd(drt, f, mask), oracle_mod.lines_forward(f, ks))


def test_lines_n64_selected_sectors(drt, oracle_mod):
    N = 64
    f = synth.c3_volume(N, seed=8)
    ks = [0, 5, 10]
    np.testing.assert_array_equal(_fwd(drt, f, ks), oracle_mod.lines_forward(f, ks))


def test_config_c3_full_size(drt, oracle_mod):
    """N = 128 int16 volume with 32 embedded lines, all 12 sectors (51.5 GB of
    output): mass per slope pair, empty displacement row/column 0, and 10^5
    random cells against the eq.(3DfDJT) definition; an x-, a y- and a
    z-driven sector (0, 6, 11) in full against Algorithm 3."""
    N = 128
    f = synth.c3_volume(N)
    J = drt.lines_forward(torch.from_numpy(f).cuda())
    total = int(f.astype(np.int64).sum())
    for k in range(12):
        mass = J[k].to(torch.int64).sum(dim=(2, 3))
        assert bool((mass == total).all()), f"sector {k}"
        assert bool((J[k][:, :, 0, :] == 0).all()) and bool((J[k][:, :, :, 0] == 0).all())
    rng = np.random.default_rng(321)
    per = 100_000 // 12 + 1
    for k in range(12):
        g = oracle_mod.sector_volume(f.astype(np.int32), k)
        idx = np.stack([rng.integers(0, N, per), rng.integers(0, N, per),
                        rng.integers(0, 2 * N, per), rng.integers(0, 2 * N, per)], axis=1)
        it = torch.from_numpy(idx).cuda()
        got = J[k][it[:, 0], it[:, 1], it[:, 2], it[:, 3]].cpu().numpy()
        for (a, b, c, d), v in zip(idx, got):
            assert oracle_mod.lines_cell(g, int(a), int(b), int(c), int(d)) == int(v)
    for k in (0, 6, 11):
        np.testing.assert_array_equal(J[k].cpu().numpy(), oracle_mod.lines_forward(f, [k])[0], err_msg=f"sector {k}")


# ---------------------------------------------------------------------------
# Adjoint (backprojection), eq.(invmap3DJsummation): bit-exact int32 against
# the oracle's reversed Algorithm 3, and the dot-product identity at scale.
# ---------------------------------------------------------------------------
def _adj(drt, r, sectors=0xFFF):
    return drt.lines_adjoint(torch.from_numpy(np.ascontiguousarray(r)).cuda(), sectors).cpu().numpy()


@pytest.mark.parametrize("N", [2, 4, 8, 16, 32])
def test_lines_adjoint_exact(drt, oracle_mod, N):
    r = synth.random_int32((12, N, N, 2 * N, 2 * N), 700 + N)  # sums wrap
    np.testing.assert_array_equal(_adj(drt, r), oracle_mod.lines_adjoint(r))


def test_lines_adjoint_sector_subsets(drt, oracle_mod):
    N = 16
    for sel in ([0], [11], [1, 6], [2, 5, 9, 10]):
        r = synth.random_int32((len(sel), N, N, 2 * N, 2 * N), 710 + sel[0], -1000, 1000)
        np.testing.assert_array_equal(_adj(drt, r, sel), oracle_mod.lines_adjoint(r, sel))


def test_lines_adjoint_n64_selected_sectors(drt, oracle_mod):
    N = 64
    sel = [3, 8]
    r = synth.random_int32((2, N, N, 2 * N, 2 * N), 720)
    np.testing.assert_array_equal(_adj(drt, r, sel), oracle_mod.lines_adjoint(r, sel))


@pytest.mark.parametrize("k", [2, 5, 9])  # x-, y- and z-driven
def test_lines_adjoint_n128_full_sector(drt, oracle_mod, k):
    """Config-3 size (N = 128): one sector's backprojection of a full-range
    random int32 cotangent (4.3 GB, sums wrap), element by element against
    the oracle's reversed Algorithm 3."""
    N = 128
    r = synth.raw_int32((1, N, N, 2 * N, 2 * N), 740 + k)
    got = drt.lines_adjoint(torch.from_numpy(r).cuda(), [k]).cpu().numpy()
    torch.cuda.empty_cache()
    np.testing.assert_array_equal(got, oracle_mod.lines_adjoint(r, [k]))


def test_lines_adjoint_dot_product_n128(drt):
    """<J f, r> == <f, J^T r> exactly (int64 sums of int32 products with no
    wrap), GPU forward and GPU adjoint, config-3 volume, one sector."""
    N = 128
    sel = [5]
    f = torch.from_numpy(synth.c3_volume(N).astype(np.int32)).cuda()
    g = torch.Generator(device="cuda").manual_seed(730)
    r = torch.randint(-8, 8, (1, N, N, 2 * N, 2 * N), generator=g, device="cuda", dtype=torch.int32)
    J = drt.lines_forward(f, sel)
    lhs = sum(int((J[0, s].to(torch.int64) * r[0, s].to(torch.int64)).sum()) for s in range(N))
    del J
    fb = drt.lines_adjoint(r, sel)
    rhs = int((f.to(torch.int64) * fb.to(torch.int64)).sum())
    assert lhs == rhs


def test_lines_adjoint_errors(drt):
    N = 8
    with pytest.raises(TypeError):
        drt.lines_adjoint(torch.zeros((12, N, N, 2 * N, 2 * N), dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        drt.lines_adjoint(torch.zeros((11, N, N, 2 * N, 2 * N), dtype=torch.int32, device="cuda"))


def test_ray_in_noise_threshold_and_backproject(drt):
    """Section 4.1's example: a ray under white noise of twice its amplitude is
    the largest coefficient of its sector's DJT; backprojecting only that
    coefficient gives back exactly the ray's voxels, and with the 16 largest
    (the ray's neighbours share voxels with it) most of them."""
    from paper_2501_13664_gb300 import demos

    N, n = 128, 7
    line = (37, 90, 150, 140)
    s1, s2, d1, d2 = line
    # the digital line of eq.(3DfDJT) in sector 0's frame (x' = x, no flips),
    # drawn with the recursive form of eq.(digitalLine)
    mask = torch.zeros((N, N, N), dtype=torch.bool)
    for x in range(N):
        y, z = lline_rec(n, s1, x) + d1 - N, lline_rec(n, s2, x) + d2 - N
        if 0 <= y < N and 0 <= z < N:
            mask[x, y, z] = True
    mask = mask.cuda()
    res = demos.ray_in_noise(mask, line, amplitude=16, noise=32, top=1)
    assert res["line_voxels"] == 128  # the line crosses the whole cube
    assert res["peak"] == line
    assert demos.recovered_fraction(res) == 1.0
    res = demos.ray_in_noise(mask, line, amplitude=16, noise=32, top=16)
    assert res["peak"] == line
    assert res["line_coefficient"] > res["largest_other"]
    assert demos.recovered_fraction(res) >= 0.8
