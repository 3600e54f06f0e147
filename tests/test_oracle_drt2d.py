"""Pins for the oracle's 2D DRT of lines (Section 2.1) and its quadrants.

The oracle's two routes -- the definition (stage n of eq.(our2Dfm)) as a
scatter and the stage recursion eq.(map2D) -- are checked against each other,
against the test suite's own restatement of eq.(map2D) (another row layout and
embedding), against the 3D planes transform that a single-slice volume
reduces to, and against closed forms and invariants.
"""
import numpy as np
import pytest

import synth
from _paper_refs import drt2d_def, drt2d_map, lline_rec


def _img(N, seed, lo=-1000, hi=1000):
    return synth.random_int32((N, N), seed, lo, hi)


@pytest.mark.parametrize("N", [2, 4, 8, 16, 64])
def test_map2d_equals_definition(oracle_mod, N):
    f = _img(N, 20 + N)
    np.testing.assert_array_equal(oracle_mod.drt2d_map2d(f).astype(np.int64), oracle_mod.drt2d_brute(f))


@pytest.mark.parametrize("N", [4, 8])
def test_map2d_wraps_like_int32(oracle_mod, N):
    f = synth.random_int32((N, N), 31)  # full range: sums wrap
    want = (oracle_mod.drt2d_brute(f) % (1 << 32)).astype(np.uint32).view(np.int32)
    np.testing.assert_array_equal(oracle_mod.drt2d_map2d(f), want)


@pytest.mark.parametrize("N", [4, 16])
def test_float_route(oracle_mod, N):
    f = synth.random_float((N, N), 5).astype(np.float64)
    np.testing.assert_allclose(oracle_mod.drt2d_map2d(f), oracle_mod.drt2d_brute(f), rtol=0, atol=1e-12)


@pytest.mark.parametrize("N", [4, 8, 16])
def test_matches_independent_restatement(oracle_mod, N):
    """The suite's eq.(map2D) restatement embeds the image at [2N, 3N) and
    keeps rows slope-minor; the oracle embeds at [N, 2N), slope-major."""
    f = _img(N, 40 + N, 0, 256)
    D = drt2d_map(f.astype(np.int64))
    assert not D[:, :N].any()
    np.testing.assert_array_equal(oracle_mod.drt2d_map2d(f).astype(np.int64), D[:, N:])
    if N <= 8:
        np.testing.assert_array_equal(drt2d_def(f.astype(np.int64))[:, N:], oracle_mod.drt2d_brute(f))


@pytest.mark.parametrize("N", [4, 8])
def test_single_slice_of_planes_transform(oracle_mod, N):
    """A volume non-zero only at y = 0 has planes R(s1, s2, d) equal to the
    2D DRT of that slice for every s2 (l_{s2}(0) = 0), one embedding apart."""
    h = _img(N, 50 + N, -50, 50)
    g = np.zeros((N, N, N), dtype=np.int64)
    g[:, 0, :] = h
    R3 = oracle_mod.planes_brute(g)
    R2 = oracle_mod.drt2d_brute(h)
    for s2 in range(N):
        assert not R3[:, s2, :N].any()
        np.testing.assert_array_equal(R3[:, s2, N:], R2)


@pytest.mark.parametrize("N", [2, 8, 32])
def test_closed_forms(oracle_mod, N):
    f = _img(N, 60 + N).astype(np.int64)
    R = oracle_mod.drt2d_map2d(f).astype(np.int64)
    # slope 0: horizontal lines are the column sums, below d = N nothing
    np.testing.assert_array_equal(R[0, N:], f.sum(0))
    assert not R[0, :N].any()
    # slope N - 1: l(u) = u, the diagonals y = u + d - N
    for d in range(2 * N):
        assert R[N - 1, d] == np.trace(f, offset=d - N)
    # d = 0 is never reached, and every slope sees the whole image once
    assert not R[:, 0].any()
    np.testing.assert_array_equal(R.sum(1), np.full(N, f.sum()))


@pytest.mark.parametrize("N", [4, 16])
def test_single_pixel_lights_one_cell_per_slope(oracle_mod, N):
    n = N.bit_length() - 1
    for (u, y) in [(0, 0), (N - 1, N - 1), (N // 2 + 1, 1)]:
        f = np.zeros((N, N), dtype=np.int32)
        f[u, y] = 1
        R = oracle_mod.drt2d_map2d(f)
        assert R.sum() == N and (R.sum(1) == 1).all()
        for s in range(N):
            assert R[s, y - lline_rec(n, s, u) + N] == 1


@pytest.mark.parametrize("q", range(4))
def test_quadrant_sees_its_own_lines(oracle_mod, q):
    """A digital line drawn in quadrant q's orientation adds up to N in that
    quadrant's transform: axes swapped by bit 1 of q, the other axis reversed
    by bit 0."""
    N, n = 16, 4
    s, d = 11, N + 2
    f = np.zeros((N, N), dtype=np.int32)
    for u in range(N):
        y = lline_rec(n, s, u) + d - N
        if 0 <= y < N:
            yy = N - 1 - y if q & 1 else y
            if q & 2:
                f[yy, u] = 1
            else:
                f[u, yy] = 1
    out = oracle_mod.drt2d_forward(f[None], range(4))[0]
    assert f.sum() == N and out[q, s, d] == N and out[q].max() == N
    # the same (s, d) in the other three quadrants is another line
    assert all(out[p, s, d] <= N // 4 for p in range(4) if p != q)


def test_quadrants_are_flips_and_transposes(oracle_mod):
    N = 8
    f = _img(N, 70)
    out = oracle_mod.drt2d_forward(np.stack([f, f[:, ::-1], f.T]), range(4))
    np.testing.assert_array_equal(out[1, 0], out[0, 1])  # flipped image, basic quadrant
    np.testing.assert_array_equal(out[2, 0], out[0, 2])  # transposed image
    np.testing.assert_array_equal(out[2, 1], out[0, 3])
    assert out.shape == (3, 4, N, 2 * N)


def test_pins_catch_a_wrong_shift(oracle_mod):
    """A stage that shifts by floor(S/2) instead of floor((S+1)/2) (slope bit
    dropped) fails the definition pin."""
    N = 8
    n = 3
    f = _img(N, 80, 0, 100).astype(np.int64)
    W = 2 * N
    fm = np.zeros((N, W), dtype=np.int64)
    fm[:, N:] = f
    for m in range(n):
        Vn = 1 << (n - m - 1)
        fn = np.zeros_like(fm)
        for S in range(2 << m):
            for V in range(Vn):
                sig, sh = S >> 1, S >> 1  # planted mistake
                lo, hi = fm[sig * 2 * Vn + 2 * V], fm[sig * 2 * Vn + 2 * V + 1]
                row = lo.copy()
                row[: W - sh] += hi[sh:]
                fn[S * Vn + V] = row
        fm = fn
    assert not np.array_equal(fm, oracle_mod.drt2d_brute(f))
