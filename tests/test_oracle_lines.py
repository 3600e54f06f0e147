"""Pins for the oracle's 3D DJT of lines (Section 4)."""
import numpy as np
import pytest

import synth
from _paper_refs import lline_rec
from test_oracle_planes import _frame_matrix


@pytest.mark.parametrize("N", [2, 4, 8, 16])
def test_alg3_equals_definition(oracle_mod, N):
    g = synth.random_int32((N, N, N), 50 + N, -1000, 1000)
    np.testing.assert_array_equal(oracle_mod.lines_alg3(g).astype(np.int64), oracle_mod.lines_brute(g))


def test_alg3_wraps_like_int32(oracle_mod):
    N = 8
    g = synth.random_int32((N, N, N), 51)
    want = (oracle_mod.lines_brute(g) % (1 << 32)).astype(np.uint32).view(np.int32)
    np.testing.assert_array_equal(oracle_mod.lines_alg3(g), want)


@pytest.mark.parametrize("N", [4, 8, 16])
def test_closed_forms(oracle_mod, N):
    g = synth.random_int32((N, N, N), 52, 0, 1024).astype(np.int64)
    J = oracle_mod.lines_alg3(g.astype(np.int32)).astype(np.int64)
    # slopes (0, 0): lines along x, J = x-column sums at (N + y, N + z)
    np.testing.assert_array_equal(J[0, 0, N:, N:], g.sum(axis=0))
    np.testing.assert_array_equal(J[0, 0, :N, :], 0)
    # slopes (N-1, N-1): the diagonal y = x + d1 - N, z = x + d2 - N
    want = np.zeros((2 * N, 2 * N), dtype=np.int64)
    x, y, z = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    np.add.at(want, ((y - x + N).ravel(), (z - x + N).ravel()), g.ravel())
    np.testing.assert_array_equal(J[N - 1, N - 1], want)
    # displacement index 0 is never reached; mass is conserved per slope pair
    np.testing.assert_array_equal(J[:, :, 0, :], 0)
    np.testing.assert_array_equal(J[:, :, :, 0], 0)
    np.testing.assert_array_equal(J.sum(axis=(2, 3)), np.full((N, N), g.sum()))


@pytest.mark.parametrize("N", [4, 8])
def test_single_voxel_lights_one_cell_per_slope(oracle_mod, N):
    n = N.bit_length() - 1
    rng = np.random.default_rng(N)
    for _ in range(4):
        x, y, z = (int(v) for v in rng.integers(0, N, size=3))
        g = np.zeros((N, N, N), dtype=np.int32)
        g[x, y, z] = 1
        J = oracle_mod.lines_alg3(g)
        assert (J != 0).sum() == N * N
        for s1 in range(N):
            for s2 in range(N):
                assert J[s1, s2, y - lline_rec(n, s1, x) + N, z - lline_rec(n, s2, x) + N] == 1


def test_cell_gather_matches_scatter(oracle_mod):
    N = 16
    g = synth.random_int32((N, N, N), 53, -100, 100)
    J = oracle_mod.lines_alg3(g)
    rng = np.random.default_rng(2)
    for _ in range(100):
        s1, s2 = (int(v) for v in rng.integers(0, N, size=2))
        d1, d2 = (int(v) for v in rng.integers(0, 2 * N, size=2))
        assert oracle_mod.lines_cell(g, s1, s2, d1, d2) == int(J[s1, s2, d1, d2])


def test_twelve_sectors_cover_all_line_directions(oracle_mod):
    """Each line direction (up to sign) falls in exactly one sector.

    In sector k's frame the lines are x' = u, y' = a u + d1, z' = b u + d2
    with a, b in [0, 1] (Section 4), direction (1, a, b)."""
    N = 16
    Ps = [_frame_matrix(oracle_mod, oracle_mod.sector_src_index, N, k) for k in range(12)]
    for k in range(12):
        idx = oracle_mod.sector_src_index(8, k).ravel()
        assert np.array_equal(np.sort(idx), np.arange(8 ** 3))
    rng = np.random.default_rng(1)
    for v in rng.standard_normal((4000, 3)):
        hits = 0
        for P in Ps:
            w = P.T @ v
            a, b = w[1] / w[0], w[2] / w[0]
            hits += (0 <= a <= 1) and (0 <= b <= 1)
        assert hits == 1


def test_sector_forward_consistency(oracle_mod):
    N = 8
    f = synth.random_int32((N, N, N), 54, 0, 1024)
    J = oracle_mod.lines_forward(f)
    Jb = oracle_mod.lines_forward(f, exact="brute")
    np.testing.assert_array_equal(J, Jb)
    for k in (0, 5, 11):
        assert oracle_mod.lines_cell_global(f, k, 3, 6, 9, 4) == int(J[k, 3, 6, 9, 4])


# ---------------------------------------------------------------------------
# Adjoint (eq.(invmap3DJsummation)): pinned to the forward definition by the
# dot-product identity, then the reversed recursion to the transposed scatter.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N", [2, 4, 8])
def test_adjoint_brute_is_transpose_of_definition(oracle_mod, N):
    g = synth.random_int32((N, N, N), 60 + N, -1000, 1000).astype(np.int64)
    r = synth.random_int32((N, N, 2 * N, 2 * N), 61 + N, -1000, 1000).astype(np.int64)
    lhs = int((oracle_mod.lines_brute(g) * r).sum())
    rhs = int((g * oracle_mod.lines_adjoint_brute_frame(r)).sum())
    assert lhs == rhs


@pytest.mark.parametrize("N", [2, 4, 8, 16])
def test_adjoint_recursion_equals_transposed_scatter(oracle_mod, N):
    r = synth.random_int32((N, N, 2 * N, 2 * N), 62 + N)
    want = (oracle_mod.lines_adjoint_brute_frame(r.astype(np.int64)) % (1 << 32)).astype(np.uint32).view(np.int32)
    np.testing.assert_array_equal(oracle_mod.lines_adjoint_frame(r), want)


def test_adjoint_single_cell_backprojects_its_line(oracle_mod):
    """One unit cell at slopes (s1, s2), displacements (d1, d2) spreads a 1 over
    exactly the voxels of its digital line y = l_{s1}(x) + d1 - N,
    z = l_{s2}(x) + d2 - N, computed from eq.(digitalLine) directly."""
    N, n = 8, 3
    for s1, s2, d1, d2 in [(0, 0, 9, 12), (5, 2, 8, 10), (7, 7, 3, 1), (3, 6, 12, 15)]:
        r = np.zeros((N, N, 2 * N, 2 * N), dtype=np.int32)
        r[s1, s2, d1, d2] = 1
        g = oracle_mod.lines_adjoint_frame(r)
        want = np.zeros((N, N, N), dtype=np.int32)
        for x in range(N):
            y, z = lline_rec(n, s1, x) + d1 - N, lline_rec(n, s2, x) + d2 - N
            if 0 <= y < N and 0 <= z < N:
                want[x, y, z] = 1
        np.testing.assert_array_equal(g, want)


def test_adjoint_sector_sum_matches_global_dot_product(oracle_mod):
    """<J f, r> = <f, J^T r> over all 12 sectors, through the sector maps."""
    N = 8
    f = synth.random_int32((N, N, N), 63, -100, 100)
    r = synth.random_int32((12, N, N, 2 * N, 2 * N), 64, -100, 100)
    J = oracle_mod.lines_forward(f).astype(np.int64)
    fb = oracle_mod.lines_adjoint(r).astype(np.int64)
    assert int((J * r.astype(np.int64)).sum()) == int((f.astype(np.int64) * fb).sum())
