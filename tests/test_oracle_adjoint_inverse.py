"""Pins for the oracle's planes adjoint (Section 5.1) and exact integer inverse."""
import numpy as np
import pytest

import synth


@pytest.mark.parametrize("N", [2, 4, 8, 16])
def test_adjoint_identity_exact(oracle_mod, N):
    """<A f, r> == <f, A^T r> exactly (integers, no wrap at these magnitudes)."""
    f = synth.random_int32((N, N, N), 21, -50, 50)
    r = synth.random_int32((12, N, N, 3 * N), 22, -50, 50)
    Af = oracle_mod.planes_forward(f).astype(np.int64)
    Atr = oracle_mod.planes_adjoint(r).astype(np.int64)
    assert int((Af * r).sum()) == int((f.astype(np.int64) * Atr).sum())


@pytest.mark.parametrize("N", [4, 8])
def test_adjoint_recursion_equals_transposed_definition(oracle_mod, N):
    rb = synth.random_float((N, N, 3 * N), 23).astype(np.float64)
    np.testing.assert_allclose(oracle_mod.planes_adjoint_frame(rb),
                               oracle_mod.planes_adjoint_brute_frame(rb), rtol=0, atol=1e-9)


@pytest.mark.parametrize("N", [4, 8])
def test_adjoint_float_matches_int(oracle_mod, N):
    r = synth.random_int32((12, N, N, 3 * N), 24, -100, 100)
    np.testing.assert_array_equal(oracle_mod.planes_adjoint(r.astype(np.float64)),
                                  oracle_mod.planes_adjoint(r).astype(np.float64))


def test_adjoint_of_single_cell_is_its_plane(oracle_mod):
    """Backprojecting one cell spreads it uniformly on the voxels of that plane."""
    N = 8
    r = np.zeros((1, N, N, 3 * N), dtype=np.int32)
    s1, s2, d = 5, 3, 2 * N - 2
    r[0, s1, s2, d] = 1
    back = oracle_mod.planes_adjoint(r, dodecants=[0])
    g = np.ones((N, N, N), dtype=np.int32)
    assert int(back.sum()) == oracle_mod.planes_cell(g, s1, s2, d)
    assert set(np.unique(back)).issubset({0, 1})


@pytest.mark.parametrize("N", [2, 4, 8, 16])
def test_inverse_round_trip_every_dodecant(oracle_mod, N):
    f = synth.random_int32((N, N, N), 30 + N)  # full range: forward sums wrap
    R = oracle_mod.planes_forward(f)
    for k in range(12):
        back, ok = oracle_mod.planes_inverse(R[k], k)
        assert ok
        np.testing.assert_array_equal(back, f)


def test_inverse_round_trip_n64(oracle_mod):
    f = synth.c2_volume(64, seed=2)
    R = oracle_mod.planes_forward(f, dodecants=[7])[0]
    back, ok = oracle_mod.planes_inverse(R, 7)
    assert ok
    np.testing.assert_array_equal(back, f.astype(np.int32))


@pytest.mark.parametrize("cell", [(0, 0, 3 * 8 - 1), (3, 5, 10), (7, 7, 2)])
def test_inverse_flags_data_outside_the_range(oracle_mod, cell):
    N = 8
    f = synth.random_int32((N, N, N), 40, 0, 256)
    R = oracle_mod.planes_forward(f, dodecants=[0])[0]
    R[cell] += 1
    _, ok = oracle_mod.planes_inverse(R, 0)
    assert not ok
