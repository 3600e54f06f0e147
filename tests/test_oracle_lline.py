"""Pins for the oracle's digital line, eq.(digitalLine) (Section 2.1)."""
import os

import numpy as np
import pytest

from _paper_refs import lline_rec_table

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lline_n8.txt")


def test_golden_table_n8(oracle_mod):
    want = np.loadtxt(GOLDEN, dtype=np.int64)
    np.testing.assert_array_equal(oracle_mod.lline_table(8), want)


@pytest.mark.parametrize("N", [2, 4, 8, 16, 32, 64])
def test_sum_form_equals_recursive_form(oracle_mod, N):
    np.testing.assert_array_equal(oracle_mod.lline_table(N), lline_rec_table(N))


@pytest.mark.parametrize("N", [2, 4, 8, 16, 32, 64, 128, 256])
def test_line_properties(oracle_mod, N):
    T = oracle_mod.lline_table(N)
    s = np.arange(N)
    # starts at 0, ends at the ascent s (the line joins p0 to p1 + s d)
    np.testing.assert_array_equal(T[:, 0], 0)
    np.testing.assert_array_equal(T[:, N - 1], s)
    # slope 0 is flat, slope N-1 is the diagonal
    np.testing.assert_array_equal(T[0], 0)
    np.testing.assert_array_equal(T[N - 1], s)
    # loose line: unit steps only
    steps = np.diff(T, axis=1)
    assert set(np.unique(steps)).issubset({0, 1})
    # central symmetry l_s(u) + l_s(N-1-u) = s
    np.testing.assert_array_equal(T + T[:, ::-1], np.repeat(s[:, None], N, axis=1))
    # exactly s ascents
    np.testing.assert_array_equal(steps.sum(axis=1), s)
