"""Pins for the oracle's iterative inverse of the planes transform
(Section 5.2: adjoint + high-pass filter h as approximate inverse, multigrid
with prolongation P and restriction S)."""
import os

import numpy as np
import pytest

import synth

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def press(oracle_mod):
    from oracle import press

    return press


def _golden_h():
    rows = [ln.split() for ln in open(os.path.join(HERE, "golden", "press_filter_h.txt")) if not ln.startswith("#")]
    return np.array(rows, dtype=np.float64).reshape(3, 3, 3) / 64.0


def test_filter_matches_printed_h(press):
    """An interior unit voxel comes back as h itself (the printed values)."""
    N = 8
    d = np.zeros((N, N, N))
    d[4, 3, 5] = 1.0
    np.testing.assert_array_equal(press.hfilter(d)[3:6, 2:5, 4:7], _golden_h()[::-1, ::-1, ::-1])


def test_filter_is_identity_minus_separable_smoothing(press):
    """h = delta - k (x) k (x) k with k = (1/4, 1/2, 1/4) along each axis in
    turn; with mirrored borders it annihilates constants."""
    N = 8
    x = synth.random_float((N, N, N), 3).astype(np.float64)
    i = np.arange(N)
    lo, hi = np.clip(i - 1, 0, N - 1), np.clip(i + 1, 0, N - 1)
    y = x
    for ax in range(3):
        y = 0.25 * y.take(lo, axis=ax) + 0.5 * y + 0.25 * y.take(hi, axis=ax)
    np.testing.assert_allclose(press.hfilter(x), x - y, rtol=0, atol=1e-12)
    assert np.abs(press.hfilter(np.full((N, N, N), 3.5))).max() < 1e-12


def test_restriction_of_prolonged_volume(press, oracle_mod):
    """S(A(P g)) equals A(g) exactly for slopes (0, 0) (slice sums), and every
    (s1, s2) column keeps the total mass."""
    for N in (4, 8):
        g = synth.random_float((N // 2,) * 3, 10 + N).astype(np.float64)
        S = press.restrict(press.A(press.prolong(g)))
        Rc = press.A(g)
        np.testing.assert_allclose(S[:, 0, 0, :], Rc[:, 0, 0, :], rtol=0, atol=1e-12)
        np.testing.assert_allclose(S.sum(-1), np.full(S.shape[:3], g.sum()), rtol=0, atol=1e-10)
        assert S.shape == Rc.shape


def test_coarsest_solve_is_exact(press):
    v = 2.75
    R1 = np.zeros((12, 1, 1, 3))
    R1[:, 0, 0, 2] = v
    assert press.coarsest(R1)[0, 0, 0] == v
    # the restriction chain of an N = 2 transform ends at the volume's mean
    g = synth.random_float((2, 2, 2), 4).astype(np.float64)
    np.testing.assert_allclose(press.coarsest(press.restrict(press.A(g)))[0, 0, 0], g.mean(), rtol=1e-12)


@pytest.mark.parametrize("N", [2, 4])
def test_power_iteration_matches_dense_spectrum(press, N):
    """lambda_N from the power iteration equals the largest eigenvalue of the
    dense matrix of h (*) A^T A built column by column."""
    M = np.zeros((N ** 3, N ** 3))
    for i in range(N ** 3):
        e = np.zeros(N ** 3)
        e[i] = 1.0
        M[:, i] = press.hfilter(press.AT(press.A(e.reshape(N, N, N)))).ravel()
    lam = np.abs(np.linalg.eigvals(M)).max()
    start = synth.random_float((N, N, N), 20 + N).astype(np.float64)
    got = press.spectral_radius(N, start, iterations=200)
    assert abs(got - lam) <= 1e-6 * lam
    assert np.linalg.eigvals(M).real.min() > -1e-9 * lam  # h (*) A^T A has no negative modes


def _steps(press, N):
    return press.step_sizes(N, {L: synth.random_float((L,) * 3, 100 + L).astype(np.float64) for L in
                                (2 ** i for i in range(1, N.bit_length()))})


def test_converges_on_random_volume(press):
    N = 8
    f = synth.random_float((N, N, N), 30).astype(np.float64)
    R = press.A(f)
    hist = press.press_inverse(R, 15, _steps(press, N), history=True)
    err = [press.nrmsd(x, f) for x in hist]
    assert err[-1] < 1e-4
    assert all(b < a for a, b in zip(err, err[1:]))
    res = [np.abs(R - press.A(x)).max() for x in hist]
    assert res[-1] < 1e-4 * np.abs(R).max()


def test_corners_and_centre_example(press):
    """The paper's inversion example (non-zero corner voxels and centre,
    Section 5 figures) at N = 16: ten iterations bring the error below 1e-3."""
    N = 16
    f = np.zeros((N, N, N))
    for x in (0, N - 1):
        for y in (0, N - 1):
            for z in (0, N - 1):
                f[x, y, z] = 1.0
    f[N // 2, N // 2, N // 2] = 1.0
    hist = press.press_inverse(press.A(f), 10, _steps(press, N), history=True)
    assert press.nrmsd(hist[0], f) < 0.05
    assert press.nrmsd(hist[-1], f) < 1e-3


def test_zero_padded_filter_breaks_convergence(press, monkeypatch):
    """Planted reading error: h with zero borders (instead of mirrored) no
    longer annihilates constants, and the same iteration diverges."""
    N = 8
    f = synth.random_float((N, N, N), 31).astype(np.float64)
    R = press.A(f)
    steps = _steps(press, N)
    H = press.H

    def zero_pad(x):
        n = x.shape[0]
        p = np.pad(x, 1)
        out = np.zeros_like(x)
        for a in range(3):
            for b in range(3):
                for c in range(3):
                    out += H[a, b, c] * p[a:a + n, b:b + n, c:c + n]
        return out

    monkeypatch.setattr(press, "hfilter", zero_pad)
    hist = press.press_inverse(R, 15, steps, history=True)
    assert press.nrmsd(hist[-1], f) > 1e-2


def test_fixed_point_is_the_least_squares_solution(press):
    """The iteration converges to the unique solution of A f = R: at N = 4
    it matches a dense least-squares solve with the 12-dodecant operator
    (built column by column from the oracle's transform), which itself
    returns f (A is injective)."""
    N = 4
    M = np.zeros((12 * N * N * 3 * N, N ** 3))
    for i in range(N ** 3):
        e = np.zeros(N ** 3)
        e[i] = 1.0
        M[:, i] = press.A(e.reshape(N, N, N)).ravel()
    f = synth.random_float((N, N, N), 90).astype(np.float64)
    R = press.A(f)
    want = np.linalg.lstsq(M, R.ravel(), rcond=None)[0].reshape(N, N, N)
    np.testing.assert_allclose(want, f, rtol=0, atol=1e-10)  # A is injective
    got = press.press_inverse(R, 60, _steps(press, N))
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-9)
