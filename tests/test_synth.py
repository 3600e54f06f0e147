"""The seeded input generators: determinism, shapes and value ranges."""
import numpy as np

import synth


def test_c1():
    a, b = synth.c1_volume(), synth.c1_volume()
    assert a.shape == (32, 32, 32) and a.dtype == np.int32
    np.testing.assert_array_equal(a, b)
    assert a.min() >= 0 and a.max() <= 255


def test_c2_small():
    f = synth.c2_volume(64)
    assert f.dtype == np.uint8 and f.shape == (64, 64, 64)
    np.testing.assert_array_equal(f, synth.c2_volume(64))
    nz = np.count_nonzero(f)
    assert 0.01 * 64 ** 3 * 0.9 <= nz <= 0.01 * 64 ** 3 + 8 * 64 * 64
    assert (f == 255).sum() >= 8 * 64  # the planes are there


def test_c3_small():
    f = synth.c3_volume(32)
    assert f.dtype == np.int16 and f.min() >= 0 and f.max() == 1023


def test_c4_sizes():
    sizes = synth.c4_sizes()
    assert len(sizes) == 96
    for N, c in synth.C4_COUNTS.items():
        assert sizes.count(N) == c
    assert sizes == synth.c4_sizes()


def test_c5_small():
    x = synth.c5_batch(N=16, batch=2)
    assert x.shape == (2, 16, 16, 16) and x.dtype == np.float32
    assert abs(float(x.mean())) < 0.1
