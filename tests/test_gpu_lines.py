"""GPU parity of the 3D DJT of lines (Algorithm 3, twelve sectors) against the
oracle: bit-exact int32 (wrapping)."""
import numpy as np
import pytest
import torch

import synth

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
    random cells against the eq.(3DfDJT) definition; sector 0 in full
    against Algorithm 3."""
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
    np.testing.assert_array_equal(J[0].cpu().numpy(), oracle_mod.lines_forward(f, [0])[0])
