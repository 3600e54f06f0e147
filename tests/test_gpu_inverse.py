"""GPU parity of the exact integer inverse (round trip through the forward)."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def drt():
    import paper_2501_13664_gb300 as drt3d

    return drt3d


@pytest.mark.parametrize("N", [2, 4, 8, 16, 32, 64])
def test_round_trip_every_dodecant_wrapping(drt, N):
    f = torch.from_numpy(synth.random_int32((N, N, N), 60 + N)).cuda()  # sums wrap
    R = drt.planes_forward(f)
    for k in range(12):
        back = drt.planes_inverse(R[k], k)
        assert torch.equal(back, f), f"dodecant {k}"


def test_gpu_forward_oracle_inverse_agree(drt, oracle_mod):
    N = 16
    f = synth.random_int32((N, N, N), 70, 0, 256)
    R = drt.planes_forward(torch.from_numpy(f).cuda()).cpu().numpy()
    for k in (0, 6, 11):
        want, ok = oracle_mod.planes_inverse(R[k], k)
        assert ok
        got = drt.planes_inverse(torch.from_numpy(R[k]).cuda(), k).cpu().numpy()
        np.testing.assert_array_equal(got, want)


def test_config_c2_round_trip_all_dodecants(drt):
    """N = 256 uint8 volume: forward over 12 dodecants, exact inverse from each."""
    N = 256
    f = torch.from_numpy(synth.c2_volume(N)).cuda()
    R = drt.planes_forward(f)
    f32 = f.to(torch.int32)
    for k in range(12):
        assert torch.equal(drt.planes_inverse(R[k], k), f32), f"dodecant {k}"


def test_round_trip_n128(drt):
    N = 128
    f = torch.from_numpy(synth.c2_volume(N, seed=9)).cuda()
    R = drt.planes_forward(f, [3, 8])
    assert torch.equal(drt.planes_inverse(R[0], 3), f.to(torch.int32))
    assert torch.equal(drt.planes_inverse(R[1], 8), f.to(torch.int32))


@pytest.mark.parametrize("N,cell", [(8, (0, 0, 23)), (8, (3, 5, 10)), (32, (7, 7, 2)), (32, (31, 0, 60))])
def test_out_of_range_input_is_flagged(drt, N, cell):
    f = torch.from_numpy(synth.random_int32((N, N, N), 80, 0, 256)).cuda()
    R = drt.planes_forward(f, [0])[0].clone()
    R[cell] += 1
    with pytest.raises(drt.NotInRangeError):
        drt.planes_inverse(R, 0)
    # the status word is cleared by the read: a valid call afterwards is clean
    R2 = drt.planes_forward(f, [0])[0]
    assert torch.equal(drt.planes_inverse(R2, 0), f)


def test_inverse_rejects_float_and_bad_index(drt):
    R = torch.zeros((8, 8, 24), dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):
        drt.planes_inverse(R, 12)
    with pytest.raises(ValueError):
        drt.planes_inverse(R.float(), 0)
