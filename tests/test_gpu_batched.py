"""The batched persistent planes forward (many uint8 volumes of uneven N in one
launch) against one-by-one calls and the oracle; schedules, graph replay and
the bounded-wait error path."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def drt():
    import paper_2501_13664_gb300 as drt3d

    return drt3d


def _vols(Ns, seed0):
    return [torch.from_numpy(synth.c2_volume(N, seed=seed0 + i)).cuda() for i, N in enumerate(Ns)]


def test_small_mixed_batch_matches_one_by_one_and_oracle(drt, oracle_mod):
    Ns = [16, 32, 64, 32, 16, 128, 64]
    vols = _vols(Ns, 40)
    bp = drt.BatchPlan(Ns)
    outs = bp.bind(vols)
    bp.run()
    assert bp.device_error() == 0
    for v, o, N in zip(vols, outs, Ns):
        assert torch.equal(o, drt.planes_forward(v))
        if N <= 32:
            np.testing.assert_array_equal(o.cpu().numpy(), oracle_mod.planes_forward(v.cpu().numpy()))


def test_schedule_overrides_give_identical_results(drt):
    Ns = [64, 128, 256, 32]
    vols = _vols(Ns, 60)
    ref = [drt.planes_forward(v) for v in vols]
    bp = drt.BatchPlan(Ns, schedules={64: (2, 2, 2), 128: (2, 3, 2), 256: (3, 3, 2), 32: (2, 3)})
    outs = bp.bind(vols)
    bp.run()
    assert bp.device_error() == 0
    for o, r in zip(outs, ref):
        assert torch.equal(o, r)
    # and the same splits on single-volume plans
    for v, r, groups in zip(vols, ref, [(2, 2, 2), (3, 2, 2), (2, 2, 2, 2), (3, 2)]):
        plan = drt.get_plan(int(v.shape[0]), torch.uint8)
        old = plan.schedule()
        plan.set_schedule(groups)
        try:
            assert torch.equal(drt.planes_forward(v), r)
        finally:
            plan.set_schedule(old)


@pytest.mark.parametrize("tiles", [1, 3, 8, 1000])
def test_item_sizes_give_identical_results(drt, tiles):
    """Work items of 1, 3 (not a divisor of a unit's tiles), 8 and more than
    a dodecant's unit-tiles, on every pass of every size."""
    Ns = [16, 32, 64, 128, 256, 64]
    vols = _vols(Ns, 80)
    ref = [drt.planes_forward(v) for v in vols]
    scheds = {16: (4,), 32: (3, 2), 64: (3, 3), 128: (4, 3), 256: (4, 4)}
    bp = drt.BatchPlan(Ns, schedules=scheds, item_tiles={N: [tiles] * len(g) for N, g in scheds.items()})
    outs = bp.bind(vols)
    bp.run()
    assert bp.device_error() == 0
    for o, r in zip(outs, ref):
        assert torch.equal(o, r)


def test_item_size_arguments_are_checked(drt):
    bp = drt.BatchPlan([32, 64], schedules={64: (3, 3)})
    for N, tiles, code in [(64, [8], 1),        # two passes at N = 64: INVALID_ARG
                           (128, [8, 8], 2),    # no volume of that size: SIZE
                           (64, [8, -1], 1)]:   # negative: INVALID_ARG
        with pytest.raises(drt.DRT3DError) as e:
            bp.set_item_tiles(N, tiles)
        assert e.value.code == code
    bp.set_item_tiles(64, [0, 2])  # 0 keeps the default


def test_config_c4_batch_matches_one_by_one(drt, oracle_mod):
    """96 volumes, sizes 16:30, 32:30, 64:20, 128:10, 256:6 shuffled."""
    sizes = synth.c4_sizes()
    vols = [torch.from_numpy(v).cuda() for v in synth.c4_batch(sizes=sizes)]
    bp = drt.BatchPlan(sizes)
    outs = bp.bind(vols)
    bp.run()
    assert bp.device_error() == 0
    checked = 0
    for i, (v, o, N) in enumerate(zip(vols, outs, sizes)):
        assert torch.equal(o, drt.planes_forward(v)), f"volume {i} (N={N})"
        if N == 16 and checked < 3:
            np.testing.assert_array_equal(o.cpu().numpy(), oracle_mod.planes_forward(v.cpu().numpy()))
            checked += 1


@pytest.mark.parametrize("streams", [1, 3, 8])
def test_multistream_mode_matches_one_by_one(drt, streams):
    """Mode 1 (per-volume launches over internal streams) on the 96-volume
    batch: identical results, also when replayed from a CUDA graph."""
    sizes = synth.c4_sizes()
    vols = [torch.from_numpy(v).cuda() for v in synth.c4_batch(sizes=sizes)]
    bp = drt.BatchPlan(sizes)
    bp.set_mode(1, streams)
    outs = bp.bind(vols)
    want = [drt.planes_forward(v) for v in vols]
    bp.run()
    torch.cuda.synchronize()
    assert bp.device_error() == 0
    for i, (o, w) in enumerate(zip(outs, want)):
        assert torch.equal(o, w), f"volume {i}"
    for o in outs:
        o.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bp.run()
    g.replay()
    torch.cuda.synchronize()
    for i, (o, w) in enumerate(zip(outs, want)):
        assert torch.equal(o, w), f"volume {i} (graph)"
    bp.set_mode(0)
    for o in outs:
        o.zero_()
    bp.run()
    torch.cuda.synchronize()
    assert all(torch.equal(o, w) for o, w in zip(outs, want))
    with pytest.raises(Exception):
        bp.set_mode(1, 9)


def test_batched_launch_replays_in_a_cuda_graph(drt):
    Ns = [32, 64, 16]
    vols = _vols(Ns, 80)
    bp = drt.BatchPlan(Ns)
    outs = bp.bind(vols)
    want = [drt.planes_forward(v) for v in vols]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        bp.run()  # warm-up outside capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    for o in outs:
        o.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bp.run()
    for _ in range(2):
        for o in outs:
            o.zero_()
        g.replay()
        torch.cuda.synchronize()
        for o, w in zip(outs, want):
            assert torch.equal(o, w)
    assert bp.device_error() == 0


def test_withheld_signal_times_out_without_a_fault(drt):
    """A first-pass completion signal that never arrives: the dependent waits
    give up after the limit, the launch ends and reports DRT3D_ERR_TIMEOUT;
    the plan works again once the hook is cleared."""
    Ns = [64, 32]
    vols = _vols(Ns, 90)
    bp = drt.BatchPlan(Ns)
    outs = bp.bind(vols)
    bp.set_wait_limit(2_000_000, withhold_vol=0, withhold_dodecant=3)  # 2 ms
    bp.run()
    assert bp.device_error() == 7  # DRT3D_ERR_TIMEOUT
    bp.set_wait_limit(2_000_000_000)
    bp.run()
    assert bp.device_error() == 0
    for v, o in zip(vols, outs):
        assert torch.equal(o, drt.planes_forward(v))
