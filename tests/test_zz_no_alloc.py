"""The allocation-free planes forward, drt3d_planes_forward_noalloc.

Some callers cannot allocate device memory where they run the transform: a
host callback or real-time loop that must stay out of the allocator, a
plug-in host that only hands out the input and output buffers, or a process
whose device memory another framework reserved up front.  This entry point
runs the forward transform with a fixed 16 MiB scratch array owned by the
library, so such a caller passes only the input and the output.

The file name sorts last so that a run stopping at the first failure has
already run every other test; the tests also pass alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def drt():
    import paper_2501_13664_gb300 as drt3d

    return drt3d


def _noalloc(drt, plan, vol, out, mask):
    lib = drt._abi.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.drt3d_planes_forward_noalloc(plan.handle, vol.data_ptr(), out.data_ptr(), mask, stream)


@pytest.mark.parametrize("N,dtype,mask", [(8, torch.int32, 0xFFF), (32, torch.int32, 0xFFF),
                                          (64, torch.uint8, 0xFFF), (16, torch.float32, 0xFFF),
                                          (128, torch.uint8, 0x020)])
def test_noalloc_matches_the_workspace_entry_point_on_two_calls(drt, N, dtype, mask):
    plan = drt.get_plan(N, dtype)
    for call in range(2):  # consecutive calls share the scratch array
        if dtype == torch.uint8:
            f = torch.from_numpy(synth.c2_volume(N, seed=100 + call)).cuda()
        elif dtype == torch.float32:
            f = torch.from_numpy(synth.random_float((N, N, N), 100 + call)).cuda()
        else:
            f = torch.from_numpy(synth.random_int32((N, N, N), 100 + call)).cuda()
        want = drt.planes_forward(f, mask)
        got = torch.full_like(want, 7)
        assert _noalloc(drt, plan, f, got, mask) == 0
        torch.cuda.synchronize()
        # same kernels on the same data: identical bit for bit, float32 included
        # (a stale or aliased scratch value would show as any difference)
        assert torch.equal(got, want), f"call {call}"


def test_noalloc_rejects_calls_beyond_its_scratch(drt):
    lib = drt._abi.lib()
    assert lib.drt3d_noalloc_scratch_bytes() == 16 << 20
    N = 128
    plan = drt.get_plan(N, torch.int32)
    f = torch.zeros((N, N, N), dtype=torch.int32, device="cuda")
    out = torch.full((12, N, N, 3 * N), 5, dtype=torch.int32, device="cuda")
    assert _noalloc(drt, plan, f, out, 0xFFF) == 11  # DRT3D_ERR_SCRATCH_LIMIT
    torch.cuda.synchronize()
    assert bool((out == 5).all())  # nothing was enqueued
    assert _noalloc(drt, plan, f, out, 0) == 1       # empty mask: INVALID_ARG
