"""Compute calls from several host threads at once, each on its own CUDA
stream (ctypes releases the GIL around every C call): every thread's results
equal the oracle's, and the iterative inverse -- whose coarser-level plans are
created on first use -- gives the same bits from concurrent first calls as
from a later single-threaded one."""
import threading

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

THREADS = 4


def _run_threads(work):
    errors, barrier = [], threading.Barrier(THREADS)

    def body(i):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                work(i, barrier)
            s.synchronize()
        except BaseException as e:  # reported by the main thread
            errors.append(e)
            barrier.abort()

    ts = [threading.Thread(target=body, args=(i,)) for i in range(THREADS)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    if errors:
        raise errors[0]


def test_forward_inverse_2d_from_threads(oracle_mod):
    import paper_2501_13664_gb300 as drt

    N = 32
    vols = [synth.random_int32((N, N, N), 940 + i, 0, 256).astype(np.uint8) for i in range(THREADS)]
    imgs = [synth.images_2d(N, 3, seed=950 + i) for i in range(THREADS)]
    want_R = [oracle_mod.planes_forward(v) for v in vols]
    want_2d = [oracle_mod.drt2d_forward(f) for f in imgs]
    got = [None] * THREADS

    def work(i, barrier):
        vol = torch.from_numpy(vols[i]).cuda()
        img = torch.from_numpy(imgs[i]).cuda()
        barrier.wait()
        outs = []
        for rep in range(3):
            R = drt.planes_forward(vol)
            k = (i + rep) % 12
            f = drt.planes_inverse(R[k], k)
            D = drt.drt2d_forward(img)
            outs.append((R.cpu().numpy(), k, f.cpu().numpy(), D.cpu().numpy()))
        got[i] = outs

    _run_threads(work)
    for i in range(THREADS):
        for R, k, f, D in got[i]:
            np.testing.assert_array_equal(R, want_R[i])
            np.testing.assert_array_equal(f, vols[i].astype(np.int32))
            np.testing.assert_array_equal(D, want_2d[i])


def test_press_inverse_first_calls_from_threads():
    import paper_2501_13664_gb300 as drt

    N = 8  # a fresh float32 plan: its level plans do not exist yet
    drt._plan_cache.pop((torch.cuda.current_device(), N, torch.float32), None)
    f = synth.random_float((N, N, N), 960)
    R = drt.planes_forward(torch.from_numpy(f).cuda())
    steps = drt.press_step_sizes(N)
    drt._plan_cache.pop((torch.cuda.current_device(), N, torch.float32), None)
    got = [None] * THREADS

    def work(i, barrier):
        barrier.wait()
        got[i] = drt.planes_press_inverse(R, 4, steps=steps).cpu().numpy()

    _run_threads(work)
    want = drt.planes_press_inverse(R, 4, steps=steps).cpu().numpy()
    for g in got:
        np.testing.assert_array_equal(g, want)
    assert np.abs(want - f).max() < np.abs(f).max()  # and it is converging
