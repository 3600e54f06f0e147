"""The FP32 differentiable planes path: forward + hand-written adjoint behind
torch.autograd.Function, checked against the FP64 oracle transpose, finite
differences, the per-cell error bound and a gradient-descent least-squares fit
(8 x 128^3 float32 volumes, standard normal)."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

RTOL = 1e-5


@pytest.fixture(scope="module")
def drt():
    import paper_2501_13664_gb300 as drt3d

    return drt3d


def _dot(a, b):
    return float(torch.dot(a.flatten().double(), b.flatten().double()))


def test_dot_product_against_oracle_transpose(drt, oracle_mod):
    """<A v, r> on the GPU vs <v, A^T r> with the oracle's FP64 backprojection."""
    N = 128
    v = synth.random_float((N, N, N), 500)
    r = synth.random_float((12, N, N, 3 * N), 501)
    Av = drt.planes_forward(torch.from_numpy(v).cuda())
    lhs = _dot(Av, torch.from_numpy(r).cuda())
    Atr = oracle_mod.planes_adjoint(r.astype(np.float64))
    rhs = float(np.dot(v.astype(np.float64).ravel(), Atr.ravel()))
    assert abs(lhs - rhs) <= RTOL * abs(rhs)
    # and the GPU adjoint against the same oracle transpose
    gpu_Atr = drt.planes_adjoint(torch.from_numpy(r).cuda()).cpu().numpy().astype(np.float64)
    mag = oracle_mod.planes_adjoint(np.abs(r).astype(np.float64))
    assert np.all(np.abs(gpu_Atr - Atr) <= RTOL * mag + 1e-30)


def test_forward_per_cell_bound_n128(drt, oracle_mod):
    N = 128
    x = synth.c5_batch(N=N, batch=1)[0]
    got = drt.planes_forward(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    ref = oracle_mod.planes_forward(x.astype(np.float64))
    mag = oracle_mod.planes_forward(np.abs(x).astype(np.float64))
    err = np.abs(got - ref)
    assert np.all(err <= RTOL * mag + 1e-30)
    rel = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    assert rel < 1e-6


def test_autograd_gradient_matches_finite_differences(drt):
    """L(x) = <A x, r> is linear, so its central difference with eps = 1 is
    <A v, r> exactly; autograd returns A^T r through the adjoint kernel."""
    N = 64
    x = torch.from_numpy(synth.random_float((N, N, N), 510)).cuda().requires_grad_(True)
    v = torch.from_numpy(synth.random_float((N, N, N), 511)).cuda()
    r = torch.from_numpy(synth.random_float((12, N, N, 3 * N), 512)).cuda()
    loss = (drt.planes(x).double() * r.double()).sum()
    loss.backward()
    g_dot_v = _dot(x.grad, v)
    with torch.no_grad():
        fd = 0.5 * (_dot(drt.planes(x + v), r) - _dot(drt.planes(x - v), r))
    assert abs(g_dot_v - fd) <= RTOL * abs(fd)


def test_autograd_batched_and_subset(drt):
    N = 16
    x = torch.from_numpy(synth.random_float((2, N, N, N), 520)).cuda().requires_grad_(True)
    y = drt.planes(x, [2, 7])
    assert y.shape == (2, 2, N, N, 3 * N)
    y.sum().backward()
    ones = torch.ones((2, N, N, 3 * N), device="cuda")
    want = drt.planes_adjoint(ones, [2, 7])
    assert torch.allclose(x.grad[0], want, rtol=1e-6, atol=1e-4)
    assert torch.allclose(x.grad[1], want, rtol=1e-6, atol=1e-4)


def test_batched_function_matches_single_volume_calls(drt):
    """The batched autograd function writes each volume's transform into its
    slice and backprojects each cotangent slice: bit for bit the single-volume
    forward and adjoint, N = 32, batch 3, all dodecants."""
    N, B = 32, 3
    x = torch.from_numpy(synth.random_float((B, N, N, N), 530)).cuda().requires_grad_(True)
    y = drt.planes(x)
    assert y.shape == (B, 12, N, N, 3 * N)
    r = torch.from_numpy(synth.random_float((B, 12, N, N, 3 * N), 531)).cuda()
    (y * r).sum().backward()
    for i in range(B):
        assert torch.equal(y[i], drt.planes_forward(x[i].detach()))
        assert torch.equal(x.grad[i], drt.planes_adjoint(r[i]))


@pytest.mark.parametrize("N,dt", [(32, torch.float32), (16, torch.int32), (16, torch.uint8), (64, torch.uint8)])
def test_forward_residual_is_forward_minus_target(drt, N, dt):
    """drt3d_planes_forward_residual: A x - b subtracted as the last pass
    stores, bit for bit the forward followed by the subtraction (float32
    rounding once, integers wrapping); also in place over the target."""
    mask = [0, 3, 7, 11]
    if dt == torch.float32:
        x = torch.from_numpy(synth.random_float((N, N, N), 540 + N)).cuda()
        b = torch.from_numpy(synth.random_float((4, N, N, 3 * N), 541 + N)).cuda()
    else:
        x = torch.from_numpy(synth.random_int32((N, N, N), 540 + N, 0, 256)).to(dt).cuda()
        b = torch.from_numpy(synth.random_int32((4, N, N, 3 * N), 541 + N)).cuda()
    want = drt.planes_forward(x, mask) - b
    assert torch.equal(drt.planes_forward_residual(x, b, mask), want)
    b2 = b.clone()
    drt.planes_forward_residual(x, b2, mask, out=b2)
    assert torch.equal(b2, want)


@pytest.mark.parametrize("N,mask", [(16, 0xFFF), (32, 0xFFF), (64, 0b100100010001)])
def test_residual_loss_is_half_the_squared_residual(drt, N, mask):
    """The loss summed in the last pass's stores equals 0.5 * sum r^2 of the
    residual it stored (float64 over the float32 cells), is the same on every
    call (fixed summation order), and leaves r bit for bit as the plain
    residual entry writes it."""
    ks = [k for k in range(12) if (mask >> k) & 1]
    x = torch.from_numpy(synth.random_float((N, N, N), 41)).cuda()
    b = torch.from_numpy(synth.random_float((len(ks), N, N, 3 * N), 42)).cuda()
    r_ref = drt.planes_forward_residual(x, b, ks)
    r, loss = drt.planes_forward_residual_loss(x, b, ks)
    assert torch.equal(r, r_ref)
    ref = 0.5 * float((r_ref.double() ** 2).sum())
    assert abs(float(loss) - ref) <= 1e-6 * ref
    _, loss2 = drt.planes_forward_residual_loss(x, b, ks)
    assert float(loss2) == float(loss)


def test_least_squares_loss_matches_autograd_of_mse(drt):
    """The least-squares autograd function (residual in the forward's store,
    adjoint of the saved residual) gives the same gradient, bit for bit, as
    autograd through the batched transform and PyTorch's squared error, and
    the same loss up to its float64 summation."""
    from paper_2501_13664_gb300 import lsq

    N, B = 32, 2
    x = torch.from_numpy(synth.random_float((B, N, N, N), 550)).cuda()
    b = torch.from_numpy(synth.random_float((B, 12, N, N, 3 * N), 551)).cuda()
    xa = x.clone().requires_grad_(True)
    la = 0.5 * torch.nn.functional.mse_loss(drt.planes(xa), b, reduction="sum")
    la.backward()
    xb = x.clone().requires_grad_(True)
    lb = lsq.least_squares_loss(xb, b)
    lb.backward()
    assert torch.equal(xa.grad, xb.grad)
    # the float32 residual, squared and summed in float64; the loss sums in float32
    ref = 0.5 * float(((drt.planes(x) - b).double() ** 2).sum())
    assert abs(float(lb.detach()) - ref) <= 1e-5 * ref
    assert abs(float(la.detach()) - ref) <= 1e-5 * ref


def test_lsq_trajectory_against_fp64_oracle(drt, oracle_mod):
    """50 steps of gradient descent (step 1/L) at N = 32, batch 2, against the
    same iteration run with the oracle's FP64 forward and backprojection."""
    from paper_2501_13664_gb300 import lsq

    N, B, steps = 32, 2, 50
    xs = synth.c5_batch(N=N, batch=B, seed=5)
    b64 = np.stack([oracle_mod.planes_forward(x.astype(np.float64)) for x in xs])
    b = torch.from_numpy(b64.astype(np.float32)).cuda()
    L = lsq.operator_norm_sq(N)
    _, losses = lsq.fit(b, steps=steps, L=L)
    x = np.zeros((B, N, N, N))
    ref = []
    for _ in range(steps):
        r = np.stack([oracle_mod.planes_forward(xi) for xi in x]) - b64
        ref.append(0.5 * float((r ** 2).sum()))
        g = np.stack([oracle_mod.planes_adjoint(ri) for ri in r])
        x = x - g / L
    ref = np.array(ref)
    got = np.array(losses)
    assert np.all(np.diff(got) <= 1e-9 * got[0])  # monotone descent
    assert np.max(np.abs(got - ref) / ref) < 1e-4
    assert got[-1] < got[0]


def test_config_c5_lsq_fit(drt, oracle_mod):
    """8 x 128^3 float32 N(0,1) volumes; target b = A x* from the FP64 oracle;
    50 steps from x = 0 with step 1/L (L from 20 power iterations of A^T A)."""
    from paper_2501_13664_gb300 import lsq

    N, B = 128, 8
    xs = synth.c5_batch(N=N, batch=B)
    b = torch.stack([torch.from_numpy(oracle_mod.planes_forward(x.astype(np.float64)).astype(np.float32))
                     for x in xs]).cuda()
    L = lsq.operator_norm_sq(N)
    assert L > 0
    x, losses = lsq.fit(b, steps=50, L=L)
    got = np.array(losses)
    assert np.all(np.diff(got) <= 1e-7 * got[0])
    assert got[-1] < got[0]
    # the fitted volumes move toward x*: residual ||x - x*|| decreases
    xt = torch.from_numpy(xs).cuda()
    assert float((x - xt).norm()) < float(xt.norm())
