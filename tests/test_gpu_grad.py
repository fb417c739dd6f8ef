"""GPU parity of the differentiable RGB -> CIELAB: forward, vector-Jacobian
product and the fused mean Delta E*ab loss + gradient against the FP64
oracle, plus torch.autograd.gradcheck of the autograd wrapper."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import tables
from paper_1009_0854_gb300 import autograd, mact, synth
from parity import LAB_TOL

pytestmark = pytest.mark.gpu

KNEE = 0.008856


@pytest.fixture(scope="module", params=[0, 1], ids=["mact", "exact"])
def hx(request):
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return mact.mact_create(exact=request.param), bool(request.param)


def _inputs(n=3, h=40, w=52, seed=0):
    x, tgt_rgb = synth.linear_rgb_batch(n=n, h=h, w=w, seed=seed)
    return x, O.lab_linear(tgt_rgb).astype(np.float32)


def _near_knee(x):
    """Pixels whose FP64 t lies within 1e-7 of the knee on some channel: FP32
    and FP64 may pick different branches there."""
    M = np.array(tables.BT709_MATRIX).reshape(3, 3) / np.array(tables.D65_WHITE)[:, None]
    t = np.einsum("cj,njp->ncp", M, x.reshape(x.shape[0], 3, -1).astype(np.float64))
    return (np.abs(t - KNEE) < 1e-7).any(axis=1).reshape(x.shape[0], *x.shape[2:])


def test_forward_matches_oracle(hx):
    h, exact = hx
    x, _ = _inputs()
    lab = mact.mact_lab_forward(h, torch.from_numpy(x).cuda()).cpu().numpy()
    ref = O.lab_linear(x, exact=exact)
    ok = ~_near_knee(x)[:, None]
    assert np.abs(np.where(ok, lab - ref, 0.0)).max() <= LAB_TOL


def test_fused_loss_and_gradient_match_oracle(hx):
    h, exact = hx
    x, tgt = _inputs(seed=1)
    loss, g = mact.mact_lab_delta_e_loss(h, torch.from_numpy(x).cuda(), torch.from_numpy(tgt).cuda())
    torch.cuda.synchronize()
    rl, rg = O.lab_loss_grad(x, tgt, exact=exact)
    assert float(loss) == pytest.approx(rl, rel=2e-6)
    g = g.cpu().numpy()
    ok = ~_near_knee(x)[:, None]
    scale = np.abs(rg).max()
    err = np.abs(np.where(ok, g - rg, 0.0))
    assert err.max() <= 1e-4 * scale
    # relative agreement elementwise where the gradient is not tiny
    big = ok & (np.abs(rg) > 1e-3 * scale)
    assert (np.abs(g - rg)[big] / np.abs(rg)[big]).max() <= 2e-3


def test_vjp_matches_oracle_and_fused(hx):
    """backward(x, dLoss/dLab) equals the fused gradient when dLoss/dLab is
    the Delta E direction divided by the pixel count."""
    h, exact = hx
    x, tgt = _inputs(seed=2)
    xt = torch.from_numpy(x).cuda()
    lab = mact.mact_lab_forward(h, xt)
    d = lab - torch.from_numpy(tgt).cuda()
    de = d.norm(dim=1, keepdim=True)
    glab = torch.where(de > 0, d / de, torch.zeros_like(d)) / (x.shape[0] * x[0, 0].size)
    g1 = mact.mact_lab_backward(h, xt, glab)
    _, g2 = mact.mact_lab_delta_e_loss(h, xt, torch.from_numpy(tgt).cuda())
    torch.cuda.synchronize()
    scale = g2.abs().max().item()
    assert (g1 - g2).abs().max().item() <= 1e-4 * scale


def _delta_e(h, x, tgt):
    """Per-pixel Delta E*ab (FP64) of the FP32 GPU forward of x against tgt."""
    lab = mact.mact_lab_forward(h, torch.from_numpy(np.ascontiguousarray(x)).cuda()).cpu().numpy()
    return np.sqrt(((lab.astype(np.float64) - tgt) ** 2).sum(axis=1))


def test_finite_differences_of_the_gpu_forward(hx):
    """Finite differences of the per-pixel Delta E*ab that the FP32 GPU
    forward computes, on 1536 pixels drawn like the gradient workload (5% gray
    pixels at exactly 0 or within 1e-4 of the knee), against the FP64 oracle's
    analytic gradient and against the GPU's own fused gradient, element by
    element.

    Away from the knee: central differences with step h = 1e-3.  Where some
    channel's t lies within h |M| of the knee (t = M x, M the matrix rows over
    the white point): the one-sided three-point difference, step 2e-4, on the
    side that keeps every channel on its own branch (the quotient across the
    knee is meaningless: the two branches meet with different slopes).

    Tolerance: |FD - g| <= c e / s + r |g|.  e is the largest
    |Delta E_gpu - Delta E_oracle| measured over every evaluated point (the
    FP32 rounding noise), c / s the stencil's noise gain (2 / (2h) central,
    8 / (2 * 2e-4) one-sided), and r the truncation allowance: 5e-3 central,
    1e-2 one-sided (the FP64 oracle's own differences on these pixels stay
    below 2.5e-3 and 5.4e-3)."""
    h, exact = hx
    x, tgt_rgb = synth.linear_rgb_batch(n=1, h=32, w=48, seed=7)
    tgt = O.lab_linear(tgt_rgb).astype(np.float32).astype(np.float64)
    P = x[0, 0].size
    assert P >= 1000
    _, g_orc = O.lab_loss_grad(x, tgt, exact=exact)
    g_orc = g_orc * P                       # d Delta E / dx per pixel (loss = mean)
    _, g_gpu = mact.mact_lab_delta_e_loss(h, torch.from_numpy(x).cuda(), torch.from_numpy(tgt.astype(np.float32)).cuda())
    g_gpu = g_gpu.cpu().numpy().astype(np.float64) * P
    M = np.array(tables.BT709_MATRIX).reshape(3, 3) / np.array(tables.D65_WHITE)[:, None]
    t = np.einsum("cj,njp->ncp", M, x.reshape(1, 3, -1).astype(np.float64)).reshape(x.shape)
    hc, hs = 1e-3, 2e-4
    noise = [0.0]

    def de(xx):
        d = _delta_e(h, xx, tgt)
        ref = np.sqrt(((O.lab_linear(xx.astype(np.float64), exact=exact) - tgt) ** 2).sum(axis=1))
        noise[0] = max(noise[0], float(np.abs(d - ref).max()))
        return d

    def shifted(c, step):
        y = x.copy()
        y[:, c] = (y[:, c].astype(np.float64) + step).astype(np.float32)
        return y

    f0 = de(x)
    checked = 0
    for c in range(3):
        col = M[:, c][None, :, None, None]
        near = (np.abs(t - KNEE) <= hc * col).any(axis=1)
        up_ok = ((t > KNEE) == (t + 2 * hs * col > KNEE)).all(axis=1)
        dn_ok = ((t > KNEE) == (t - 2 * hs * col > KNEE)).all(axis=1)
        ambiguous = (np.abs(t - KNEE) < 1e-6).any(axis=1) | (near & ~up_ok & ~dn_ok)
        assert ambiguous.sum() <= 4
        xp, xm = shifted(c, hc), shifted(c, -hc)
        central = (de(xp) - de(xm)) / (xp[:, c].astype(np.float64) - xm[:, c])
        # quadratic through (x0, f0), (x1, f1), (x2, f2), differentiated at x0
        # (the exact spacing of the FP32 points)
        sides = []
        for sgn in (1, -1):
            x1, x2 = shifted(c, sgn * hs), shifted(c, 2 * sgn * hs)
            a0, a1, a2 = x[:, c].astype(np.float64), x1[:, c].astype(np.float64), x2[:, c].astype(np.float64)
            f1, f2 = de(x1), de(x2)
            sides.append(f0 * (2 * a0 - a1 - a2) / ((a0 - a1) * (a0 - a2)) +
                         f1 * (a0 - a2) / ((a1 - a0) * (a1 - a2)) + f2 * (a0 - a1) / ((a2 - a0) * (a2 - a1)))
        one_sided = np.where(up_ok, sides[0], sides[1])
        fd = np.where(near, one_sided, central)
        tol_noise = np.where(near, 8.0 / (2 * hs), 2.0 / (2 * hc))
        tol_rel = np.where(near, 1e-2, 5e-3)
        use = ~ambiguous
        for what, g in (("oracle", g_orc[:, c]), ("gpu", g_gpu[:, c])):
            tol = tol_noise * noise[0] + tol_rel * np.abs(g)
            bad = use & (np.abs(fd - g) > tol)
            assert not bad.any(), "%s channel %d: FD %r vs %r at %s" % (
                what, c, fd[bad][:3], g[bad][:3], np.argwhere(bad)[:3].tolist())
        checked += int(use.sum())
    assert noise[0] <= np.sqrt(3) * LAB_TOL
    assert checked >= 3 * 1500


def test_autograd_gradcheck(hx):
    """torch.autograd.gradcheck of the Lab wrapper (FP32, central differences
    with eps = 1e-3) on inputs away from the knee."""
    h, _ = hx
    rng = np.random.default_rng(3)
    x = torch.from_numpy(rng.uniform(0.2, 0.9, size=(1, 3, 4)).astype(np.float32)).cuda().requires_grad_()
    fn = lambda v: autograd.lab(v, h)
    assert torch.autograd.gradcheck(fn, (x,), eps=1e-3, atol=5e-2, rtol=2e-2, nondet_tol=0.0)


def test_loss_autograd_and_knee_sides(hx):
    """The fused loss through autograd; gray pixels on either side of the knee
    get the one-sided derivative of their own branch (oracle)."""
    h, exact = hx
    eps = 3e-5
    x = np.empty((1, 3, 4), dtype=np.float32)
    x[0, :, 0] = KNEE + eps
    x[0, :, 1] = KNEE - eps
    x[0, :, 2] = 0.0
    x[0, :, 3] = 0.6
    tgt = np.array([[[10, 20, 0, 50], [5, -5, 1, 3], [-3, 4, 0, -2]]], dtype=np.float32)
    xt = torch.from_numpy(x).cuda().requires_grad_()
    loss = autograd.delta_e_loss(xt, torch.from_numpy(tgt).cuda(), h)
    loss.backward()
    rl, rg = O.lab_loss_grad(x, tgt, exact=exact)
    assert loss.item() == pytest.approx(rl, rel=1e-5)
    assert np.abs(xt.grad.cpu().numpy() - rg).max() <= 1e-3 * np.abs(rg).max()


def test_unaligned_and_odd_sizes(hx):
    """hw not a multiple of 4 and an offset view take the scalar path."""
    h, exact = hx
    x, tgt = _inputs(n=2, h=7, w=9, seed=4)
    big = torch.zeros(x.size + 1, device="cuda")
    xt = big[1:].view(x.shape)
    xt.copy_(torch.from_numpy(x))
    loss, g = mact.mact_lab_delta_e_loss(h, xt, torch.from_numpy(tgt).cuda())
    rl, rg = O.lab_loss_grad(x, tgt, exact=exact)
    assert float(loss) == pytest.approx(rl, rel=2e-6)
    assert np.abs(g.cpu().numpy() - rg).max() <= 1e-3 * np.abs(rg).max()


def test_full_size_workload_properties(hx):
    """The 64 x 3 x 512 x 512 workload: the loss matches the oracle on the
    whole tensor; gradients match on a sample of images."""
    h, exact = hx
    x, tgt_rgb = synth.linear_rgb_batch(n=64, h=512, w=512, seed=0)
    tgt = O.lab_linear(tgt_rgb).astype(np.float32)
    loss, g = mact.mact_lab_delta_e_loss(h, torch.from_numpy(x).cuda(), torch.from_numpy(tgt).cuda())
    torch.cuda.synchronize()
    rl, rg = O.lab_loss_grad(x, tgt, exact=exact)
    assert float(loss) == pytest.approx(rl, rel=1e-5)
    g = g.cpu().numpy()
    ok = ~_near_knee(x)[:, None]
    assert np.abs(np.where(ok, g - rg, 0.0)).max() <= 2e-4 * np.abs(rg).max()


def test_packed_conversion_kernel_bit_identical_to_scalar_forward():
    """The conversion kernel evaluates MACT CIELAB with packed FP32x2
    instructions (the matrix rows X and Y, the d and q Horner chains, a* and
    b*); the differentiable forward evaluates the same formulas with scalar
    FMAs in the same order.  Fed the same linear values (each 8-bit code's
    FP64 inverse gamma rounded to FP32, as both tables hold it), the two give
    the same bits on every one of the 2^24 colours."""
    h = mact.mact_create()
    lin = np.array([O.gamma_inverse(v / 255.0) for v in range(256)], dtype=np.float32)
    codes = np.arange(1 << 24, dtype=np.int64)
    rgb = np.stack([(codes >> 16) & 255, (codes >> 8) & 255, codes & 255], axis=1).astype(np.uint8)
    x = np.ascontiguousarray(lin[rgb.astype(np.int64)].T[None])         # (1, 3, 2^24) linear RGB
    lab_fwd = mact.mact_lab_forward(h, torch.from_numpy(x).cuda())
    lab_cnv = mact.mact_convert(h, torch.from_numpy(rgb.reshape(4096, 4096, 3)).cuda(), "cielab")
    torch.cuda.synchronize()
    assert torch.equal(lab_fwd.view(3, -1), lab_cnv.view(3, -1))
    h.close()
