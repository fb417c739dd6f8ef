"""Cube-root rationals fitted by the library at create time (lab_coeffs = 1):
degrees up to (6, 6) that Table tab_cbrt_rat does not print.  The library's
Remez exchange (C++) and the oracle's (numpy) are separate implementations of
the same minimax problem; each GPU result is compared with the oracle
evaluating its own fit, within the parity tolerances."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1009_0854_gb300 import mact, synth
from parity import LAB_TOL, check_space

pytestmark = pytest.mark.gpu

DEGREES = [(4, 4), (5, 5), (6, 6), (3, 5)]


@pytest.fixture(scope="module")
def images():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    img = synth.gradient_noise_image(512, 512, seed=0)
    cube = synth.rgb_cube().reshape(-1, 3)
    sample = cube[:: 16].copy().reshape(1024, 1024, 3)          # every 16th colour of the cube
    return [img, sample]


@pytest.mark.parametrize("n,m", DEGREES)
def test_fitted_rational_matches_oracle(images, n, m):
    h = mact.mact_create(lab_coeffs=1, lab_n=n, lab_m=m)
    p, q, _ = O.cbrt_minimax(n, m)
    for im in images:
        got = mact.mact_convert(h, torch.from_numpy(im).cuda(), "cielab")
        torch.cuda.synchronize()
        ref = O.cielab(im, p=p, q=q)
        check_space("cielab", got, ref, torch.float32, "(%d,%d)" % (n, m))


@pytest.mark.parametrize("n,m", [(5, 5), (6, 6)])
def test_fitted_rational_cube_error(n, m):
    """Device error statistics over every 24-bit colour (production FP32
    kernel vs FP64 exact) against the oracle's FP64 statistics of its fit."""
    a, b = mact.mact_cube_error(mact.mact_create(lab_coeffs=1, lab_n=n, lab_m=m), "cielab")
    p, q, _ = O.cbrt_minimax(n, m)
    ra, rb = O.cube_eps_cielab(p=p, q=q)
    assert abs(a - ra) <= 2e-5 and abs(b - rb) <= 3.5e-4
    if (n, m) == (6, 6):
        # the approximant's error is down at the level of the exact FP32 path's
        e_exact = mact.mact_cube_error(mact.mact_create(exact=1), "cielab")[1]
        assert b < 3 * e_exact


def test_fitted_rational_batched_and_single_agree(images):
    h = mact.mact_create(lab_coeffs=1, lab_n=6, lab_m=6)
    items = [(torch.from_numpy(im).cuda(), sp) for im, sp in synth.batch_images(count=10, seed=5, lo=8, hi=700)]
    items += [(torch.from_numpy(images[0]).cuda(), "cielab")]
    for lst in (items, items * 4):           # by-value list, then device work list
        outs = mact.mact_convert_batch(h, lst)
        torch.cuda.synchronize()
        for (rgb, sp), o in zip(lst, outs):
            assert torch.equal(o, mact.mact_convert(h, rgb, sp))


def test_fitted_rational_forward_and_gradient():
    h = mact.mact_create(lab_coeffs=1, lab_n=6, lab_m=6)
    p, q, _ = O.cbrt_minimax(6, 6)
    x, tgt_rgb = synth.linear_rgb_batch(n=2, h=40, w=52, seed=3)
    tgt = O.lab_linear(tgt_rgb).astype(np.float32)
    lab = mact.mact_lab_forward(h, torch.from_numpy(x).cuda()).cpu().numpy()
    ref = O.lab_linear(x, p=p, q=q)
    t = np.einsum("cj,njp->ncp", np.array(O.tables.BT709_MATRIX).reshape(3, 3) /
                  np.array(O.tables.D65_WHITE)[:, None], x.reshape(2, 3, -1).astype(np.float64))
    ok = ~(np.abs(t - 0.008856) < 1e-7).any(axis=1).reshape(2, 1, 40, 52)
    assert np.abs(np.where(ok, lab - ref, 0.0)).max() <= LAB_TOL
    loss, g = mact.mact_lab_delta_e_loss(h, torch.from_numpy(x).cuda(), torch.from_numpy(tgt).cuda())
    torch.cuda.synchronize()
    rl, rg = O.lab_loss_grad(x, tgt, p=p, q=q)
    assert float(loss) == pytest.approx(rl, rel=2e-6)
    scale = np.abs(rg).max()
    assert np.abs(np.where(ok, g.cpu().numpy() - rg, 0.0)).max() <= 1e-4 * scale


@pytest.mark.parametrize("kw", [dict(lab_coeffs=2), dict(lab_coeffs=1, lab_n=7, lab_m=6),
                                dict(lab_coeffs=1, lab_n=4, lab_m=0)])
def test_fitted_rational_config_is_validated(kw):
    with pytest.raises(mact.MactError) as e:
        mact.mact_create(**kw)
    assert e.value.status == mact.MACT_E_INVAL
