"""HSI LUT with angular hue interpolation on the GPU against the oracle: the
(cos H, sin H, S, I) node table, trilinear S and I, and the pairwise hue mix
of Eq. equ_angular along B, G, R.  Hue is compared where the oracle's mix
stays well conditioned (smallest mix modulus >= 0.1; antipodal hues mixed
near a = 0.5 have no reliable direction in any precision); S and I
everywhere."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_1009_0854_gb300 import mact, synth
from parity import HUE_TOL, SI_TOL

pytestmark = pytest.mark.gpu
TWO_PI = 2.0 * math.pi


@pytest.fixture(scope="module")
def h():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return mact.mact_create()


def _circ(a, b):
    d = np.abs(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)) % TWO_PI
    return np.minimum(d, TWO_PI - d)


def test_node_table_matches_oracle_lut(h):
    for n in (17, 33):
        lut4 = mact.mact_lut_build_hsi(h, n).cpu().numpy().reshape(-1, 4).astype(np.float64)
        ref = O.lut_build_hsi(n).reshape(-1, 3).astype(np.float64)
        gray = ref[:, 1] == 0.0
        assert np.all((lut4[gray, :3] == 0.0))
        assert np.abs(lut4[:, 2] - ref[:, 1]).max() == 0.0 and np.abs(lut4[:, 3] - ref[:, 2]).max() == 0.0
        hue = np.arctan2(lut4[~gray, 1], lut4[~gray, 0]) % TWO_PI
        assert _circ(hue, ref[~gray, 0]).max() <= 2e-7
        assert np.abs(np.hypot(lut4[~gray, 0], lut4[~gray, 1]) - 1.0).max() <= 2e-7


@pytest.mark.parametrize("n", [17, 33, 18])
def test_interpolation_matches_oracle(h, n):
    lut4 = mact.mact_lut_build_hsi(h, n)
    lut = O.lut_build_hsi(n)
    cube = synth.rgb_cube().reshape(-1, 3)
    for rgb in (synth.gradient_noise_image(512, 512, seed=0).reshape(-1, 3), cube[7::13].copy()):
        got = mact.mact_lut_interp_hsi(h, lut4, torch.from_numpy(rgb).cuda()).cpu().numpy().astype(np.float64)
        (H, S, I), cond = O.lut_interp_hsi(lut, rgb)
        assert np.abs(got[1] - S).max() <= SI_TOL and np.abs(got[2] - I).max() <= SI_TOL
        ok = (cond >= 0.1) & (S > 0)
        assert ok.mean() > 0.999
        assert _circ(got[0][ok], H[ok]).max() <= HUE_TOL
        assert np.all(got[0][S == 0] == 0.0)
        assert got[0].min() >= 0.0 and got[0].max() < TWO_PI


def test_cube_error_average(h):
    """Over every 24-bit colour, D_HSI of the GPU result against the exact
    HSI averages to the oracle's eps^T_avg (33^3, trilinear)."""
    lut4 = mact.mact_lut_build_hsi(h, 33)
    cube = synth.rgb_cube().reshape(-1, 3)
    got = mact.mact_lut_interp_hsi(h, lut4, torch.from_numpy(cube).cuda()).cpu().numpy().astype(np.float64)
    eh, es, ei = O.hsi(cube, mode="exact")
    th = _circ(got[0], eh)
    d = np.sqrt(np.maximum(got[1] ** 2 + es ** 2 - 2 * got[1] * es * np.cos(th) + (got[2] - ei) ** 2, 0.0))
    ra, rm = O.cube_eps_hsi_lut(O.lut_build_hsi(33))
    assert abs(d.mean() - ra) <= 2e-6
    assert d.max() <= rm + 1e-3


def test_arguments_are_validated(h):
    lut4 = mact.mact_lut_build_hsi(h, 17)
    rgb = torch.zeros((10, 3), dtype=torch.uint8, device="cuda")
    out = torch.empty((3, 10), dtype=torch.float32, device="cuda")
    ptrs = (mact._VP * 3)(*(out[c].data_ptr() for c in range(3)))
    L, st = mact.lib(), mact._stream(None)
    assert L.mact_lut_interp_hsi(h.ptr, mact._VP(lut4.data_ptr() + 4), 17, mact._VP(rgb.data_ptr()), 10, ptrs,
                                 st) == mact.MACT_E_INVAL
    assert L.mact_lut_interp_hsi(h.ptr, mact._VP(lut4.data_ptr()), 65, mact._VP(rgb.data_ptr()), 10, ptrs,
                                 st) == mact.MACT_E_INVAL
    assert L.mact_lut_build_hsi(h.ptr, 1, mact._VP(lut4.data_ptr()), st) == mact.MACT_E_INVAL
