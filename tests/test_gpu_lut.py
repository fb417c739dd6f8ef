"""GPU parity of the LUT packing and the four interpolators against the
oracle: selection (cell and simplex) bit-identical, values within 2e-4."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1009_0854_gb300 import mact
from parity import LAB_TOL, to_np

pytestmark = pytest.mark.gpu

METHODS = ["trilinear", "prism", "pyramid", "tetra"]


@pytest.fixture(scope="module")
def h():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return mact.mact_create()


_LUT = {}


def oracle_lut(N):
    if N not in _LUT:
        _LUT[N] = O.lut_build(N)
    return _LUT[N]


@pytest.mark.parametrize("N", [2, 9, 17, 33, 64])
def test_lut_build_matches_oracle(h, N):
    """Packing on the GPU (FP64 then rounded) equals the oracle's FP32 LUT to
    one FP32 ulp (plus 1e-12 where the value is 0 up to cancellation)."""
    g = mact.mact_lut_build(h, N).cpu().numpy()
    ref = oracle_lut(N) if N != 64 else O.lut_build(64)
    d = np.abs(g.astype(np.float64) - ref.astype(np.float64))
    assert np.all(d <= np.spacing(np.abs(ref)).astype(np.float64) + 1e-12)


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("N", [9, 17, 33])
def test_interp_full_cube(h, cube_rgb, method, N):
    """Every 24-bit colour, the oracle-built LUT fed to both sides."""
    lut = oracle_lut(N)
    rgb = cube_rgb.reshape(-1, 3)
    out, sel = mact.mact_lut_interp(h, method, torch.from_numpy(lut).cuda(),
                                    torch.from_numpy(rgb).cuda(), sel=True)
    torch.cuda.synchronize()
    ref, rsel = O.lut_interp(method, lut, rgb)
    assert np.array_equal(sel.cpu().numpy(), rsel)
    for c in range(3):
        d = np.abs(to_np(out[c]) - ref[c])
        assert d.max() <= LAB_TOL, (method, N, c, d.max())


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("N", [2, 5, 18, 40, 64])
def test_interp_other_sizes_and_ragged(h, method, N):
    rng = np.random.default_rng(N)
    lut = rng.normal(scale=50.0, size=(N, N, N, 3)).astype(np.float32)
    for npix in (1, 7, 2047, 4099):
        rgb = rng.integers(0, 256, size=(npix, 3), dtype=np.uint8)
        rgb[0] = (255, 255, 255)
        out, sel = mact.mact_lut_interp(h, method, torch.from_numpy(lut).cuda(), torch.from_numpy(rgb).cuda(),
                                        sel=True)
        torch.cuda.synchronize()
        ref, rsel = O.lut_interp(method, lut, rgb)
        assert np.array_equal(sel.cpu().numpy(), rsel)
        for c in range(3):
            assert np.abs(to_np(out[c]) - ref[c]).max() <= LAB_TOL


def test_interp_without_selection_output(h, cube_rgb):
    lut = oracle_lut(17)
    rgb = torch.from_numpy(cube_rgb.reshape(-1, 3)[:100000].copy()).cuda()
    a = mact.mact_lut_interp(h, "tetra", torch.from_numpy(lut).cuda(), rgb)
    b, _ = mact.mact_lut_interp(h, "tetra", torch.from_numpy(lut).cuda(), rgb, sel=True)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
