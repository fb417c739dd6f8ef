"""The paper's error tables recomputed on the GPU (production FP32 kernels
against an FP64 exact transform on the device, every 24-bit colour) and
compared with the oracle's FP64 statistics and the printed values."""
import pytest
import torch

import oracle as O
from conftest import read_golden
from paper_1009_0854_gb300 import mact

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"


@pytest.mark.parametrize("row", read_golden("tab_cielab.txt"), ids=lambda r: "n%s_m%s" % (r[0], r[1]))
def test_tab_cielab_on_gpu(dev, row):
    """The FP32 kernel's own rounding (<= 2e-4 per Lab component) may move
    Delta E by at most 3.5e-4 per colour."""
    n, m = int(row[0]), int(row[1])
    a, b = mact.mact_cube_error(mact.mact_create(lab_n=n, lab_m=m), "cielab")
    ra, rb = O.cube_eps_cielab(n, m)
    assert abs(a - ra) <= 2e-5 and abs(b - rb) <= 3.5e-4
    assert a == pytest.approx(float(row[2]), rel=2e-3)
    assert b == pytest.approx(float(row[3]), rel=2e-3)


def test_exact_cielab_error_is_rounding_only(dev):
    a, b = mact.mact_cube_error(mact.mact_create(exact=1), "cielab")
    assert a < 2e-5 and b < 3.5e-4


@pytest.mark.parametrize("row", read_golden("tab_hsi.txt"), ids=lambda r: "n%s" % r[0])
def test_tab_hsi_on_gpu(dev, row):
    n = int(row[0])
    a, b = mact.mact_cube_error(mact.mact_create(hsi_n=n), "hsi")
    ra, rb = O.cube_eps_hsi(n)
    assert abs(a - ra) <= 1e-6 and abs(b - rb) <= 2e-6
    assert abs(b - float(row[2])) <= 2e-6


@pytest.mark.parametrize("row", read_golden("tab_sct.txt"), ids=lambda r: "n%s_m%s_r%s" % tuple(r[:3]))
def test_tab_sct_on_gpu(dev, row):
    n, m, r = (int(v) for v in row[:3])
    a, b = mact.mact_cube_error(mact.mact_create(sct_n=n, sct_m=m, sct_r=r), "sct")
    ra, rb = O.cube_eps_sct(n, m, r)
    assert abs(a - ra) <= 1e-5 and abs(b - rb) <= 2e-4
    assert abs(a - float(row[3])) <= 1e-5


_LUT = {}


@pytest.mark.parametrize("row", read_golden("tab_lut.txt"), ids=lambda r: "%s_%s" % (r[0], r[1]))
def test_tab_lut_on_gpu(dev, row):
    meth, N = row[0], int(row[1])
    if N not in _LUT:
        _LUT[N] = O.lut_build(N)
    lut = _LUT[N]
    a, b = mact.mact_cube_error_lut(mact.mact_create(), meth, torch.from_numpy(lut).cuda())
    ra, rb = O.cube_eps_lut(meth, lut)
    assert abs(a - ra) <= 2e-5 and abs(b - rb) <= 3.5e-4
    assert abs(b - float(row[3])) <= 3.5e-4
