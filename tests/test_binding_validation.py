"""The Python binding refuses caller-supplied tensors whose size, type or
layout differ from what the kernels read or write.  The C ABI takes plain
pointers and cannot see buffer sizes, so a short output or gradient buffer
would otherwise be overrun on the device; the binding checks every such
tensor before it calls into the library (no GPU and no handle needed)."""
import pytest
import torch

from paper_1009_0854_gb300 import mact

H, W = 4, 6
NPIX = H * W


def rgb():
    return torch.zeros((H, W, 3), dtype=torch.uint8)


def lut(n=5, c=3):
    return torch.zeros((n, n, n, c), dtype=torch.float32)


def test_convert_output_dtype_and_shape():
    with pytest.raises(ValueError, match="float32 or float16"):
        mact.mact_convert(None, rgb(), "cielab", out=torch.zeros((3, H, W), dtype=torch.float64))
    with pytest.raises(ValueError, match="shape"):
        mact.mact_convert(None, rgb(), "cielab", out=torch.zeros((3, H, W - 1)))


def test_batch_needs_one_output_per_image():
    imgs = [(rgb(), "cielab"), (rgb(), "hsi")]
    outs = [torch.zeros((3, H, W))]
    for fn in (mact.mact_convert_batch, mact.mact_convert_batch_static):
        with pytest.raises(ValueError, match="one output per image"):
            fn(None, imgs, outs=outs)
    with pytest.raises(ValueError, match="one output per image"):
        mact.mact_batch_plan_create(None, imgs, outs=outs)


@pytest.mark.parametrize("shape,dtype", [((4, 4, 4, 3), torch.float32), ((5, 5, 5, 4), torch.float32),
                                         ((5, 5, 5, 3), torch.float64)])
def test_lut_build_output(shape, dtype):
    with pytest.raises(ValueError, match="out"):
        mact.mact_lut_build(None, 5, out=torch.zeros(shape, dtype=dtype))


def test_lut_build_hsi_output():
    with pytest.raises(ValueError, match="out"):
        mact.mact_lut_build_hsi(None, 5, out=lut(5, 3))


@pytest.mark.parametrize("out", [torch.zeros((3, NPIX - 1)), torch.zeros((3, NPIX), dtype=torch.float16),
                                 torch.zeros((NPIX, 3)).t()])
def test_lut_interp_output(out):
    with pytest.raises(ValueError, match="out"):
        mact.mact_lut_interp(None, "trilinear", lut(), rgb(), out=out)
    with pytest.raises(ValueError, match="out"):
        mact.mact_lut_interp_hsi(None, lut(5, 4), rgb(), out=out)


def test_lut_must_be_a_cube():
    bad = torch.zeros((5, 5, 4, 3), dtype=torch.float32)
    with pytest.raises(ValueError, match="cube"):
        mact.mact_lut_interp(None, "trilinear", bad, rgb())
    with pytest.raises(ValueError, match="lut"):
        mact.mact_cube_error_lut(None, "trilinear", bad)
    with pytest.raises(ValueError, match="cube"):
        mact.mact_lut_interp_hsi(None, torch.zeros((5, 4, 5, 4)), rgb())


def test_caching_layout_buffers():
    n = 5
    with pytest.raises(ValueError, match="out"):
        mact.mact_lut_cache_build(None, lut(n), out=torch.zeros(((n - 1) ** 3 - 1, 8, 4)))
    with pytest.raises(ValueError, match="cache"):
        mact.mact_lut_interp_cached(None, "trilinear", torch.zeros(((n - 1) ** 3, 8, 3)), n, rgb())
    with pytest.raises(ValueError, match="out"):
        mact.mact_lut_interp_cached(None, "trilinear", torch.zeros(((n - 1) ** 3, 8, 4)), n, rgb(),
                                    out=torch.zeros((3, NPIX + 1)))


def test_gradient_buffers():
    x = torch.zeros((2, 3, H, W))
    for bad in (torch.zeros((2, 3, H, W - 1)), torch.zeros((1, 3, H, W)), torch.zeros((2, 3, H, W), dtype=torch.float64)):
        with pytest.raises(ValueError):
            mact.mact_lab_backward(None, x, bad)
        with pytest.raises(ValueError):
            mact.mact_lab_forward(None, x, out=bad)
        with pytest.raises(ValueError):
            mact.mact_lab_delta_e_loss(None, x, bad)
        with pytest.raises(ValueError):
            mact.mact_lab_delta_e_loss(None, x, torch.zeros_like(x), grad_out=bad)
    with pytest.raises(ValueError, match="loss"):
        mact.mact_lab_delta_e_loss(None, x, torch.zeros_like(x), loss=torch.zeros(1))
    with pytest.raises(TypeError):
        mact.mact_lab_backward(None, x, None)
