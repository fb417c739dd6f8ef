"""Memory layouts and the three tile paths of the conversion engine.

Full tiles with 16-byte aligned input and outputs take the vector path; full
tiles whose output planes are aligned only to their element size (three
adjacent planes of H*W elements, H*W not a multiple of 4, or of 8 for FP16)
take the shifted path (warp transpose through shared memory); everything else
(partial tiles, byte-offset pointers) takes the guarded path or its shifted
variant.  Whatever the path, each pixel's value must be bit-identical to the
same conversion into separately allocated, 16-byte aligned planes, which the
parity tests tie to the oracle.  Output planes must be aligned to their
element size; others are refused on the host before any launch."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1009_0854_gb300 import mact, synth
from parity import check_space, oracle_planes

pytestmark = pytest.mark.gpu

SPACES = ("cielab", "hsi", "sct")


@pytest.fixture(scope="module")
def handles():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return {0: mact.mact_create(), 1: mact.mact_create(exact=1)}


def _aligned_reference(h, rgb, space, dtype):
    """Each plane in its own allocation (256-byte aligned)."""
    H, W = rgb.shape[:2]
    planes = [torch.empty((H, W), dtype=dtype, device="cuda") for _ in range(3)]
    img = mact._image(rgb, space, torch.empty((3, H, W), dtype=dtype, device="cuda"))
    for c in range(3):
        img.out[c] = planes[c].data_ptr()
    mact._check(mact.lib().mact_convert(h.ptr, ctypes.byref(img), mact._stream(None)), "mact_convert")
    torch.cuda.synchronize()
    return torch.stack(planes)


# (H, W) with H*W mod 8 covering 1..7, tile-boundary sizes (4096 px tiles),
# one warp's 128 pixels, a single pixel
SHAPES = [(33, 31), (37, 62), (41, 41), (52, 61), (45, 89), (47, 90), (51, 93), (64, 64),
          (34, 33), (53, 55), (146, 157), (151, 157),
          (1, 4095), (1, 4096), (1, 4097), (3, 2731), (1, 127), (1, 129), (1, 1), (509, 1021)]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
@pytest.mark.parametrize("space", SPACES)
@pytest.mark.parametrize("exact", [0, 1])
def test_adjacent_planes_any_size(handles, space, dtype, exact):
    h = handles[exact]
    for k, (H, W) in enumerate(SHAPES):
        im = synth.gradient_noise_image(H, W, seed=100 + k)
        rgb = torch.from_numpy(im).cuda()
        got = mact.mact_convert(h, rgb, space, dtype=dtype)     # adjacent planes
        ref = _aligned_reference(h, rgb, space, dtype)
        assert torch.equal(got, ref), (H, W)
        if dtype == torch.float32 and k % 5 == 0:
            check_space(space, got, oracle_planes(space, im, exact=bool(exact)), dtype, "%dx%d" % (H, W))


def _raw_image(rgb_ptr, H, W, pitch, space, dtype, outs, opitch):
    img = mact.Image()
    img.rgb = rgb_ptr
    img.width, img.height, img.pitch_bytes = W, H, pitch
    img.space = mact.SPACES[space]
    img.dtype = mact.DTYPES[dtype]
    for c in range(3):
        img.out[c] = outs[c]
    img.out_pitch_elems = opitch
    return img


@pytest.mark.parametrize("space", SPACES)
@pytest.mark.parametrize("in_off,out_off", [(1, 0), (0, 4), (3, 8), (5, 12), (16, 4)])
def test_offset_pointers(handles, space, in_off, out_off):
    """Input at any byte offset, output planes at any FP32-element offset
    (not 16-byte aligned): the guarded and shifted paths."""
    h = handles[0]
    H, W = 37, 301
    im = synth.gradient_noise_image(H, W, seed=7)
    raw_in = torch.zeros(H * W * 3 + 64, dtype=torch.uint8, device="cuda")
    raw_in[in_off: in_off + H * W * 3] = torch.from_numpy(im.reshape(-1)).cuda()
    nbytes = H * W * 4
    raw_out = torch.zeros(3 * (nbytes + 64), dtype=torch.uint8, device="cuda")
    outs = [raw_out.data_ptr() + c * (nbytes + 64) + out_off for c in range(3)]
    img = _raw_image(raw_in.data_ptr() + in_off, H, W, 3 * W, space, torch.float32, outs, W)
    mact._check(mact.lib().mact_convert(h.ptr, ctypes.byref(img), mact._stream(None)), "mact_convert")
    torch.cuda.synchronize()
    ref = _aligned_reference(h, torch.from_numpy(im).cuda(), space, torch.float32).cpu()
    for c in range(3):
        b = raw_out[c * (nbytes + 64) + out_off: c * (nbytes + 64) + out_off + nbytes].cpu()
        assert torch.equal(b.view(torch.float32).view(H, W), ref[c])


@pytest.mark.parametrize("dtype,off", [(torch.float32, 1), (torch.float32, 2), (torch.float32, 3),
                                       (torch.float16, 1)])
def test_output_not_element_aligned_is_rejected(handles, dtype, off):
    """An output plane that is not aligned to its element size is refused on
    the host before any launch (MACT_E_INVAL); nothing is written."""
    h = handles[0]
    H, W = 8, 40
    rgb = torch.zeros((H, W, 3), dtype=torch.uint8, device="cuda")
    esz = 4 if dtype == torch.float32 else 2
    raw_out = torch.full((3 * (H * W * esz + 64),), 0x5A, dtype=torch.uint8, device="cuda")
    outs = [raw_out.data_ptr() + c * (H * W * esz + 64) + (off if c == 1 else 0) for c in range(3)]
    img = _raw_image(rgb.data_ptr(), H, W, 3 * W, "cielab", dtype, outs, W)
    st = mact.lib().mact_convert(h.ptr, ctypes.byref(img), mact._stream(None))
    assert st == mact.MACT_E_INVAL
    torch.cuda.synchronize()
    assert bool((raw_out == 0x5A).all())


@pytest.mark.parametrize("space", SPACES)
def test_pinned_host_adjacent_planes(handles, space):
    """The serving layout: pinned host input and adjacent, element-aligned
    host planes, written in place by the kernel."""
    h = handles[0]
    for H, W in [(45, 89), (511, 1023), (1, 4097)]:
        im = synth.gradient_noise_image(H, W, seed=H)
        ref = _aligned_reference(h, torch.from_numpy(im).cuda(), space, torch.float32).cpu()
        out = torch.full((3, H, W), float("nan")).pin_memory()
        mact.mact_convert(h, torch.from_numpy(im).pin_memory(), space, out=out)
        torch.cuda.synchronize()
        assert torch.equal(out, ref), (H, W)


def test_batch_with_misaligned_planes(handles):
    """The batched kernel's shifted and tail paths, in one launch with both
    list forms (by value and in device memory)."""
    h = handles[0]
    imgs = [(torch.from_numpy(synth.gradient_noise_image(H, W, seed=H * W)).cuda(), SPACES[k % 3])
            for k, (H, W) in enumerate(SHAPES)]
    for lst in (imgs, imgs * 3):             # 16 images, then 48 (device work list)
        outs = mact.mact_convert_batch(h, lst)
        torch.cuda.synchronize()
        for (rgb, space), o in zip(lst, outs):
            assert torch.equal(o, _aligned_reference(h, rgb, space, torch.float32))
