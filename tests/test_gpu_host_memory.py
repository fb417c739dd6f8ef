"""Host memory given straight to the kernels: pinned (and, where the device
walks the host page tables, pageable) input and output buffers are read and
written across the host link by the conversion kernels themselves.  Results
must be bit-identical to the device-memory path and within the oracle's
tolerances; unaddressable host memory must be rejected before any launch."""
import os

import numpy as np
import pytest
import torch

from paper_1009_0854_gb300 import mact, synth
from parity import check_space, oracle_planes

pytestmark = pytest.mark.gpu

SPACES = ("cielab", "hsi", "sct")


@pytest.fixture(scope="module")
def image():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return synth.gradient_noise_image(333, 517, seed=41)     # ragged: not a whole number of tiles


def _device_result(h, rgb_np, space, dtype):
    d = torch.from_numpy(rgb_np).cuda()
    out = mact.mact_convert(h, d, space, dtype=dtype)
    torch.cuda.synchronize()
    return out.cpu()


@pytest.mark.parametrize("exact", [0, 1])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
@pytest.mark.parametrize("space", SPACES)
def test_pinned_in_out_equals_device(image, space, dtype, exact):
    h = mact.mact_create(exact=exact)
    ref = _device_result(h, image, space, dtype)
    rgb = torch.from_numpy(image).pin_memory()
    out = torch.full((3,) + image.shape[:2], float("nan"), dtype=dtype).pin_memory()
    mact.mact_convert(h, rgb, space, out=out)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    if dtype == torch.float32:
        check_space(space, out, oracle_planes(space, image, exact=bool(exact)), dtype, "pinned")


@pytest.mark.parametrize("space", SPACES)
def test_pinned_pitched_views(image, space):
    """Row pitch wider than the row and output planes with padded rows, all in
    pinned memory: the guarded tile path on host memory."""
    H, W = image.shape[:2]
    h = mact.mact_create()
    ref = _device_result(h, image, space, torch.float32)
    big = torch.zeros((H, W + 7, 3), dtype=torch.uint8).pin_memory()
    big[:, :W] = torch.from_numpy(image)
    obig = torch.full((3, H, W + 5), -7.0, dtype=torch.float32).pin_memory()
    mact.mact_convert(h, big[:, :W], space, out=obig[:, :, :W])
    torch.cuda.synchronize()
    assert torch.equal(obig[:, :, :W], ref)
    assert bool((obig[:, :, W:] == -7.0).all())       # padding untouched


@pytest.mark.parametrize("n", [17, 33])
@pytest.mark.parametrize("method", ["trilinear", "prism", "pyramid", "tetra"])
def test_lut_interp_pinned(image, n, method):
    h = mact.mact_create()
    lut = mact.mact_lut_build(h, n)
    rgb_d = torch.from_numpy(image).cuda()
    ref, ref_sel = mact.mact_lut_interp(h, method, lut, rgb_d, sel=True)
    rgb = torch.from_numpy(image).pin_memory()
    npix = image.shape[0] * image.shape[1]
    out = torch.full((3, npix), float("nan"), dtype=torch.float32).pin_memory()
    got, sel = mact.mact_lut_interp(h, method, lut, rgb, out=out, sel=True)
    torch.cuda.synchronize()
    assert torch.equal(got, ref.cpu())
    assert torch.equal(sel.cpu(), ref_sel.cpu())


def test_batch_pinned_outputs():
    """The batched kernel with every input and output plane in pinned memory."""
    h = mact.mact_create()
    items = synth.batch_images(count=12, seed=23, lo=8, hi=600)
    dev = [(torch.from_numpy(im).cuda(), sp) for im, sp in items]
    ref = mact.mact_convert_batch(h, dev)
    host = [(torch.from_numpy(im).pin_memory(), sp) for im, sp in items]
    outs = [torch.full((3,) + im.shape[:2], float("nan"), dtype=torch.float32).pin_memory() for im, _ in items]
    mact.mact_convert_batch(h, host, outs=outs)
    torch.cuda.synchronize()
    for a, b in zip(outs, ref):
        assert torch.equal(a, b.cpu())


def test_pageable_when_device_walks_host_page_tables(image):
    h = mact.mact_create()
    if mact.mact_host_memory_access(h) != 1:
        pytest.skip("the device cannot address pageable host memory")
    ref = _device_result(h, image, "cielab", torch.float32)
    rgb = torch.from_numpy(image.copy())                       # pageable, every page written
    out = torch.zeros((3,) + image.shape[:2], dtype=torch.float32)
    mact.mact_convert(h, rgb, "cielab", out=out)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)


def test_checked_mode_rejects_unregistered_host_memory(image):
    """With the pointer check forced on, pageable host memory is refused
    before launch (nothing touches it) and pinned memory still works."""
    os.environ["MACT_CHECK_HOST_POINTERS"] = "1"
    try:
        h = mact.mact_create()
    finally:
        del os.environ["MACT_CHECK_HOST_POINTERS"]
    assert mact.mact_host_memory_access(h) == 0
    shape = (3,) + image.shape[:2]
    pageable_in = torch.from_numpy(image.copy())
    pinned_in = torch.from_numpy(image).pin_memory()
    sentinel = torch.full(shape, -3.0, dtype=torch.float32)
    with pytest.raises(mact.MactError) as ei:
        mact.mact_convert(h, pageable_in, "cielab", out=torch.empty(shape, dtype=torch.float32).pin_memory())
    assert ei.value.status == mact.MACT_E_INVAL
    with pytest.raises(mact.MactError) as ei:
        mact.mact_convert(h, pinned_in, "cielab", out=sentinel)
    assert ei.value.status == mact.MACT_E_INVAL
    assert bool((sentinel == -3.0).all())
    with pytest.raises(mact.MactError):
        mact.mact_lut_interp(h, "tetra", mact.mact_lut_build(h, 17), pageable_in)
    out = torch.empty(shape, dtype=torch.float32).pin_memory()
    mact.mact_convert(h, pinned_in, "cielab", out=out)
    torch.cuda.synchronize()
    assert torch.equal(out, _device_result(h, image, "cielab", torch.float32))
    # device memory passes the check too
    d_out = mact.mact_convert(h, torch.from_numpy(image).cuda(), "cielab")
    torch.cuda.synchronize()
    assert torch.equal(d_out.cpu(), out)
