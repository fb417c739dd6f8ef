"""GPU parity: the CUDA kernels of libmact.so, called through the C ABI,
against the FP64 oracle, element by element on seeded inputs."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import tables
from paper_1009_0854_gb300 import mact, synth
from parity import LAB_TOL, check_space, oracle_planes

pytestmark = pytest.mark.gpu

SPACES = ["cielab", "hsi", "sct"]


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch.device("cuda", 0)


_HANDLES = {}


def handle(**kw):
    key = tuple(sorted(kw.items()))
    if key not in _HANDLES:
        _HANDLES[key] = mact.mact_create(**kw)
    return _HANDLES[key]


@pytest.fixture(scope="module")
def c1():
    """512 x 512 gradient + noise image, seed 0."""
    return synth.gradient_noise_image(512, 512, seed=0)


@pytest.mark.parametrize("space", SPACES)
@pytest.mark.parametrize("exact", [False, True])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_c1_image(dev, c1, space, exact, dtype):
    h = handle(exact=int(exact))
    out = mact.mact_convert(h, torch.from_numpy(c1).to(dev), space, dtype=dtype)
    torch.cuda.synchronize()
    check_space(space, out, oracle_planes(space, c1, exact=exact), dtype=dtype, what="%s exact=%s" % (space, exact))


@pytest.mark.parametrize("space", SPACES)
@pytest.mark.parametrize("exact", [False, True])
def test_full_cube(dev, cube_rgb, space, exact):
    """All 2^24 colours, lexicographic, one 4096 x 4096 image."""
    h = handle(exact=int(exact))
    out = mact.mact_convert(h, torch.from_numpy(cube_rgb).to(dev), space)
    torch.cuda.synchronize()
    check_space(space, out, oracle_planes(space, cube_rgb.reshape(-1, 3), exact=exact),
                what="cube %s exact=%s" % (space, exact))


@pytest.mark.parametrize("nm", sorted(tables.CBRT_RAT) + [(n, 0) for n in sorted(tables.CBRT_POLY)],
                         ids=lambda nm: "n%d_m%d" % nm)
def test_cielab_every_degree(dev, c1, nm):
    h = handle(lab_n=nm[0], lab_m=nm[1])
    out = mact.mact_convert(h, torch.from_numpy(c1).to(dev), "cielab")
    torch.cuda.synchronize()
    check_space("cielab", out, O.cielab(c1, n=nm[0], m=nm[1]), what="lab %s" % (nm,))


@pytest.mark.parametrize("n", [2, 3, 4, 5])
@pytest.mark.parametrize("printed", [0, 1])
def test_hsi_every_degree(dev, cube_rgb, n, printed):
    """Every degree and both coefficient sets.  The library fits [0,1] with
    its own Remez exchange, the oracle with its own: parity checks both."""
    h = handle(hsi_n=n, hsi_coeffs=printed)
    rgb = cube_rgb.reshape(-1, 3)[::7].copy()
    out = mact.mact_convert(h, torch.from_numpy(rgb.reshape(1, -1, 3)).to(dev), "hsi")
    torch.cuda.synchronize()
    check_space("hsi", out, O.hsi(rgb, n=n, printed=bool(printed)), what="hsi n=%d printed=%d" % (n, printed))


@pytest.mark.parametrize("nmr", [(4, 4, 4), (4, 5, 4), (5, 4, 4), (5, 5, 4), (4, 4, 5), (4, 5, 5), (5, 4, 5)])
def test_sct_every_degree(dev, cube_rgb, nmr):
    h = handle(sct_n=nmr[0], sct_m=nmr[1], sct_r=nmr[2])
    rgb = cube_rgb.reshape(-1, 3)[::5].copy()
    out = mact.mact_convert(h, torch.from_numpy(rgb.reshape(1, -1, 3)).to(dev), "sct")
    torch.cuda.synchronize()
    check_space("sct", out, O.sct(rgb, n=nmr[0], m=nmr[1], r=nmr[2]), what="sct %s" % (nmr,))


@pytest.mark.parametrize("hw", [(1, 1), (3, 5), (7, 1023), (2, 1025), (31, 33), (1, 4097), (129, 3)])
@pytest.mark.parametrize("space", SPACES)
def test_ragged_sizes(dev, hw, space):
    rng = np.random.default_rng(hw[0] * 10007 + hw[1])
    img = rng.integers(0, 256, size=(hw[0], hw[1], 3), dtype=np.uint8)
    h = handle()
    for dtype in (torch.float32, torch.float16):
        out = mact.mact_convert(h, torch.from_numpy(img).to(dev), space, dtype=dtype)
        torch.cuda.synchronize()
        check_space(space, out, oracle_planes(space, img), dtype=dtype, what="%s %s" % (space, hw))


@pytest.mark.parametrize("space", SPACES)
def test_pitched_and_misaligned(dev, space):
    """Rows with padding on both sides and pointers off the 16-byte grid take
    the tail path; results must not change."""
    rng = np.random.default_rng(99)
    H, W = 37, 1500
    big = torch.from_numpy(rng.integers(0, 256, size=(H, W + 7, 3), dtype=np.uint8)).to(dev)
    view = big[:, 1:W + 1, :]                      # pitch 3*(W+7), base offset 3 bytes
    out_big = torch.full((3, H, W + 5), float("nan"), device=dev)
    out = out_big[:, :, 1:W + 1]                   # out pitch W+5, offset 4 bytes
    h = handle()
    mact.mact_convert(h, view, space, out=out)
    torch.cuda.synchronize()
    ref = oracle_planes(space, view.cpu().numpy())
    check_space(space, out, ref, what="pitched %s" % space)
    assert torch.isnan(out_big[:, :, 0]).all() and torch.isnan(out_big[:, :, W + 1:]).all()


def test_empty_image_is_a_no_op(dev):
    h = handle()
    out = mact.mact_convert(h, torch.empty((0, 5, 3), dtype=torch.uint8, device=dev), "cielab")
    assert out.shape == (3, 0, 5)


def test_closed_forms_on_gpu(dev):
    """Grays have equal t values in exact arithmetic, so a* = b* = 0; in FP32
    the three matrix rows round differently, so they are 0 to within the
    parity tolerance (one FP32 ulp of f is 6e-5 in a*); exact white ->
    (100, 0, 0); gray hue and saturation are exactly 0."""
    v = torch.arange(256, dtype=torch.uint8, device=dev)
    grays = torch.stack([v, v, v], dim=1).reshape(1, 256, 3)
    for exact in (0, 1):
        out = mact.mact_convert(handle(exact=exact), grays, "cielab")
        torch.cuda.synchronize()
        assert out[1].abs().max().item() <= LAB_TOL and out[2].abs().max().item() <= LAB_TOL
        if exact:
            assert abs(out[0, 0, 255].item() - 100.0) < 2e-4
        hsi = mact.mact_convert(handle(exact=exact), grays, "hsi")
        assert (hsi[0] == 0).all() and (hsi[1] == 0).all()


@pytest.mark.parametrize("space", SPACES)
def test_batch_equals_single(dev, space):
    """One persistent launch over uneven images == per-image launches,
    bit for bit (same kernel body, same tiles)."""
    specs = synth.batch_images(count=24, seed=5, lo=16, hi=700)
    h = handle()
    imgs = [(torch.from_numpy(im).to(dev), space) for im, _ in specs]
    outs = mact.mact_convert_batch(h, imgs)
    singles = [mact.mact_convert(h, r, space) for r, _ in imgs]
    torch.cuda.synchronize()
    for a, b in zip(outs, singles):
        assert torch.equal(a, b)


def test_batch_mixed_spaces_and_dtypes(dev):
    specs = synth.batch_images(count=40, seed=11, lo=8, hi=900)
    h = handle()
    imgs, outs = [], []
    for i, (im, space) in enumerate(specs):
        r = torch.from_numpy(im).to(dev)
        dt = torch.float16 if i % 3 == 0 else torch.float32
        imgs.append((r, space))
        outs.append(torch.empty((3,) + im.shape[:2], dtype=dt, device=dev))
    mact.mact_convert_batch(h, imgs, outs=outs)
    # a second launch reuses the work list and counters
    outs2 = [torch.empty_like(o) for o in outs]
    mact.mact_convert_batch(h, imgs, outs=outs2)
    torch.cuda.synchronize()
    for (im, space), o, o2 in zip(specs, outs, outs2):
        check_space(space, o, oracle_planes(space, im), dtype=o.dtype, what="batch %s %s" % (space, im.shape))
        assert torch.equal(o, o2)


def test_batch_empty(dev):
    h = handle()
    assert mact.mact_convert_batch(h, []) == []
