"""GPU parity of the CIELUV variant (CIE 1976 L*u*v*, which the paper's
Conclusions say the method carries over to): the kernels against the FP64
oracle over the whole 2^24 cube, in FP32 and FP16 planes, for the printed
(4,4) cube-root rational, the exact form, the library's fitted (6,6) and the
FP64 polynomial option, in single-image, batched and served calls.
Tolerance: 2e-4 per component, as for CIELAB (tests/parity.py)."""
import numpy as np
import pytest
import torch

from paper_1009_0854_gb300 import mact, synth
from parity import check_space, oracle_planes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch.device("cuda", 0)


@pytest.mark.parametrize("exact", [False, True])
def test_full_cube(dev, cube_rgb, exact):
    h = mact.mact_create(exact=int(exact))
    out = mact.mact_convert(h, torch.from_numpy(cube_rgb).to(dev), "cieluv")
    torch.cuda.synchronize()
    check_space("cieluv", out, oracle_planes("cieluv", cube_rgb.reshape(-1, 3), exact=exact),
                what="cube cieluv exact=%s" % exact)
    h.close()


@pytest.mark.parametrize("exact", [False, True])
def test_fp16_planes(dev, exact):
    img = synth.gradient_noise_image(512, 512, seed=0)
    h = mact.mact_create(exact=int(exact))
    out = mact.mact_convert(h, torch.from_numpy(img).to(dev), "cieluv", dtype=torch.float16)
    torch.cuda.synchronize()
    check_space("cieluv", out, oracle_planes("cieluv", img, exact=exact), dtype=torch.float16, what="fp16")
    h.close()


def test_polynomial_cube_root_option(dev):
    """lab_m = 0 (Table tab_cbrt_poly n = 5, evaluated in FP64 on the device)."""
    img = synth.gradient_noise_image(256, 384, seed=3)
    h = mact.mact_create(lab_n=5, lab_m=0)
    out = mact.mact_convert(h, torch.from_numpy(img).to(dev), "cieluv")
    torch.cuda.synchronize()
    check_space("cieluv", out, oracle_planes("cieluv", img, cfg={"lab_n": 5, "lab_m": 0}), what="poly")
    h.close()


def test_white_black_and_grays(dev):
    v = np.arange(256, dtype=np.uint8)
    grays = np.stack([v, v, v], axis=1)[None]
    h = mact.mact_create()
    L, U, V = (x.cpu().numpy() for x in mact.mact_convert(h, torch.from_numpy(grays).to(dev), "cieluv"))
    assert L[0, 0] == 0.0 and U[0, 0] == 0.0 and V[0, 0] == 0.0
    assert np.abs(U).max() < 2e-4 and np.abs(V).max() < 2e-4
    assert np.all(np.diff(L[0]) > 0)
    h.close()


def test_batched_and_served_mix(dev):
    """CIELUV images in one batched launch and through the server, mixed with
    the other spaces, FP32 and FP16: each matches the oracle."""
    specs = synth.batch_images(count=24, seed=12, lo=16, hi=600)
    spaces = ["cieluv" if i % 2 == 0 else sp for i, (_, sp) in enumerate(specs)]
    imgs = [(torch.from_numpy(im).to(dev), sp) for (im, _), sp in zip(specs, spaces)]
    dts = [torch.float16 if i % 3 == 1 else torch.float32 for i in range(len(imgs))]
    outs = [torch.empty((3,) + tuple(r.shape[:2]), dtype=dt, device=dev) for (r, _), dt in zip(imgs, dts)]
    h = mact.mact_create()
    got = mact.mact_convert_batch(h, imgs, outs=outs)
    torch.cuda.synchronize()
    srv = mact.mact_serve_create(h, 256 << 20, max_slots=8)
    pend = [mact.mact_serve_submit(srv, torch.from_numpy(im).pin_memory(), sp, dtype=dt)
            for (im, _), sp, dt in zip(specs, spaces, dts)]
    for (im, _), sp, dt, g, (t, o) in zip(specs, spaces, dts, got, pend):
        ref = oracle_planes(sp, im)
        check_space(sp, g, ref, dtype=dt, what="batch %s" % sp)
        mact.mact_serve_wait(srv, t, 60000)
        check_space(sp, o, ref, dtype=dt, what="served %s" % sp)
    srv.close()
    h.close()
