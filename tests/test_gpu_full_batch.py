"""The batched form at its full size, in the launch configuration the
benchmark times: 256 uneven images (seed 0, sides log-uniform in [64, 4096],
273 Mpx, mixed spaces), launch shape picked by the autotuner, one work-list
plan replayed as a CUDA graph, FP32 and FP16 planes.  The oracle checks
sampled pixels of every image (random positions plus each image's first
pixel, last pixel and the end of its first row), within the parity
tolerances; a few images are also compared bit for bit with single-image
conversion."""
import numpy as np
import pytest
import torch

from paper_1009_0854_gb300 import mact, synth
from parity import check_space, oracle_planes

pytestmark = pytest.mark.gpu

SAMPLES = 2048


@pytest.fixture(scope="module")
def batch():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    specs = synth.batch_images(count=256, seed=0)
    return specs, [(torch.from_numpy(im).cuda(), space) for im, space in specs]


def _positions(rng, H, W):
    n = H * W
    idx = rng.integers(0, n, size=min(SAMPLES, n))
    return np.unique(np.concatenate([idx, [0, W - 1, n - 1]]))


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_full_batch_graph_replay_sampled(batch, dtype):
    specs, imgs = batch
    assert sum(im.shape[0] * im.shape[1] for im, _ in specs) > 2.7e8
    h = mact.mact_create()
    outs = [torch.full((3,) + tuple(r.shape[:2]), float("nan"), dtype=dtype, device="cuda") for r, _ in imgs]
    mact.mact_autotune_batch(h, imgs, outs=outs, reps=1)
    for o in outs:
        o.fill_(float("nan"))
    plan, _ = mact.mact_batch_plan_create(h, imgs, outs=outs)
    plan.graph_launch()
    plan.graph_launch()              # a replay rewrites the same values
    torch.cuda.synchronize()
    rng = np.random.default_rng(1234)
    for i, ((im, space), o) in enumerate(zip(specs, outs)):
        H, W = im.shape[:2]
        pos = _positions(rng, H, W)
        got = o.view(3, -1)[:, torch.from_numpy(pos).cuda()]
        ref = oracle_planes(space, im.reshape(-1, 3)[pos])
        check_space(space, got, ref, dtype, "image %d (%dx%d %s)" % (i, H, W, space))
    for k in (0, 1, 127, 255):
        rgb, space = imgs[k]
        single = mact.mact_convert(h, rgb, space, dtype=dtype)
        torch.cuda.synchronize()
        assert torch.equal(single, outs[k]), k
    plan.close()
