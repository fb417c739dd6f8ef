"""The batched form for repeated lists: plans, CUDA-graph replay, every
launch shape of the batched kernel, and the autotuner."""
import numpy as np
import pytest
import torch

from paper_1009_0854_gb300 import mact, synth
from parity import check_space, oracle_planes

pytestmark = pytest.mark.gpu

SHAPES = [(128, 16), (256, 16), (512, 16), (256, 32), (128, 32)]


@pytest.fixture(scope="module")
def imgs():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return [(torch.from_numpy(im).cuda(), space) for im, space in synth.batch_images(count=30, seed=17, lo=8, hi=800)]


def test_plan_and_graph_equal_convert_batch(imgs):
    h = mact.mact_create()
    ref = mact.mact_convert_batch(h, imgs)
    plan, outs = mact.mact_batch_plan_create(h, imgs)
    plan.launch()
    torch.cuda.synchronize()
    for a, b in zip(outs, ref):
        assert torch.equal(a, b)
    for o in outs:
        o.fill_(float("nan"))
    plan.graph_launch()
    plan.graph_launch()          # replay: counters reset themselves
    torch.cuda.synchronize()
    for a, b in zip(outs, ref):
        assert torch.equal(a, b)
    plan.close()


def test_graph_replay_sees_new_contents(imgs):
    """Same addresses, new pixel values: a replay converts the new values."""
    h = mact.mact_create()
    src = [(r.clone(), s) for r, s in imgs[:8]]
    plan, outs = mact.mact_batch_plan_create(h, src)
    plan.graph_launch()
    for (r, _), (r0, _) in zip(src, imgs[:8]):
        r.copy_(255 - r0)
    plan.graph_launch()
    torch.cuda.synchronize()
    for (r, space), o in zip(src, outs):
        check_space(space, o, oracle_planes(space, r.cpu().numpy()), what="replay %s" % space)
    plan.close()


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "t%d_px%d" % s)
def test_every_launch_shape_gives_identical_results(imgs, shape):
    h = mact.mact_create()
    ref = mact.mact_convert_batch(h, imgs)
    mact.mact_set_batch_shape(h, shape[0], shape[1], 0)
    assert mact.mact_get_batch_shape(h) == (shape[0], shape[1], 0)
    got = mact.mact_convert_batch(h, imgs)
    torch.cuda.synchronize()
    for a, b in zip(got, ref):
        assert torch.equal(a, b)


def test_autotuner_picks_a_timed_shape(imgs):
    h = mact.mact_create()
    table, chosen = mact.mact_autotune_batch(h, imgs, reps=3)
    assert len(table) >= len(SHAPES)
    best = min(table, key=lambda r: r["ms"])
    assert (chosen[0], chosen[1]) == (best["threads"], best["px_per_thread"])
    assert all(r["ms"] > 0 for r in table)
    ref = mact.mact_convert_batch(mact.mact_create(), imgs)
    got = mact.mact_convert_batch(h, imgs)
    torch.cuda.synchronize()
    for a, b in zip(got, ref):
        assert torch.equal(a, b)


def test_unsupported_shape_rejected():
    h = mact.mact_create()
    with pytest.raises(mact.MactError) as e:
        mact.mact_set_batch_shape(h, 96, 16, 0)
    assert e.value.status == -4


def test_short_list_by_value_equals_device_list(imgs):
    """Up to 32 non-empty images travel in the kernel parameters, more go
    through the device work list: both give each image's mact_convert result,
    bit for bit, with empty images anywhere in the list."""
    h = mact.mact_create()
    empty = (torch.empty((0, 7, 3), dtype=torch.uint8, device="cuda"), "hsi")
    more = imgs + imgs[:3]                                  # 33 non-empty
    short = [empty] + more[:16] + [empty] + more[16:32]     # 32 non-empty + 2 empty
    out_short = mact.mact_convert_batch(h, short)
    out_long = mact.mact_convert_batch(h, more)
    torch.cuda.synchronize()
    got_short = [o for (r, _), o in zip(short, out_short) if r.shape[0] != 0]
    assert len(got_short) == 32
    for k, (rgb, space) in enumerate(more):
        ref = mact.mact_convert(h, rgb, space)
        torch.cuda.synchronize()
        assert torch.equal(out_long[k], ref), k
        if k < 32:
            assert torch.equal(got_short[k], ref), k
    outs = mact.mact_convert_batch(h, [empty, empty])       # nothing to launch
    assert [tuple(o.shape) for o in outs] == [(3, 0, 7)] * 2


@pytest.mark.parametrize("px_per_thread,threads", [(16, 128), (16, 512), (32, 256)])
def test_short_list_every_shape(imgs, px_per_thread, threads):
    h = mact.mact_create()
    mact.mact_set_batch_shape(h, threads, px_per_thread, 0)
    few = imgs[:5]
    outs = mact.mact_convert_batch(h, few)
    torch.cuda.synchronize()
    for (rgb, space), o in zip(few, outs):
        assert torch.equal(o, mact.mact_convert(h, rgb, space))
