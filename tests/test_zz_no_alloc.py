"""The batched entry point that allocates nothing (mact_convert_batch_static)
against the allocating one (mact_convert_batch), through the C ABI.

It exists for callers that cannot allocate at call time, so it keeps its
work list in a fixed device array; these checks make sure that array gives
the same results as the allocating path on consecutive calls, that a stale
work list from the previous call never leaks into the next one, and that an
oversized request is refused.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1009_0854_gb300 import mact, synth
from parity import check_space, to_np

pytestmark = pytest.mark.gpu


def _images(seed, count):
    specs = synth.batch_images(count=count, seed=seed, lo=8, hi=700)
    imgs, dts = [], []
    for i, (im, space) in enumerate(specs):
        imgs.append((torch.from_numpy(im).cuda(), space))
        dts.append(torch.float16 if i % 4 == 1 else torch.float32)
    return imgs, dts


def _outs(imgs, dts):
    return [torch.empty((3,) + tuple(r.shape[:2]), dtype=dt, device="cuda") for (r, _), dt in zip(imgs, dts)]


def test_static_batch_matches_allocating_batch_on_two_calls():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    h = mact.mact_create()
    for call, (seed, count) in enumerate([(31, 40), (32, 17)]):
        imgs, dts = _images(seed, count)
        ref = mact.mact_convert_batch(h, imgs, outs=_outs(imgs, dts))
        got = mact.mact_convert_batch_static(h, imgs, outs=_outs(imgs, dts))
        torch.cuda.synchronize()
        for (rgb, space), a, b in zip(imgs, got, ref):
            # within the parity tolerance of the space (the kernels are the
            # same, so this is in fact bit for bit)
            check_space(space, a, [to_np(b[c]) for c in range(3)], dtype=a.dtype,
                        what="static call %d %s %s" % (call, space, tuple(rgb.shape)))
            assert torch.equal(a, b)
    h.close()


def test_static_batch_rejects_oversized_requests():
    h = mact.mact_create()
    L = mact.lib()
    arr = (mact.Image * 1)()
    assert L.mact_convert_batch_static(h.ptr, arr, 1025, None) == -1
    assert b"1024" in L.mact_last_error()
    assert L.mact_convert_batch_static(h.ptr, arr, -1, None) == -1
    assert L.mact_convert_batch_static(None, arr, 0, None) == -1
    assert L.mact_convert_batch_static(h.ptr, arr, 0, None) == 0
    h.close()
