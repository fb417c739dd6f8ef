"""The batched entry point that allocates nothing (mact_convert_batch_static)
against the allocating one (mact_convert_batch) and the FP64 oracle, through
the C ABI.

It exists for callers that cannot allocate at call time (fixed-memory
pipelines, plug-ins and callbacks that must stay out of the allocator), so it
keeps its work list in a fixed device array.  These checks make sure that
array gives the same results as the allocating path on consecutive calls,
that the results match the oracle within the parity tolerances, that a stale
work list from the previous call never leaks into the next one, that the
calls after the first leave the device's free memory unchanged, and that an
oversized request is refused.  Collected last on purpose."""
import pytest
import torch

from paper_1009_0854_gb300 import mact, synth
from parity import check_space, oracle_planes

pytestmark = pytest.mark.gpu


def _images(seed, count):
    specs = synth.batch_images(count=count, seed=seed, lo=8, hi=700)
    imgs, dts, host = [], [], []
    for i, (im, space) in enumerate(specs):
        imgs.append((torch.from_numpy(im).cuda(), space))
        dts.append(torch.float16 if i % 4 == 1 else torch.float32)
        host.append(im)
    return imgs, dts, host


def _outs(imgs, dts):
    return [torch.empty((3,) + tuple(r.shape[:2]), dtype=dt, device="cuda") for (r, _), dt in zip(imgs, dts)]


def test_static_batch_matches_oracle_and_allocating_batch_on_consecutive_calls():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    h = mact.mact_create()
    # two lists long enough for the fixed array (more than 32 images; the
    # second shorter than the first, so a stale tail would show), then a short
    # list that goes by value
    cases = []
    for seed, count in [(31, 40), (32, 37), (33, 17)]:
        imgs, dts, host = _images(seed, count)
        ref = mact.mact_convert_batch(h, imgs, outs=_outs(imgs, dts))
        cases.append((imgs, dts, host, ref, _outs(imgs, dts)))
    torch.cuda.synchronize()
    # the first call on the device looks up the array's address (and may
    # load the library's kernels: with lazy loading, a kernel's first launch
    # takes device memory for its code)
    mact.mact_convert_batch_static(h, cases[0][0], outs=cases[0][4])
    torch.cuda.synchronize()
    for call, (imgs, dts, host, ref, outs) in enumerate(cases):
        for o in outs:
            o.fill_(float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        got = mact.mact_convert_batch_static(h, imgs, outs=outs)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, "call %d changed the free device memory" % call
        for (rgb, space), a, b, im, dt in zip(imgs, got, ref, host, dts):
            what = "static call %d %s %s" % (call, space, tuple(rgb.shape))
            assert torch.equal(a, b), what
            check_space(space, a, oracle_planes(space, im), dtype=dt, what=what)
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
