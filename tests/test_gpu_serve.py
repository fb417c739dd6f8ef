"""The served form: continuous batching with a memory budget.  Every result
must equal the single-image conversion of the same image, whether the
request ran alone or in a mix with others, and must match the FP64 oracle
element by element within the parity tolerances of its space."""
import time

import numpy as np
import pytest
import torch

from paper_1009_0854_gb300 import mact, synth
from parity import check_space, oracle_planes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return mact.mact_create()


def _requests(seed, count, lo=16, hi=900):
    out = []
    for i, (im, space) in enumerate(synth.batch_images(count=count, seed=seed, lo=lo, hi=hi)):
        dt = torch.float16 if i % 5 == 2 else torch.float32
        out.append((im, space, dt))
    return out


def _reference(h, reqs):
    refs = []
    for im, space, dt in reqs:
        refs.append(mact.mact_convert(h, torch.from_numpy(im).cuda(), space, dtype=dt).cpu())
    torch.cuda.synchronize()
    return refs


@pytest.fixture(scope="module")
def mix_requests():
    """48 uneven requests (FP32 and FP16 planes, all three spaces) with their
    FP64 oracle planes."""
    reqs = _requests(3, 48)
    return reqs, [oracle_planes(space, im) for im, space, _ in reqs]


@pytest.mark.parametrize("mode", ["direct", "staged"])
def test_each_result_same_alone_and_in_the_mix(h, mode, mix_requests):
    """Alone and in the mix, in both serving modes: each result equals the
    single-image conversion bit for bit and the oracle within tolerance."""
    reqs, orc = mix_requests
    refs = _reference(h, reqs)
    srv = mact.mact_serve_create(h, 256 << 20, max_slots=16)
    mact.mact_serve_set_mode(srv, mode)
    # alone: one request at a time
    for (im, space, dt), ref, o in zip(reqs[:12], refs[:12], orc[:12]):
        t, out = mact.mact_serve_submit(srv, torch.from_numpy(im).pin_memory(), space, dtype=dt)
        mact.mact_serve_wait(srv, t, 30000)
        assert torch.equal(out, ref)
        check_space(space, out, o, dtype=dt, what="served alone (%s) %s %s" % (mode, space, im.shape))
        mact.mact_serve_release(srv, t)
    # in the mix: everything at once, host (pinned), pageable and device buffers
    pending = []
    for i, ((im, space, dt), ref) in enumerate(zip(reqs, refs)):
        if i % 3 == 0:
            rgb = torch.from_numpy(im).pin_memory()
        elif i % 3 == 1:
            rgb = torch.from_numpy(im.copy())            # pageable host memory
        else:
            rgb = torch.from_numpy(im).cuda()
        t, out = mact.mact_serve_submit(srv, rgb, space, dtype=dt)
        pending.append((t, out, ref))
    for (t, out, ref), (im, space, dt), o in zip(pending, reqs, orc):
        mact.mact_serve_wait(srv, t, 60000)
        assert torch.equal(out.cpu(), ref)
        check_space(space, out, o, dtype=dt, what="served in the mix (%s) %s %s" % (mode, space, im.shape))
    st = mact.mact_serve_stats(srv)
    assert st["completed"] == 12 + 48 and st["failed"] == 0
    assert st["batches"] >= 2
    assert mact.mact_serve_destroy(srv) == 0


@pytest.mark.parametrize("mode", ["staged", "direct"])
def test_admission_respects_the_budget(h, mode):
    """A budget that holds one 512x512 FP32 request (0.75 + 3 MB of input and
    output) at a time, in either mode: all requests complete, one per batch,
    and the admitted bytes never exceed the budget; a request larger than the
    whole budget is refused at submit with MACT_E_NOMEM.  A server with a
    larger budget takes it."""
    im = synth.gradient_noise_image(512, 512, seed=1)
    budget = 4 << 20
    srv = mact.mact_serve_create(h, budget, max_slots=8)
    mact.mact_serve_set_mode(srv, mode)
    ref = mact.mact_convert(h, torch.from_numpy(im).cuda(), "cielab").cpu()
    ts = [mact.mact_serve_submit(srv, torch.from_numpy(im).pin_memory(), "cielab") for _ in range(6)]
    for t, out in ts:
        mact.mact_serve_wait(srv, t, 30000)
        assert torch.equal(out, ref)
    big = torch.zeros((1024, 1024, 3), dtype=torch.uint8).pin_memory()
    with pytest.raises(mact.MactError) as e:
        mact.mact_serve_submit(srv, big, "cielab")
    assert e.value.status == -2
    st = mact.mact_serve_stats(srv)
    assert st["completed"] == 6 and st["batches"] == 6
    assert 0 < st["inflight_bytes_max"] <= budget
    srv.close()
    srv = mact.mact_serve_create(h, 64 << 20, max_slots=8)
    mact.mact_serve_set_mode(srv, mode)
    t, out = mact.mact_serve_submit(srv, big, "cielab")
    mact.mact_serve_wait(srv, t, 30000)
    assert torch.equal(out, mact.mact_convert(h, big.cuda(), "cielab").cpu())
    srv.close()


def test_cancel_queued_request(h):
    """With one slot and a large first request in flight, a queued request
    can be cancelled; an admitted one cannot."""
    big = torch.from_numpy(synth.gradient_noise_image(4096, 4096, seed=2)).pin_memory()
    small = torch.from_numpy(synth.gradient_noise_image(64, 64, seed=3)).pin_memory()
    srv = mact.mact_serve_create(h, 1 << 30, max_slots=1)
    t0, _ = mact.mact_serve_submit(srv, big, "sct")
    queued = [mact.mact_serve_submit(srv, small, "hsi")[0] for _ in range(4)]
    cancelled = 0
    for t in queued[1:]:
        try:
            mact.mact_serve_cancel(srv, t)
            cancelled += 1
        except mact.MactError as e:
            assert e.status == -6     # already admitted
    mact.mact_serve_wait(srv, t0, 60000)
    for t in queued:
        mact.mact_serve_wait(srv, t, 60000)
        done, _ = mact.mact_serve_poll(srv, t)
        assert done
    assert cancelled >= 1
    srv.close()


def test_stream_of_arrivals_overlaps(h):
    """Requests submitted while earlier ones run are batched into later
    launches; latency percentiles are reported."""
    reqs = _requests(9, 64, lo=64, hi=1500)
    srv = mact.mact_serve_create(h, 1 << 30, max_slots=32)
    pend = []
    for im, space, dt in reqs:
        pend.append(mact.mact_serve_submit(srv, torch.from_numpy(im).pin_memory(), space, dtype=dt))
        time.sleep(0.0005)
    for t, _ in pend:
        mact.mact_serve_wait(srv, t, 60000)
    st = mact.mact_serve_stats(srv)
    assert st["completed"] == 64 and st["p99_ms"] >= st["p50_ms"] > 0
    srv.close()


def test_wait_times_out_and_destroy_drains(h):
    big = torch.from_numpy(synth.gradient_noise_image(4096, 4096, seed=4)).pin_memory()
    srv = mact.mact_serve_create(h, 1 << 30, max_slots=1)
    ts = [mact.mact_serve_submit(srv, big, "cielab")[0] for _ in range(3)]
    with pytest.raises(mact.MactError) as e:
        mact.mact_serve_wait(srv, ts[-1], 0.0)
    assert e.value.status in (-5,)
    assert srv.close(60000.0) == 0


def test_direct_and_staged_modes_agree(h):
    """Direct mode (host buffers used in place by the kernel) and staged mode
    (copied through the arena) give the same bits; only staged mode copies
    outputs back."""
    reqs = _requests(5, 24)
    refs = _reference(h, reqs)
    for mode in ("staged", "direct"):
        srv = mact.mact_serve_create(h, 256 << 20, max_slots=8)
        mact.mact_serve_set_mode(srv, mode)
        pending = []
        for i, ((im, space, dt), ref) in enumerate(zip(reqs, refs)):
            rgb = torch.from_numpy(im).pin_memory() if i % 2 == 0 else torch.from_numpy(im.copy())
            t, out = mact.mact_serve_submit(srv, rgb, space, dtype=dt)   # out: pinned host
            pending.append((t, out, ref))
        for t, out, ref in pending:
            mact.mact_serve_wait(srv, t, 60000)
            assert torch.equal(out, ref)
        st = mact.mact_serve_stats(srv)
        assert st["completed"] == len(reqs)
        if mode == "staged":
            assert st["d2h_busy_ms"] > 0
        else:
            assert st["d2h_busy_ms"] == 0
        with pytest.raises(mact.MactError):
            mact.mact_serve_set_mode(srv, 7)
        srv.close()


def test_failed_batches_report_and_return_their_memory(h, monkeypatch):
    """Host-side fault injection (every 3rd batch fails after its input
    copies are enqueued): failed requests report MACT_E_CUDA with the reason,
    the others still equal mact_convert, and the staging memory of the failed
    ones comes back (a request needing most of the budget is admitted)."""
    monkeypatch.setenv("MACT_SERVE_FAIL_EVERY", "3")
    srv = mact.mact_serve_create(h, 8 << 20, max_slots=4)
    monkeypatch.delenv("MACT_SERVE_FAIL_EVERY")
    mact.mact_serve_set_mode(srv, "staged")
    reqs = _requests(11, 12, lo=16, hi=300)
    refs = _reference(h, reqs)
    failed = 0
    for k, ((im, space, dt), ref) in enumerate(zip(reqs, refs)):
        t, out = mact.mact_serve_submit(srv, torch.from_numpy(im).pin_memory(), space, dtype=dt)
        try:
            mact.mact_serve_wait(srv, t, 30000)
            assert torch.equal(out, ref)
        except mact.MactError as e:
            assert e.status == mact.MACT_E_CUDA and "injected" in str(e)
            failed += 1
        mact.mact_serve_release(srv, t)
    assert failed == 4
    st = mact.mact_serve_stats(srv)
    assert st["failed"] == 4 and st["completed"] == 8
    big = torch.from_numpy(synth.gradient_noise_image(700, 700, seed=9)).pin_memory()   # 1.5 + 5.9 MB of 8 MB
    for _ in range(2):                 # the 3rd batch after this point would fail: stop before it
        t, out = mact.mact_serve_submit(srv, big, "cielab")
        mact.mact_serve_wait(srv, t, 30000)
        assert torch.equal(out, mact.mact_convert(h, big.cuda(), "cielab").cpu())
        mact.mact_serve_release(srv, t)
    srv.close()
