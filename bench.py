"""Benchmark of the MACT per-pixel hot path on GB300.

Workload (one step): every 24-bit colour (2^24 pixels, lexicographic, one
4096 x 4096 uint8 image) converted by each per-pixel row of the hot path:
MACT RGB->CIELAB (4,4), HSI (n=5), SCT (5,5,5); the exact (libm) forms of
the three; and trilinear / prism / pyramidal / tetrahedral interpolation in
17^3 and 33^3 FP32 LUTs (built and packed to 16-byte nodes once, before the
timed region) -- 14 conversions, FP32 planar output.

value = pixel-conversions per second over the whole step (14 x 2^24 pixels
per step per GPU), in Gpix/s; the MACT CIELAB row's own Gpix/s and HBM
roofline fraction are reported under "rows" and "roofline_mact_cielab".
Inputs rotate over 8 distinct copies of the cube (400 MB > the 129 MB L2),
so no row reads its input from L2.

The same line (one GPU only) also carries the metric's other halves:
  large  -- MACT CIELAB (4,4) on one 16384 x 16384 image, FP32 and FP16
            planes: Gpix/s and fraction of the measured HBM bandwidth;
  served -- a seeded Poisson trace (2000 requests/s of 0.1-24 Mpx images,
            --served-seconds long) through the continuous-batching server
            (direct mode, MACT (4,4) and the fitted (6,6) rational) and
            through the plain per-image exact-libm path, in the same process:
            p50/p99/max latency and Gpix/s of each, with the max Delta E*ab of
            each transform over the cube.

--impl reference times the FP64 CPU oracle (the deliberately slow reference
arm) on a bounded sample of the same workload.
"""
import argparse
import collections
import gc
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PIX = 1 << 24
IN_COPIES = 8
METRIC = "Gpix/s and % of HBM roofline (MACT RGB→CIELAB); served p99 vs plain, same ΔE"
WORKLOAD = ("exhaustive RGB cube: 2^24 uint8 triplets (4096x4096, lexicographic) through MACT "
            "CIELAB(4,4)/HSI(5)/SCT(5,5,5), exact CIELAB/HSI/SCT, and tri/prism/pyr/tet from 17^3 and "
            "33^3 FP32 LUTs; FP32 planar out; 14 conversions per step")

ROWS = ([("mact_cielab", "mact", "cielab"), ("mact_hsi", "mact", "hsi"), ("mact_sct", "mact", "sct"),
         ("exact_cielab", "exact", "cielab"), ("exact_hsi", "exact", "hsi"), ("exact_sct", "exact", "sct")] +
        [("lut%d_%s" % (n, m), "lut", (m, n)) for n in (17, 33)
         for m in ("trilinear", "prism", "pyramid", "tetra")])


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001 - fall back to the recipe's figure
        return 6800.0, "fallback"


KERNEL_FILES = {
    "convert": ("common.cuh", "engine.cuh", "pixel.cuh", "convert_common.cuh", "k_convert.cu"),
    "lut": ("common.cuh", "engine.cuh", "k_lut.cu", "k_lut_interp.cuh", "k_lut_inst.cu"),
}


def kernel_group(row):
    return "lut" if row.startswith("lut") else "convert"


def source_hash(group):
    """Hash of the source files that define a row's kernel: a recorded DRAM
    traffic figure is only reported while these are unchanged."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1009_0854_gb300", "csrc")
    for name in KERNEL_FILES[group]:
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode())
            h.update(fh.read())
    return h.hexdigest()[:12]


def profile_table(fname):
    """Per-row figures from a committed ncu summary under profiles/ (lines
    "row value source_hash"), for rows whose kernel sources still hash the
    same as when the figure was taken."""
    path = os.path.join(ROOT, "profiles", fname)
    out = {}
    if not os.path.exists(path):
        return out
    cur = {g: source_hash(g) for g in KERNEL_FILES}
    for line in open(path):
        line = line.split("#", 1)[0].split()
        if len(line) == 3 and line[2] == cur[kernel_group(line[0])]:
            out[line[0]] = float(line[1])
    return out


def traffic_table():
    """Per-launch DRAM bytes (read + write) from profiles/traffic.txt."""
    return profile_table("traffic.txt")


def instruction_table():
    """Instructions per pixel (warp instructions x 32 / pixels) from
    profiles/instructions.txt."""
    return profile_table("instructions.txt")


# Rows bound by instruction issue rather than by memory: the exact SCT runs two
# atan2f and two IEEE sqrtf per pixel.  Their roofline is the issue rate.
ALU_ROWS = ("exact_sct",)


def issue_peak(num_sms):
    """Lane-instructions per second at full issue, in T/s: SMs x 4 schedulers
    x one warp instruction per cycle x 32 lanes x the maximum SM clock (from
    MEASURED_PEAKS.json, else the GB300's 2070 MHz)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            mhz, kind = float(json.load(fh)["sm_max_mhz"]), "measured sm_max_mhz"
    except Exception:  # noqa: BLE001 - the part's maximum clock
        mhz, kind = 2070.0, "nominal 2070 MHz"
    return num_sms * 4 * 32 * mhz * 1e6 / 1e12, "%d SMs x 4 issue x 32 lanes x %s" % (num_sms, kind)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:  # noqa: BLE001 - no nvidia-smi: no clock record
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:  # noqa: BLE001
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)
        if not self.rows:
            return None
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def max_over_ranks(value, device=None):
    """The largest value over all ranks (the slowest replica sets the step
    time); the identity without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------- GPU arm

def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1009_0854_gb300 import mact, synth

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    h_mact = mact.mact_create()
    h_exact = mact.mact_create(exact=1)
    cube = synth.rgb_cube()
    cube_h = torch.from_numpy(cube)
    inputs = [cube_h.to(dev) for _ in range(IN_COPIES)]
    # the LUTs are built and packed to 16-byte nodes once, outside the timed
    # region (mact_lut_pack: the layout the kernels read)
    luts = {n: mact.mact_lut_pack(h_mact, mact.mact_lut_build(h_mact, n, device=dev)) for n in (17, 33)}
    outs = {name: torch.empty((3, 4096, 4096), dtype=torch.float32, device=dev) for name, _, _ in ROWS}
    torch.cuda.synchronize()

    def run_row(name, kind, arg, rgb, out):
        if kind == "mact":
            mact.mact_convert(h_mact, rgb, arg, out=out, stream=stream)
        elif kind == "exact":
            mact.mact_convert(h_exact, rgb, arg, out=out, stream=stream)
        else:
            m, n = arg
            mact.mact_lut_interp_packed(h_mact, m, luts[n], n, rgb, out=out.view(3, -1), stream=stream)

    ev = {name: [] for name, _, _ in ROWS}

    def step(i, timed):
        for r, (name, kind, arg) in enumerate(ROWS):
            rgb = inputs[(i * len(ROWS) + r) % IN_COPIES]
            if timed:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            run_row(name, kind, arg, rgb, outs[name])
            if timed:
                e1.record(stream)
                ev[name].append((e0, e1))

    for i in range(args.warmup):
        step(i, False)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.25)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(args.steps):
        step(args.warmup + i, True)
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(t0.elapsed_time(t1), dev)
    launches = args.steps * len(ROWS)

    row_ms = {name: statistics.mean(a.elapsed_time(b) for a, b in ev[name]) for name in ev}
    hbm, peak_kind = peaks()
    traffic = traffic_table()
    insts = instruction_table()
    ipeak, ipeak_kind = issue_peak(torch.cuda.get_device_properties(dev).multi_processor_count)
    bytes_px = 3 + 12

    def roof(name):
        t = row_ms[name] * 1e-3
        tr = traffic.get(name)
        if name in ALU_ROWS and name in insts:
            achieved = insts[name] * PIX / t / 1e12
            return {"bound": "alu", "achieved": round(achieved, 2), "peak": round(ipeak, 2), "unit": "Tinst/s",
                    "frac": round(achieved / ipeak, 4), "traffic": tr, "kernel": name,
                    "peak_source": ipeak_kind, "inst_per_px": insts[name],
                    "ms_per_launch": round(row_ms[name], 5)}
        achieved = PIX * bytes_px / t / 1e9
        return {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4), "traffic": tr, "kernel": name,
                "peak_source": peak_kind, "ms_per_launch": round(row_ms[name], 5)}

    dominant = max(row_ms, key=row_ms.get)
    rows = {name: {"gpix_s": round(PIX / (row_ms[name] * 1e-3) / 1e9, 2), "ms": round(row_ms[name], 5),
                   "hbm_frac": round(PIX * bytes_px / (row_ms[name] * 1e-3) / 1e9 / hbm, 4)}
            for name in row_ms}

    # end to end through the C ABI with host buffers, inside the timed region:
    # the pinned input is copied to the device once, and every row's kernel
    # writes its three planes straight into pinned host memory across the host
    # link (the kernels address mapped host memory; no staging copy)
    e2e = None
    if not args.no_e2e:
        pin_in = cube_h.pin_memory()
        pin_out = {name: torch.empty((3, 4096, 4096), dtype=torch.float32).pin_memory() for name, _, _ in ROWS}
        dev_in = inputs[0]

        def e2e_step():
            dev_in.copy_(pin_in, non_blocking=True)
            for name, kind, arg in ROWS:
                run_row(name, kind, arg, dev_in, pin_out[name])

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        k = max(2, args.steps // 4)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            e2e_step()
        b.record(stream)
        torch.cuda.synchronize()
        ems = max_over_ranks(a.elapsed_time(b) / k, dev)
        e2e = {"value": round(world * len(ROWS) * PIX / (ems * 1e-3) / 1e9, 3), "unit": "Gpix/s",
               "h2d_bytes_per_step": 3 * PIX, "d2h_bytes_per_step": len(ROWS) * 12 * PIX,
               "ms_per_step": round(ems, 4)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:   # the host baseline is a 1-GPU figure
        cpu = cpu_baseline(args.cpu_pixels)

    # the metric's other halves, on one GPU: MACT CIELAB on a single large
    # image (the HBM-roofline row), and the serving trace (served p50/p99
    # against the plain per-image exact path, with each path's max Delta E)
    large = served = clk_more = None
    if rank == 0 and world == 1 and not (args.no_large and args.no_served):
        del outs, inputs
        if e2e is not None:
            del pin_out
        torch.cuda.empty_cache()
        more = ClockSampler(local)
        more.start()
        if not args.no_large:
            large = large_headline(args.steps)
        if not args.no_served:
            served = serve_experiment(args.served_seconds, paths=("direct", "direct_fitted66", "plain"),
                                      ring_bytes=8 << 30, budget=16 << 30)
        clk_more = more.stop()

    if rank == 0:
        value = world * len(ROWS) * PIX / (ms / args.steps * 1e-3) / 1e9
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "Gpix/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "pixels_per_conversion": PIX, "conversions_per_step": len(ROWS),
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs rotate over %d distinct 50 MB copies (400 MB > 129 MB L2)" % IN_COPIES},
            "roofline": roof(dominant),
            "roofline_mact_cielab": roof("mact_cielab"),
            "mact_cielab_gpix_s": rows["mact_cielab"]["gpix_s"],
            "rows": rows,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clk,
            "gpu_launches": launches,
            "large": large,
            "served": served,
            "clocks_large_and_served": clk_more,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------- oracle (CPU) arm

def _oracle_rows(rgb, luts, nthreads):
    import oracle as O
    for name, kind, arg in ROWS:
        if kind == "mact":
            if arg == "cielab":
                O.cielab(rgb, nthreads=nthreads)
            elif arg == "hsi":
                O.hsi(rgb, nthreads=nthreads)
            else:
                O.sct(rgb, nthreads=nthreads)
        elif kind == "exact":
            if arg == "cielab":
                O.cielab(rgb, exact=True, nthreads=nthreads)
            elif arg == "hsi":
                O.hsi(rgb, mode="exact", nthreads=nthreads)
            else:
                O.sct(rgb, exact=True, nthreads=nthreads)
        else:
            m, n = arg
            O.lut_interp(m, luts[n], rgb, nthreads=nthreads)


def cpu_baseline(npix):
    """The FP64 oracle, as it stands, on the host cores: the first npix
    colours of the cube through all 14 conversions."""
    import oracle as O
    from paper_1009_0854_gb300 import synth
    cores = O.max_threads()
    rgb = synth.rgb_cube().reshape(-1, 3)[:npix].copy()
    luts = {n: O.lut_build(n) for n in (17, 33)}
    _oracle_rows(rgb[:4096], luts, cores)
    t = time.perf_counter()
    _oracle_rows(rgb, luts, cores)
    dt = time.perf_counter() - t
    # one thread, for comparison with the paper's single-threaded timings
    n1 = min(npix, 1 << 20)
    t = time.perf_counter()
    _oracle_rows(rgb[:n1], luts, 1)
    dt1 = time.perf_counter() - t
    return {"value": round(len(ROWS) * npix / dt / 1e9, 6), "unit": "Gpix/s", "cores": cores, "kind": "oracle",
            "sample": "first %d cube colours x %d conversions (%.1f s wall)" % (npix, len(ROWS), dt),
            "single_thread": {"value": round(len(ROWS) * n1 / dt1 / 1e9, 6), "unit": "Gpix/s", "cores": 1,
                              "sample": "first %d cube colours x %d conversions (%.1f s wall)" % (n1, len(ROWS), dt1)}}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle as O
    from paper_1009_0854_gb300 import synth
    cores = O.max_threads()
    npix = args.ref_pixels
    rgb_all = synth.rgb_cube().reshape(-1, 3)
    luts = {n: O.lut_build(n) for n in (17, 33)}
    times = []
    for i in range(args.warmup + args.steps):
        off = (i * npix) % PIX
        rgb = rgb_all[off:off + npix].copy()
        t = time.perf_counter()
        _oracle_rows(rgb, luts, cores)
        if i >= args.warmup:
            times.append(time.perf_counter() - t)
    sec = sum(times) / len(times)
    value = len(ROWS) * npix / sec / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "Gpix/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(sec * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "pixels_per_conversion_sampled": npix,
                   "conversions_per_step": len(ROWS)},
        "cpu_baseline": {"value": round(value, 6), "unit": "Gpix/s", "cores": cores, "kind": "oracle",
                         "sample": "%d consecutive cube colours per step x %d conversions" % (npix, len(ROWS))},
        "e2e": {"value": round(value, 6), "unit": "Gpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line))


# ------------------------------------------------ other workloads (--workload; one JSON line each)

def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def time_convert(torch, mact, h, rgb, space, out, k):
    """Mean CUDA-event time (ms) of k back-to-back conversions after 3
    untimed ones, on the current stream."""
    fn = lambda: mact.mact_convert(h, rgb, space, out=out)      # noqa: E731
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    a, b = _events(torch)
    a.record()
    for _ in range(k):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / k


def large_headline(steps):
    """MACT RGB->CIELAB (4,4) on one 16384 x 16384 image (the 512 x 512 parity
    generator's recipe: gradients above, uniform noise below), FP32 and FP16
    planes: Gpix/s and fraction of the measured HBM bandwidth.  Input 805 MB,
    output 3.2 / 1.6 GB: far larger than L2, so no flush is needed."""
    import torch
    from paper_1009_0854_gb300 import mact, synth
    dev = torch.device("cuda", 0)
    hbm, kind = peaks()
    h = mact.mact_create()
    side = 16384
    npx = side * side
    rgb = torch.from_numpy(synth.gradient_noise_image(side, side, seed=0)).to(dev)
    rows = {}
    for dt, dname, bpp in ((torch.float32, "f32", 15), (torch.float16, "f16", 9)):
        out = torch.empty((3, side, side), dtype=dt, device=dev)
        ms = time_convert(torch, mact, h, rgb, "cielab", out, max(10, steps))
        rows[dname] = {"ms": round(ms, 4), "gpix_s": round(npx / ms / 1e6, 2), "bytes_per_px": bpp,
                       "gb_s": round(npx * bpp / ms / 1e6, 1), "hbm_frac": round(npx * bpp / ms / 1e6 / hbm, 4),
                       "peak_gbs": hbm, "peak_source": kind}
        del out
    del rgb
    h.close()
    torch.cuda.empty_cache()
    return {"workload": "MACT CIELAB (4,4), one 16384x16384 uint8 image (gradients + noise)", "rows": rows}


def run_large_workload(args):
    """Single large images: the 512x512 parity generator (smooth gradients
    over the upper half, uniform noise below) at 8192x8192 and 16384x16384,
    MACT and exact CIELAB/HSI/SCT and the CIELUV variant, FP32 and FP16
    planes; inputs and outputs are far larger than L2."""
    import torch
    from paper_1009_0854_gb300 import mact, synth
    dev = torch.device("cuda", 0)
    hbm, _ = peaks()
    hm, he = mact.mact_create(), mact.mact_create(exact=1)
    h66 = mact.mact_create(lab_coeffs=1, lab_n=6, lab_m=6)   # fitted (6,6) cube root
    rows = {}
    for side in (8192, 16384):
        rgb = torch.from_numpy(synth.gradient_noise_image(side, side, seed=0)).to(dev)
        npx = side * side
        for dt, dname, bpp in ((torch.float32, "f32", 15), (torch.float16, "f16", 9)):
            out = torch.empty((3, side, side), dtype=dt, device=dev)
            for hname, h in (("mact", hm), ("exact", he), ("mact66", h66)):
                for space in (("cielab", "cieluv") if hname == "mact66" else ("cielab", "hsi", "sct", "cieluv")):
                    ms = time_convert(torch, mact, h, rgb, space, out, max(5, args.steps // 4))
                    rows["%d_%s_%s_%s" % (side, hname, space, dname)] = {
                        "ms": round(ms, 4), "gpix_s": round(npx / ms / 1e6, 2),
                        "gb_s": round(npx * bpp / ms / 1e6, 1), "hbm_frac": round(npx * bpp / ms / 1e6 / hbm, 4)}
            del out
        del rgb
        torch.cuda.empty_cache()
    print(json.dumps({"workload": "large: 8192^2 and 16384^2 single images (gradients + noise), %d B/px FP32, "
                      "%d B/px FP16, peak %.1f GB/s measured; mact66 = the library's fitted (6,6) cube-root "
                      "rational" % (15, 9, hbm), "rows": rows}))


def run_batch_workload(args):
    """256 uneven images (log-uniform sides in [64, 4096], mixed content and
    spaces): one batched launch vs per-image launches (MACT) vs per-image exact
    launches (plain), FP32 and FP16 outputs."""
    import torch
    from paper_1009_0854_gb300 import mact, synth
    dev = torch.device("cuda", 0)
    specs = synth.batch_images(count=256, seed=0)
    imgs = [(torch.from_numpy(im).to(dev), space) for im, space in specs]
    npx = sum(r.shape[0] * r.shape[1] for r, _ in imgs)
    h = mact.mact_create()
    he = mact.mact_create(exact=1)
    out = {}
    for dt, name in ((torch.float32, "f32"), (torch.float16, "f16")):
        outs = [torch.empty((3,) + tuple(r.shape[:2]), dtype=dt, device=dev) for r, _ in imgs]
        table, shape = mact.mact_autotune_batch(h, imgs, outs=outs, reps=3)
        plan, _ = mact.mact_batch_plan_create(h, imgs, outs=outs)

        def t(fn, k=args.steps):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            a, b = _events(torch)
            a.record()
            for _ in range(k):
                fn()
            b.record()
            torch.cuda.synchronize()
            return a.elapsed_time(b) / k

        ms_graph = t(plan.graph_launch)
        ms_batch = t(lambda: mact.mact_convert_batch(h, imgs, outs=outs))
        ms_single = t(lambda: [mact.mact_convert(h, r, s, out=o) for (r, s), o in zip(imgs, outs)])
        ms_plain = t(lambda: [mact.mact_convert(he, r, s, out=o) for (r, s), o in zip(imgs, outs)])
        # the same calls with the image descriptors marshalled once: the C
        # entry points' own per-call cost, without the binding's per-call
        # marshalling of 256 descriptors
        import ctypes
        arr = mact._image_array(imgs, outs)
        st = mact._stream(None)
        L = mact.lib()
        singles = [ctypes.byref(arr[i]) for i in range(len(imgs))]
        ms_batch_c = t(lambda: L.mact_convert_batch(h.ptr, arr, len(imgs), st))
        ms_single_c = t(lambda: [L.mact_convert(h.ptr, p, st) for p in singles])
        bpp = 3 + 3 * (4 if dt == torch.float32 else 2)
        hbm, _ = peaks()
        out[name] = {"graph_gpix_s": round(npx / ms_graph / 1e6, 2), "batch_gpix_s": round(npx / ms_batch / 1e6, 2),
                     "batch_c_gpix_s": round(npx / ms_batch_c / 1e6, 2),
                     "per_image_c_gpix_s": round(npx / ms_single_c / 1e6, 2),
                     "per_image_mact_gpix_s": round(npx / ms_single / 1e6, 2),
                     "per_image_exact_gpix_s": round(npx / ms_plain / 1e6, 2),
                     "graph_hbm_frac": round(npx * bpp / (ms_graph * 1e-3) / 1e9 / hbm, 4),
                     "autotuned_shape": {"threads": shape[0], "px_per_thread": shape[1], "ctas_per_sm": shape[2]},
                     "tune_table_ms": {"%dx%d/%d" % (r["threads"], r["px_per_thread"], r["ctas_per_sm"]):
                                       round(r["ms"], 4) for r in table}}
        plan.close()
    print(json.dumps({"workload": "batch: 256 uneven images, %d px" % npx, "rows": out}))


def run_grad_workload(args):
    """Fused forward + mean Delta E*ab + backward on 64 x 3 x 512 x 512."""
    import torch
    from paper_1009_0854_gb300 import mact, synth
    dev = torch.device("cuda", 0)
    x, tgt_rgb = synth.linear_rgb_batch(n=64, h=512, w=512, seed=0)
    xt = torch.from_numpy(x).to(dev)
    rows = {}
    for exact in (0, 1):
        h = mact.mact_create(exact=exact)
        tgt = mact.mact_lab_forward(h, torch.from_numpy(tgt_rgb).to(dev))
        loss = torch.empty((), device=dev)
        g = torch.empty_like(xt)
        for _ in range(3):
            mact.mact_lab_delta_e_loss(h, xt, tgt, loss=loss, grad_out=g)
        torch.cuda.synchronize()
        a, b = _events(torch)
        a.record()
        for _ in range(args.steps):
            mact.mact_lab_delta_e_loss(h, xt, tgt, loss=loss, grad_out=g)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / args.steps
        npx = x.shape[0] * x.shape[2] * x.shape[3]
        hbm, _ = peaks()
        rows["exact" if exact else "mact"] = {"ms": round(ms, 4), "gpix_s": round(npx / ms / 1e6, 2),
                                              "hbm_frac": round(npx * 36 / (ms * 1e-3) / 1e9 / hbm, 4),
                                              "loss": float(loss)}
    print(json.dumps({"workload": "grad: fused mean-DeltaE loss + backward, 64x3x512x512 FP32", "rows": rows}))


def run_lut_workload(args):
    """Standard (packed float3, 16-byte copy made per call above 17^3), packed
    once (mact_lut_pack) and caching LUT layouts, 4 methods x {9, 17, 33}^3, on the
    2^24-colour cube (coherent) and on i.i.d. uniform noise (incoherent); and
    HSI through a 17^3 / 33^3 LUT with angular hue interpolation beside the
    exact and MACT HSI transforms."""
    import numpy as np
    import torch
    from paper_1009_0854_gb300 import mact, synth
    dev = torch.device("cuda", 0)
    h = mact.mact_create()
    inputs = {"cube": torch.from_numpy(synth.rgb_cube()).to(dev),
              "noise": torch.from_numpy(np.random.default_rng(0).integers(0, 256, size=(4096, 4096, 3),
                                                                        dtype=np.uint8)).to(dev)}
    out = torch.empty((3, PIX), device=dev)
    hbm, _ = peaks()
    rows = {}
    for n in (9, 17, 33):
        lut = mact.mact_lut_build(h, n, device=dev)
        lut4 = mact.mact_lut_pack(h, lut)
        cache = mact.mact_lut_cache_build(h, lut)
        for name, x in inputs.items():
            xs = [x.clone() for _ in range(4)]
            for m in ("trilinear", "prism", "pyramid", "tetra"):
                for layout in ("standard", "packed", "caching"):
                    if layout == "standard":
                        fn = lambda v: mact.mact_lut_interp(h, m, lut, v, out=out)
                    elif layout == "packed":
                        fn = lambda v: mact.mact_lut_interp_packed(h, m, lut4, n, v, out=out)
                    else:
                        fn = lambda v: mact.mact_lut_interp_cached(h, m, cache, n, v, out=out)
                    for i in range(3):
                        fn(xs[i % 4])
                    torch.cuda.synchronize()
                    a, b = _events(torch)
                    a.record()
                    for i in range(args.steps):
                        fn(xs[i % 4])
                    b.record()
                    torch.cuda.synchronize()
                    ms = a.elapsed_time(b) / args.steps
                    rows["%s_lut%d_%s_%s" % (name, n, m, layout)] = {
                        "gpix_s": round(PIX / ms / 1e6, 1), "hbm_frac": round(PIX * 15 / (ms * 1e-3) / 1e9 / hbm, 4)}

    def timed(fn, xs):
        for i in range(3):
            fn(xs[i % 4])
        torch.cuda.synchronize()
        a, b = _events(torch)
        a.record()
        for i in range(args.steps):
            fn(xs[i % 4])
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / args.steps

    # HSI through a LUT with angular hue interpolation (the paper's trilinear
    # case) beside the exact and MACT HSI transforms on the same input
    he = mact.mact_create(exact=1)
    out3 = out.view(3, 4096, 4096)
    for name, x in inputs.items():
        xs = [x.clone() for _ in range(4)]
        for n in (17, 33):
            lut4 = mact.mact_lut_build_hsi(h, n)
            ms = timed(lambda v: mact.mact_lut_interp_hsi(h, lut4, v, out=out), xs)
            rows["%s_hsi_angular_lut%d_trilinear" % (name, n)] = {
                "gpix_s": round(PIX / ms / 1e6, 1), "hbm_frac": round(PIX * 15 / (ms * 1e-3) / 1e9 / hbm, 4)}
        for hn, hh in (("exact", he), ("mact", h)):
            ms = timed(lambda v: mact.mact_convert(hh, v, "hsi", out=out3), xs)
            rows["%s_hsi_%s" % (name, hn)] = {
                "gpix_s": round(PIX / ms / 1e6, 1), "hbm_frac": round(PIX * 15 / (ms * 1e-3) / 1e9 / hbm, 4)}
    print(json.dumps({"workload": "lut: standard vs caching layout, cube and uniform noise, 2^24 px; HSI through "
                      "an angular-hue LUT vs the exact and MACT HSI transforms", "rows": rows}))


def run_kernels_workload(args):
    """One launch of each row of the cube step, then MACT CIELAB with FP16
    planes, on one copy of the cube, after the LUTs are built and packed:
    a short, fixed launch sequence for profilers (ncu -k / -c).  Prints the
    launch order."""
    import torch
    from paper_1009_0854_gb300 import mact, synth
    dev = torch.device("cuda", 0)
    h, he = mact.mact_create(), mact.mact_create(exact=1)
    x = torch.from_numpy(synth.rgb_cube()).to(dev)
    luts = {n: mact.mact_lut_pack(h, mact.mact_lut_build(h, n, device=dev)) for n in (17, 33)}
    out = torch.empty((3, 4096, 4096), device=dev)
    o16 = torch.empty((3, 4096, 4096), dtype=torch.float16, device=dev)
    torch.cuda.synchronize()
    order = []
    for name, kind, arg in ROWS:
        if kind in ("mact", "exact"):
            mact.mact_convert(h if kind == "mact" else he, x, arg, out=out)
        else:
            m, n = arg
            mact.mact_lut_interp_packed(h, m, luts[n], n, x, out=out.view(3, -1))
        order.append(name)
    mact.mact_convert(h, x, "cielab", out=o16)
    order.append("mact_cielab_f16")
    torch.cuda.synchronize()
    print(json.dumps({"workload": "kernels: one launch per row on the 2^24 cube, then MACT CIELAB FP16",
                      "order": order}))


class PinnedRing:
    """Request output buffers carved from one pinned host allocation, made
    before the run: first in, first out, with out-of-order release (a slot is
    reused once every older slot is released too).  When the ring is full,
    take() calls reclaim() (which must release the oldest request) until the
    new buffer fits: back-pressure instead of a pinned allocation mid-run."""

    ALIGN = 256

    def __init__(self, torch, nbytes):
        self.buf = torch.empty(nbytes // 4, dtype=torch.float32).pin_memory()
        self.n = (nbytes // 4) * 4
        self.head = 0
        self.live = collections.deque()      # [offset, size, released]

    def _fit(self, size):
        if not self.live:
            self.head = 0
            return 0 if size <= self.n else None
        tail = self.live[0][0]
        if self.head > tail:                  # occupied [tail, head): free [head, n) and [0, tail)
            if self.head + size <= self.n:
                return self.head
            return 0 if size <= tail else None
        return self.head if self.head + size <= tail else None   # wrapped: free [head, tail)

    def take(self, nbytes, reclaim):
        size = -(-nbytes // self.ALIGN) * self.ALIGN
        if size > self.n:
            raise MemoryError("request larger than the output ring")
        while True:
            off = self._fit(size)
            if off is not None:
                break
            reclaim()
        entry = [off, size, False]
        self.live.append(entry)
        self.head = off + size
        return self.buf[off // 4: (off + nbytes) // 4], entry

    def give(self, entry):
        entry[2] = True
        while self.live and self.live[0][2]:
            self.live.popleft()


def serve_experiment(seconds, paths=("direct", "staged", "direct_fitted66", "plain"), ring_bytes=16 << 30,
                     budget=16 << 30):
    """Poisson arrivals (2000/s) of 0.1-24 Mpx images, 50/25/25% CIELAB/HSI/SCT,
    pinned host input and output (outputs carved from one pinned ring shared by
    every path), through the continuous-batching server (MACT, a device-memory
    admission budget of ``budget`` bytes) in direct mode (the kernel reads and
    writes the pinned buffers in place) and in staged mode (copies through the
    arena), in direct mode with the library's fitted (6,6) cube-root rational
    (max Delta E near the exact path's), and through the plain path (one
    request at a time: H2D, exact-libm kernel, D2H).  ``paths`` picks which
    run.  Every path first serves an untimed 0.25 s warm-up trace.  Latency
    counts from the trace's arrival time.  Returns a dict of results."""
    import torch
    from paper_1009_0854_gb300 import mact, synth
    dev = torch.device("cuda", 0)
    trace = synth.serve_trace(rate=2000.0, duration=seconds, seed=0)
    warm_trace = synth.serve_trace(rate=2000.0, duration=0.25, seed=1)
    maxpx = max(h * w for _, h, w, _, _ in trace + warm_trace)
    pool_in = torch.from_numpy(synth.request_image(4096, 6144, 2, 7).reshape(-1)).pin_memory()  # 75 MB
    ring = PinnedRing(torch, ring_bytes)

    def link_gbs(dst_views, src):
        """Copy-engine D2H bandwidth into the given pinned views (one copy each)."""
        st = torch.cuda.current_stream()
        for v in dst_views[:2]:
            v.copy_(src[: v.numel()], non_blocking=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for v in dst_views:
            v.copy_(src[: v.numel()], non_blocking=True)
        e1.record(st)
        torch.cuda.synchronize()
        return round(sum(v.numel() * 4 for v in dst_views) / (e0.elapsed_time(e1) * 1e-3) / 1e9, 1)

    cal_src = torch.empty(64 << 20, dtype=torch.float32, device=dev)      # 256 MB
    step = ring.buf.numel() // 16
    ring_gbs = link_gbs([ring.buf[k * step: k * step + min(step, 64 << 20)] for k in range(16)], cal_src)
    ring0_gbs = link_gbs([ring.buf[: min(step, 64 << 20)]] * 16, cal_src)
    del cal_src

    def req_in(hgt, wid):
        return pool_in[: hgt * wid * 3].view(hgt, wid, 3)

    def summary(lat, npx, wall, extra=None):
        lat = sorted(lat)
        d = {"requests": len(lat), "p50_ms": round(lat[len(lat) // 2], 3),
             "p99_ms": round(lat[int(0.99 * (len(lat) - 1))], 3), "max_ms": round(lat[-1], 3),
             "gpix_s": round(npx / wall / 1e9, 3)}
        d.update(extra or {})
        return d

    h = mact.mact_create()

    h66 = mact.mact_create(lab_coeffs=1, lab_n=6, lab_m=6)

    def served(tr, mode, hs=None):
        """The load generator submits at each arrival time and, while waiting for the
        next one, retires every finished request (its ring slot is released)."""
        srv = mact.mact_serve_create(hs or h, budget, max_slots=128)
        mact.mact_serve_set_mode(srv, mode)
        inflight = collections.OrderedDict()    # ticket -> (arrival, submit, ring entry)
        lat = []
        stats = {"reclaim_waits": 0, "inflight_max": 0, "lag_max_ms": 0.0}
        lag_series = []                          # worst lag in each 0.5 s of the trace

        def retire(tk, wait=False):
            ta, t_sub, entry = inflight.pop(tk)
            if wait:
                mact.mact_serve_wait(srv, tk, 600000)
            _, server_ms = mact.mact_serve_poll(srv, tk)
            mact.mact_serve_release(srv, tk)
            ring.give(entry)
            lat.append((t_sub - ta) * 1e3 + server_ms)

        last_scan = [0.0]

        def reap():
            """Retire finished requests: from the oldest while they are done
            (the server is first-in first-out), and every 2 ms a full scan."""
            n = 0
            while inflight and mact.mact_serve_poll(srv, next(iter(inflight)))[0]:
                retire(next(iter(inflight)))
                n += 1
            now = time.perf_counter()
            if now - last_scan[0] > 2e-3:
                last_scan[0] = now
                for tk in [tk for tk in inflight if mact.mact_serve_poll(srv, tk)[0]]:
                    retire(tk)
                    n += 1
            return n > 0

        def reclaim():                             # ring full: wait for the oldest
            stats["reclaim_waits"] += 1
            if not reap():
                retire(next(iter(inflight)), wait=True)

        npx = 0
        t0 = time.perf_counter()
        for ta, hgt, wid, _, space in tr:
            while time.perf_counter() - t0 < ta:
                if not (inflight and reap()):
                    time.sleep(5e-5)
            buf, entry = ring.take(12 * hgt * wid, reclaim)
            t_sub = time.perf_counter() - t0
            tk, _ = mact.mact_serve_submit(srv, req_in(hgt, wid), space, out=buf.view(3, hgt, wid))
            inflight[tk] = (ta, t_sub, entry)
            stats["inflight_max"] = max(stats["inflight_max"], len(inflight))
            stats["lag_max_ms"] = max(stats["lag_max_ms"], round((t_sub - ta) * 1e3, 3))
            k = int(ta / 0.5)
            while len(lag_series) <= k:
                lag_series.append(0.0)
            lag_series[k] = max(lag_series[k], round((t_sub - ta) * 1e3, 1))
            npx += hgt * wid
        while inflight:
            retire(next(iter(inflight)), wait=True)
        wall = time.perf_counter() - t0
        st = mact.mact_serve_stats(srv)
        srv.close()
        stats["lag_ms_per_half_second"] = lag_series
        stages = {k[:-3]: round(st[k], 3) for k in ("queue_p50_ms", "h2d_p50_ms", "compute_p50_ms", "d2h_p50_ms",
                                                   "queue_p99_ms", "h2d_p99_ms", "compute_p99_ms", "d2h_p99_ms")}
        stages["d2h_busy_ms"] = round(st["d2h_busy_ms"], 1)
        stages["d2h_copy_gbs"] = round(st["d2h_copy_gbs"], 1)
        return summary(lat, npx, wall, {"mode": mode, "budget_bytes": budget,
                                        "admitted_bytes_max": int(st["inflight_bytes_max"]), "batches": st["batches"],
                                        "server_p50_ms": round(st["p50_ms"], 3),
                                        "server_p99_ms": round(st["p99_ms"], 3), "server_stages_ms": stages,
                                        "client": stats})

    # plain: one request at a time, exact libm kernels
    he = mact.mact_create(exact=1)
    dbuf_in = torch.empty(3 * maxpx, dtype=torch.uint8, device=dev)
    dbuf_out = torch.empty(3 * maxpx, dtype=torch.float32, device=dev)
    s = torch.cuda.current_stream()

    def plain(tr):
        lat = []
        npx = 0
        t0 = time.perf_counter()
        for ta, hgt, wid, _, space in tr:
            while time.perf_counter() - t0 < ta:
                pass
            inp = req_in(hgt, wid)
            buf, entry = ring.take(12 * hgt * wid, None)     # the ring is empty here: never reclaims
            din = dbuf_in[: hgt * wid * 3].view(hgt, wid, 3)
            dout = dbuf_out[: 3 * hgt * wid].view(3, hgt, wid)
            din.copy_(inp, non_blocking=True)
            mact.mact_convert(he, din, space, out=dout, stream=s)
            buf.view(3, hgt, wid).copy_(dout, non_blocking=True)
            s.synchronize()
            ring.give(entry)
            lat.append((time.perf_counter() - t0 - ta) * 1e3)
            npx += hgt * wid
        return summary(lat, npx, time.perf_counter() - t0)

    def quiet(fn):
        """Run one path of the trace with Python's cyclic garbage collector
        off (collected first): a collection pause of tens of milliseconds in
        the load generator delays every arrival behind it, and the burst it
        then submits shows as server latency."""
        def run(tr):
            gc.collect()
            gc.disable()
            try:
                return fn(tr)
            finally:
                gc.enable()
        return run

    runners = {"direct": quiet(lambda tr: served(tr, "direct")), "staged": quiet(lambda tr: served(tr, "staged")),
               "direct_fitted66": quiet(lambda tr: served(tr, "direct", h66)), "plain": quiet(plain)}

    def same_delta_e():
        """Served results equal single-image conversions bit for bit (checked
        on a sample of the trace's requests), so their max Delta E*ab is the
        MACT transform's own: reported over the whole cube by the device error
        kernels, beside the exact-libm path's."""
        srv = mact.mact_serve_create(h, 1 << 30, max_slots=16)
        same, k = True, 0
        for ta, hgt, wid, _, space in trace[:: max(1, len(trace) // 24)][:24]:
            rgb = req_in(hgt, wid)
            tk, out = mact.mact_serve_submit(srv, rgb, space)
            mact.mact_serve_wait(srv, tk, 60000)
            ref = mact.mact_convert(h, rgb.to(dev), space).cpu()
            torch.cuda.synchronize()
            same = same and torch.equal(out, ref)
            mact.mact_serve_release(srv, tk)
            k += 1
        srv.close()
        e_mact = mact.mact_cube_error(h, "cielab")
        e_66 = mact.mact_cube_error(h66, "cielab")
        e_exact = mact.mact_cube_error(he, "cielab")
        return {"sampled_requests": k, "served_bit_identical_to_single_image": same,
                "mact_cielab_delta_e_max_cube": round(e_mact[1], 6),
                "mact_cielab_delta_e_avg_cube": round(e_mact[0], 6),
                "fitted66_cielab_delta_e_max_cube": round(e_66[1], 8),
                "fitted66_cielab_delta_e_avg_cube": round(e_66[0], 8),
                "exact_fp32_cielab_delta_e_max_cube": round(e_exact[1], 8)}
    names = {"direct": "served_direct", "staged": "served_staged", "direct_fitted66": "served_direct_fitted66",
             "plain": "plain_exact_per_image"}
    results = {}
    for p in paths:
        # each path serves the untimed warm-up trace right before its timed
        # trace: with all warm-ups first, whichever path ran second measured
        # 30-40x higher p99 (its server's kernel times grew), while two
        # experiments run one after the other were both unaffected
        runners[p](warm_trace)
        results[names[p]] = runners[p](trace)
    results["same_delta_e"] = same_delta_e()
    results["link"] = {"d2h_gbs_ring_spread": ring_gbs, "d2h_gbs_ring_start": ring0_gbs}
    results["trace"] = {"rate_per_s": 2000.0, "seconds": seconds, "requests": len(trace),
                        "offered_gpix_s": round(sum(hh * ww for _, hh, ww, _, _ in trace) / seconds / 1e9, 3)}
    del ring, pool_in, dbuf_in, dbuf_out
    torch.cuda.empty_cache()
    return results


def run_serve_workload(args):
    """The serving trace through every path (see serve_experiment)."""
    results = serve_experiment(args.serve_seconds)
    print(json.dumps({"workload": "serve: Poisson 2000 req/s for %g s, 0.1-24 Mpx, pinned host buffers"
                      % args.serve_seconds, "rows": results}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mact", choices=["mact", "reference"])
    ap.add_argument("--cpu-pixels", type=int, default=PIX)
    ap.add_argument("--ref-pixels", type=int, default=1 << 22)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="cube",
                    choices=["cube", "batch", "serve", "grad", "lut", "large", "kernels"],
                    help="cube: the default step; the others measure the batched, served and "
                         "differentiable forms on their own workloads; kernels: one launch of "
                         "each row, for profilers")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="length of --workload serve's trace")
    ap.add_argument("--served-seconds", type=float, default=10.0,
                    help="length of the serving trace in the default line's 'served' key")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-large", action="store_true")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)   # at least 3 untimed warm-up steps
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch_workload(args)
    elif args.workload == "serve":
        run_serve_workload(args)
    elif args.workload == "grad":
        run_grad_workload(args)
    elif args.workload == "lut":
        run_lut_workload(args)
    elif args.workload == "large":
        run_large_workload(args)
    elif args.workload == "kernels":
        run_kernels_workload(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
