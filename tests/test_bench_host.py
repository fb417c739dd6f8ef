"""Host-side logic of bench.py that needs no GPU: the pinned output ring of
the serving load generator (no overlap between live slots, every slot in
bounds, back-pressure that always makes progress) and the determinism of the
serving trace."""
import random

import pytest

import bench
from paper_1009_0854_gb300 import synth


class _FakeTensor:
    def __init__(self, n):
        self.n = n

    def pin_memory(self):
        return self

    def numel(self):
        return self.n

    def __getitem__(self, sl):
        return (sl.start, sl.stop)


class _FakeTorch:
    float32 = "float32"

    @staticmethod
    def empty(n, dtype=None):
        return _FakeTensor(n)


def _check_live(ring):
    spans = sorted((e[0], e[0] + e[1]) for e in ring.live if not e[2])
    for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
        assert a1 <= b0
    for a0, a1 in spans:
        assert 0 <= a0 and a1 <= ring.n


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ring_slots_never_overlap(seed):
    ring = bench.PinnedRing(_FakeTorch, 1 << 20)
    rng = random.Random(seed)
    held = []
    reclaims = [0]

    def reclaim():
        reclaims[0] += 1
        ring.give(held.pop(0))

    for _ in range(5000):
        if held and (rng.random() < 0.45 or len(held) > 24):
            e = held.pop(rng.randrange(len(held)) if rng.random() < 0.3 else 0)
            ring.give(e)
        else:
            n = rng.randrange(1, 180000)
            view, e = ring.take(n, reclaim)
            assert view[1] - view[0] == n // 4
            assert view[0] == e[0] // 4 and e[0] % bench.PinnedRing.ALIGN == 0
            held.append(e)
        _check_live(ring)
    assert reclaims[0] > 0                   # back-pressure was exercised


def test_ring_rejects_oversize_and_resets_when_empty():
    ring = bench.PinnedRing(_FakeTorch, 4096)
    with pytest.raises(MemoryError):
        ring.take(8192, lambda: None)
    _, e1 = ring.take(1000, None)
    _, e2 = ring.take(1000, None)
    ring.give(e2)
    ring.give(e1)
    assert not ring.live
    _, e3 = ring.take(4000, None)            # whole ring again after a full release
    assert e3[0] == 0


def test_serve_trace_is_deterministic():
    a = synth.serve_trace(rate=2000.0, duration=0.5, seed=3)
    b = synth.serve_trace(rate=2000.0, duration=0.5, seed=3)
    assert a == b
    assert all(0 < t < 0.5 for t, *_ in a)
    assert all(0.09e6 <= h * w <= 24.5e6 for _, h, w, _, _ in a)


def test_clock_summary_reports_median_max_and_throttle_reasons():
    """The clocks record of the bench line: median SM clock under load, the
    maximum clock, and every throttle reason seen active in any sample
    (hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap);
    unreadable clock fields are skipped."""
    cs = bench.ClockSampler(0)
    na, act = "Not Active", "Active"
    cs.rows = [
        ["0", "2070", "2070", "900.1", "0x0", na, na, na, na],
        ["0", "1965", "2070", "1400.0", "0x4", na, na, na, act],
        ["0", "[N/A]", "2070", "1200.0", "0x0", na, na, na, na],
        ["0", "2055", "2070", "1100.0", "0x8", act, na, na, na],
    ]
    s = cs.stop()
    assert s["samples"] == 4
    assert s["sm_mhz"] == 2055.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_summary_without_samples_is_none():
    assert bench.ClockSampler(0).stop() is None


def test_traffic_figures_only_for_unchanged_kernel_sources(tmp_path, monkeypatch):
    """profiles/traffic.txt rows are reported only while the recorded hash of
    their kernel sources matches the current one; comments are ignored."""
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.txt").write_text(
        "# comment line\nmact_cielab 191098880 aaaa  # trailing comment\nlut33_trilinear 195258368 bbbb\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_hash", lambda g: {"convert": "aaaa", "lut": "cccc"}[g])
    assert bench.traffic_table() == {"mact_cielab": 191098880.0}


def test_committed_traffic_rows_name_known_kernel_groups():
    for fname in ("traffic.txt", "instructions.txt"):
        rows = [l.split("#", 1)[0].split() for l in open(bench.os.path.join(bench.ROOT, "profiles", fname))]
        rows = [r for r in rows if r]
        assert rows and all(len(r) == 3 and bench.kernel_group(r[0]) in bench.KERNEL_FILES for r in rows)
        assert all(r[0] in {name for name, _, _ in bench.ROWS} for r in rows)


def test_instruction_figures_only_for_unchanged_kernel_sources(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "instructions.txt").write_text("exact_sct 150.5 aaaa\nlut17_tetra 90.4 bbbb\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_hash", lambda g: {"convert": "aaaa", "lut": "cccc"}[g])
    assert bench.instruction_table() == {"exact_sct": 150.5}


def test_issue_peak_is_lanes_times_schedulers_times_clock(tmp_path, monkeypatch):
    """The ALU roofline's peak: 152 SMs x 4 schedulers x 32 lanes x 2070 MHz
    = 40.29 T lane-instructions per second."""
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))   # no MEASURED_PEAKS.json: the nominal clock
    peak, kind = bench.issue_peak(152)
    assert abs(peak - 152 * 4 * 32 * 2070e6 / 1e12) < 1e-9 and "2070" in kind
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6700.0, "sm_max_mhz": 1965.0}')
    peak, kind = bench.issue_peak(152)
    assert abs(peak - 152 * 128 * 1965e6 / 1e12) < 1e-9 and "measured" in kind


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the oracle on the host cores and
    prints one JSON line with the contract's keys; it needs no GPU."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, bench.os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], capture_output=True, text=True, timeout=600,
                       cwd=bench.ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "dtype", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1 and d["warmup"] >= 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun only rank 0 runs the reference arm; another rank exits 0
    without work and prints nothing."""
    import subprocess
    import sys
    env = dict(bench.os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, bench.os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"], capture_output=True, text=True,
                       timeout=300, cwd=bench.ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]
