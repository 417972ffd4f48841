"""Host-side logic of the benchmark (CPU): clock sampling summary and throttle reasons,
the single-process rank combination, and the roofline denominators."""
import io
import subprocess

import bench


class _FakeProc:
    def __init__(self, lines, stdout):
        stdout.write("".join(lines))
        stdout.flush()

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _sample(monkeypatch, tmp_path, lines):
    monkeypatch.setenv("CHFSI_CLOCKS_CSV", str(tmp_path / "clocks_{rank}.csv"))
    monkeypatch.setattr(subprocess, "Popen", lambda args, stdout=None, stderr=None: _FakeProc(lines, stdout))
    s = bench.ClockSampler(3)
    assert s.path.endswith("clocks_3.csv")
    s.start()
    return s.stop()


def test_clock_summary_median_under_load_and_reasons(monkeypatch, tmp_path):
    idle = "0, 345, 2070, 120.5, 0x0, Not Active, Not Active, Not Active, Not Active\n"
    busy = "0, {mhz}, 2070, 980.0, 0x4, Not Active, Not Active, Not Active, {cap}\n"
    lines = [idle] + [busy.format(mhz=m, cap="Not Active") for m in (2070, 2055, 2070)]
    lines.append(busy.format(mhz=1980, cap="Active"))
    out = _sample(monkeypatch, tmp_path, lines)
    assert out["sm_max_mhz"] == 2070.0
    assert out["sm_mhz"] == 2062.5           # median of the loaded samples (idle one dropped)
    assert out["reasons"] == ["sw_power_cap"]
    assert out["samples"] == 5


def test_clock_summary_flags_thermal_and_hw_slowdown(monkeypatch, tmp_path):
    lines = ["0, 1500, 2070, 1300.0, 0x48, Active, Not Active, Active, Not Active\n"] * 3
    out = _sample(monkeypatch, tmp_path, lines)
    assert out["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples(monkeypatch, tmp_path):
    out = _sample(monkeypatch, tmp_path, ["garbage\n", "[N/A], [N/A]\n"])
    assert out["sm_mhz"] is None and out["reasons"] == ["no samples"]


def test_single_process_rank_combination_is_identity():
    assert bench.combine_ranks(123.5, 40) == (123.5, 40.0)


def test_peaks_are_measured_or_the_stated_fallback(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peaks, kind = bench._peaks()
    assert kind == "fallback"
    assert peaks == {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6768.1, "bf16_tflops_sustained": 1718.6}')
    peaks, kind = bench._peaks()
    assert kind == "measured" and peaks["bf16_tflops_sustained"] == 1718.6


def test_step_schedule_is_cyclic_with_one_cold_problem_per_pass():
    # K = N steps after W warm-up steps cover every problem once, exactly one of them cold
    N, W = 20, 3
    sched = bench.step_schedule(W, N, N)
    assert sorted(p for p, _ in sched) == list(range(N))
    assert sum(cold for _, cold in sched) == 1
    assert sched[0] == (3, False) and sched[N - W] == (0, True)
    assert bench.step_schedule(0, 3, 20) == [(0, True), (1, False), (2, False)]


def test_segments_split_where_the_sequence_starts_over():
    assert bench.segments(3, 20, 20) == [(3, 17, False), (0, 3, True)]
    assert bench.segments(0, 20, 20) == [(0, 20, True)]
    assert bench.segments(18, 45, 20) == [(18, 2, False), (0, 20, True), (0, 20, True), (0, 3, True)]
    assert sum(ln for _, ln, _ in bench.segments(7, 33, 10)) == 33


def test_summary_percentiles_of_per_eigenpair_errors():
    s = bench.summary([0.0, 1.0, 2.0, 3.0, 4.0])
    assert s == {"count": 5, "p50": 2.0, "p90": 3.6, "p99": 3.96, "max": 4.0}
    assert bench.summary([]) == {}
