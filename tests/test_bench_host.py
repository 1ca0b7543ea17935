"""Host logic of bench.py that needs no GPU: how the reference arm sizes its per-step sample
so that K + W oracle steps end within about two minutes, when the committed DRAM traffic of
the timed kernel applies, and the summary of the clock samples."""
import sys

import pytest


@pytest.fixture()
def bench(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    import bench as b
    return b


def _fake_oracle(t_fixed, per_cell):
    def oracle_mlups(nx, ny, rows, steps, kw, cols=None):
        cols = nx if cols is None else cols
        dt = steps * (t_fixed + per_cell * cols * rows)
        return cols * rows * steps / dt / 1e6, dt
    return oracle_mlups


def test_reference_window_whole_rows_while_they_fit(bench, monkeypatch):
    monkeypatch.setattr(bench, "oracle_mlups", _fake_oracle(0.0, 1e-5))
    # 8 whole rows of 1024 take 0.08192 s per step
    assert bench.reference_window(1024, 1024, 4, {}) == (1024, 1024)           # capped at ny
    cols, rows = bench.reference_window(1024, 1024, 200, {}, seconds=120.0)
    assert cols == 1024 and rows == int(8 * 0.6 / 0.08192)


def test_reference_window_square_when_rows_do_not_fit(bench, monkeypatch):
    t_fixed, per_cell = 4e-3, 1e-5
    monkeypatch.setattr(bench, "oracle_mlups", _fake_oracle(t_fixed, per_cell))
    nsteps = 20020
    cols, rows = bench.reference_window(1024, 1024, nsteps, {}, seconds=120.0)
    assert cols == rows and 8 <= cols < 1024
    per_step = t_fixed + per_cell * cols * rows
    assert per_step * nsteps <= 120.0 * 1.001                 # within the time asked for
    assert (t_fixed + per_cell * (cols + 1) ** 2) * nsteps > 120.0   # and the largest such square


def test_reference_window_never_below_the_smallest_lattice(bench, monkeypatch):
    monkeypatch.setattr(bench, "oracle_mlups", _fake_oracle(50e-3, 1e-5))
    assert bench.reference_window(1024, 1024, 20020, {}, seconds=120.0) == (8, 8)


class _Args:
    nx, ny, precision = 1024, 1024, "f32"


def test_committed_traffic_only_for_the_same_sources_and_workload(bench, monkeypatch, tmp_path):
    f = tmp_path / "summary.txt"
    body = "# header\nworkload: 1024x1024 f32\nsource_digest: %s\ndram_bytes_per_launch: 123456\n"
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    f.write_text(body % bench.csrc_digest())
    assert bench.committed_traffic(_Args) == 123456.0
    f.write_text(body % "0000000000000000")                  # counters taken on other sources
    assert bench.committed_traffic(_Args) is None
    f.write_text((body % bench.csrc_digest()).replace("1024x1024", "4096x4096"))
    assert bench.committed_traffic(_Args) is None            # another workload
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.txt"))
    assert bench.committed_traffic(_Args) is None


def test_clock_samples_summary(bench):
    class FakeProc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c = bench.Clocks(0)
    c.proc = FakeProc()
    c.lines = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1100.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    s = c.stop()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c.lines = ["0, 1500, 2070, 800, 0x8, Active, Not Active, Active, Not Active"]
    assert c.stop()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    c.lines = []
    assert c.stop() is None


def test_nvml_clock_samples_summary(bench):
    """Dense NVML samples: the median and the reasons of the samples inside the timed
    region; all samples when none falls inside."""
    s = [(0.9, 2070.0, 0), (1.0, 2055.0, 0x4), (1.5, 2070.0, 0x1), (2.5, 1500.0, 0x8)]
    out = bench.summarise_clock_samples(s, 2070.0, 1.0, 2.0)
    assert out["sm_mhz"] == 2062.5 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 2
    assert out["reasons"] == ["sw_power_cap"] and out["in_timed_region"]
    out = bench.summarise_clock_samples(s, 2070.0, 3.0, 4.0)
    assert out["samples"] == 4 and not out["in_timed_region"]
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert bench.summarise_clock_samples([], None) is None
