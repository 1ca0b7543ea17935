"""Host logic of bench.py that needs no GPU: how the reference arm sizes its per-step sample
so that K + W oracle steps end within about two minutes."""
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
