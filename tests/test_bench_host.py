"""Host arithmetic of bench.py that needs no GPU: the exact rain integral the whole-storm
record compares the applied rain with (Appendix C's triangular hyetograph, whose volume
per unit area is i_a T_d / 2, and the catchment's double-peak storm by hand), and the
step kernel's traffic record (scaling and its lapse when the kernel's sources change)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2406_14933_gb300 import inputs  # noqa: E402


def test_rain_integral_of_the_triangular_hyetograph():
    # Appendix C: T_d = 1000 s, i_a = 0.0732 mm/s at t_a = 250 s
    rt, rr = [0.0, 250.0, 1000.0], [0.0, 0.0732e-3, 0.0]
    assert bench.rain_integral(rt, rr, 1000.0) == pytest.approx(0.0732e-3 * 1000.0 / 2.0, rel=1e-14)
    assert bench.rain_integral(rt, rr, 5000.0) == pytest.approx(0.0732e-3 * 1000.0 / 2.0, rel=1e-14)
    # the rising limb alone, and a window that cuts it: i(t) = i_a t / t_a
    assert bench.rain_integral(rt, rr, 250.0) == pytest.approx(0.0732e-3 * 250.0 / 2.0, rel=1e-14)
    assert bench.rain_integral(rt, rr, 100.0) == pytest.approx(0.0732e-3 / 250.0 * 100.0 ** 2 / 2.0, rel=1e-14)
    assert bench.rain_integral(rt, rr, 0.0) == 0.0


def test_rain_integral_of_the_catchment_storm():
    """(0, 0) - (30 min, 80) - (60, 20) - (90, 120) - (120, 0) mm/h: 40 + 50 + 70 + 60 mm/h
    over four half hours, 110 mm in all; 36.25 mm by t = 2700 s."""
    sc = inputs.carved_catchment(rows=64, cols=64)
    rt, rr = [float(x) for x in sc.rain_t], [float(x) for x in sc.rain_r]
    mm_h = 1e-3 / 3600.0
    assert bench.rain_integral(rt, rr, sc.t_end) == pytest.approx(110.0 * mm_h * 3600.0, rel=1e-12)
    assert bench.rain_integral(rt, rr, 2700.0) == pytest.approx(36.25 * mm_h * 3600.0, rel=1e-12)


def test_rain_integral_outside_the_table_is_zero():
    assert bench.rain_integral([100.0, 200.0], [1.0, 1.0], 150.0) == pytest.approx(50.0)
    assert bench.rain_integral([100.0, 200.0], [1.0, 1.0], 50.0) == 0.0
    assert bench.rain_integral([100.0, 200.0], [1.0, 3.0], 1e9) == pytest.approx(200.0)



def test_traffic_record_scales_by_cells_and_lapses_when_a_source_changes(tmp_path, monkeypatch):
    """The step kernel's DRAM traffic comes from a committed record of one ncu capture,
    keyed by a hash of the kernel's sources: per cell (read + write) / cells, times the
    cells of the timed window; null once any of those sources differs from the hashed
    ones, or when the record is missing."""
    import hashlib
    for src in bench.TRAFFIC_SOURCES:
        dst = tmp_path / src
        dst.parent.mkdir(parents=True, exist_ok=True)
        dst.write_bytes((src + " v1\n").encode())
    h = hashlib.sha256()
    for src in bench.TRAFFIC_SOURCES:
        h.update((tmp_path / src).read_bytes())
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "step_strip_kernel__traffic.txt").write_text(
        "# a record\n"
        f"kernel_sources_sha256 {h.hexdigest()}\n"
        "cells 1000\n"
        "dram_bytes_read 30000\n"
        "dram_bytes_write 8800\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._read_traffic(1000) == pytest.approx(38800.0)
    assert bench._read_traffic(16777216) == pytest.approx(38.8 * 16777216)
    (tmp_path / bench.TRAFFIC_SOURCES[-1]).write_bytes(b"a changed header\n")
    assert bench._read_traffic(1000) is None
    (tmp_path / "profiles" / "step_strip_kernel__traffic.txt").unlink()
    assert bench._read_traffic(1000) is None
