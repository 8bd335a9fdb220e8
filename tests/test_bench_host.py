"""Host pieces of bench.py (no GPU): the clock record parser, the algorithmic
bytes per lattice update and the ALU roofline arithmetic."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_clock_parser():
    out = "\n".join([
        "2070, 2070, 850.12, Not Active, Not Active, Not Active, Not Active",
        "2055, 2070, 1390.50, Not Active, Not Active, Not Active, Active",
        "2070, 2070, [N/A], Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "[N/A], 2070, 100.0, Not Active, Not Active, Not Active, Not Active",
    ])
    c = bench.ClockSampler.parse(out)
    assert c["samples"] == 3 and c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]
    hot = bench.ClockSampler.parse("1200, 2070, 1400, Active, Not Active, Active, Not Active")
    assert hot["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and hot["sm_mhz"] == 1200.0
    assert bench.ClockSampler.parse("")["sm_mhz"] is None


def test_bytes_per_lattice_update():
    """The roofline's algorithmic bytes B = 2 Q s_f + 2 s_rho (populations and
    the density read and written once), and the bytes the fused step moves
    (populations only; the density never leaves the chip)."""
    assert [bench.bytes_per_lu(s) for s in ("f16dev", "bf16dev", "f32", "f64")] == [88, 88, 160, 320]
    assert [bench.bytes_moved_per_lu(s) for s in ("f16dev", "bf16dev", "f32", "f64")] == [80, 80, 152, 304]
    assert bench.bytes_moved_per_lu("f16dev", q=9) == 40 and bench.bytes_moved_per_lu("f64", q=9) == 144


def test_alu_roofline_arithmetic():
    fp = bench.kernel_fingerprint()
    fma = {"f64": 1.25, "f32": 78.5}
    a = bench.alu_roofline(fp, "f16dev", 128, 27.0, fma)
    if a is None:
        pytest.skip("no flop count recorded for these kernel sources")
    assert a["achieved"] == pytest.approx(a["flop_per_lu"] * 27.0e9 / 1e12)
    assert a["frac"] == pytest.approx(a["achieved"] / 78.5)
    d = bench.alu_roofline(fp, "f64", 128, 1.115, fma)
    if d is None:
        pytest.skip("no float64 flop count recorded for these kernel sources")
    assert d["precision"] == "f64" and d["pipe_frac"] == pytest.approx(
        d["fp64_pipe_ops_per_lu"] * 1.115e9 / (1.25e12 / 2))
    assert bench.alu_roofline(fp, "f16dev", 128, 27.0, None) is None
    assert bench.alu_roofline("0" * 12, "f16dev", 128, 27.0, fma) is None


def test_oracle_table_on_tiny_workloads(monkeypatch):
    """bench.py --oracle-table logic on the host: every row timed on one core
    and on every core (spawned single-threaded processes), positive rates."""
    import bench
    monkeypatch.setattr(bench, "ORACLE_TABLE", {
        "tiny 2D": ("D2Q9", (1, 12, 10), "equilibrium", 0.55, 0.01, 1.0, "centre3", 2, 1),
        "tiny 3D": ("D3Q19", (6, 6, 8), "forcing", 0.55, 0.01, 1.0, "centre2", 1, 0),
    })
    monkeypatch.setattr(bench.os, "sched_getaffinity", lambda pid: {0, 1})
    res = bench.oracle_table()
    assert res["cores"] == 2 and set(res["rows"]) == {"tiny 2D", "tiny 3D"}
    for row in res["rows"].values():
        assert row["one_core_mlups"] > 0 and row["all_cores_mlups"] > 0 and row["cores"] == 2
