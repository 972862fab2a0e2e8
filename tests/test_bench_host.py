"""Host logic of bench.py (no GPU): the clock sampler's parsing of nvidia-smi rows, and the byte
and throughput formulas the bench line reports."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _clocks_from(rows):
    c = bench.Clocks.__new__(bench.Clocks)
    import tempfile
    c.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
    c.p = None
    c.f.write("\n".join(rows) + "\n")
    return c.stop()


def test_clock_rows_give_the_median_and_the_active_reasons():
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
            "garbage line"]
    out = _clocks_from(rows)
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    out = _clocks_from(["0, 1200, 2070, 700, 0x8, Active, Not Active, Active, Not Active"])
    assert out["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_no_clock_rows_reads_as_unsampled():
    out = _clocks_from([])
    assert out["sm_mhz"] is None and out["reasons"] == ["unsampled"] and out["samples"] == 0


def test_spmv_bytes_formula():
    class Info:
        nnz_blocks = 100
        n_nodes = 10
    # nnzb (dim^2 b + 4) + 4 (n_rows + 1) + 2 b n_dof + n_dof
    assert bench._spmv_bytes(Info, 2, 8) == 100 * (4 * 8 + 4) + 4 * 11 + 2 * 8 * 20 + 20
    assert bench._spmv_bytes(Info, 3, 4) == 100 * (9 * 4 + 4) + 4 * 11 + 2 * 4 * 30 + 30


def test_job_value_counts_every_rank():
    assert bench.job_value(4, 1000, 10, 2.0) == 4 * 1000 * 10 / 0.002 / 1e9
