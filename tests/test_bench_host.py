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


def test_assembly_bytes_scale_the_tangent_part_with_the_plastic_elements():
    class Info:
        n_int, n_elem, n_nodes, nnz_blocks = 700, 100, 250, 2000
    full = bench._assembly_bytes(Info, 2, 6, 4, 8, 1.0)
    none = bench._assembly_bytes(Info, 2, 6, 4, 8, 0.0)
    half = bench._assembly_bytes(Info, 2, 6, 4, 8, 0.5)
    # the plastic elements' slot map and K blocks (read and written once) are the only difference
    assert full - none == 100 * 36 * 4 + 2000 * 4 * 8 * 2
    assert abs(half - (none + full) / 2) < 1e-6


def test_chebyshev_bytes_average_the_zero_start_step():
    class Info:
        nnz_blocks, n_nodes = 3000, 400
    n = 800
    step0 = 400 * 16 + n + 12 * n                     # no matrix: inverse, mask, b read; d, x written
    later = 3000 * 20 + 401 * 4 + 400 * 16 + n + 20 * n
    assert bench._cheb0_bytes(Info, 2, deg=1) == step0
    assert bench._cheb0_bytes(Info, 2, deg=2) == (step0 + later) / 2
    assert bench._cheb0_bytes(Info, 2, deg=3) == (step0 + 2 * later) / 3
