"""The benchmark's roofline and error arithmetic on the CPU: the itemised operation counts of each
kernel form against the totals the design notes state (Kerr 3-D 518, Kerr 2-D 448, a = 0 362 per
in-grid step; 98 and 63 per predictor pass), the achieved fraction as counts x counters / time / peak,
and the spectrum-error rule max(1%, 3 combined sigma) on constructed spectra."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_operation_counts_per_form():
    assert bench.ops_grid_step("kerr", 3) == 518
    assert bench.ops_grid_step("kerr", 2) == 448
    assert bench.ops_grid_step("schw", 2) == 362
    assert bench.ops_pass("kerr") == 98 and bench.ops_pass("schw") == 63
    assert bench.ops_geodesic_step("kerr") == 178 and bench.ops_geodesic_step("schw") == 102


def test_fp64_roofline_is_counts_times_counters_over_time():
    st = {"n_steps_grid": 1_000_000, "n_iters_grid": 1_200_000, "n_events": 500, "grid_ms": 2.0,
          "init_ms": 0.5, "free_ms": 1.0}
    r = bench.fp64_roofline(st, "kerr", 3, 1.0e12, "k")
    ops = 518 * 1_000_000 + 98 * 1_200_000 + 30 * 500
    assert r["achieved"] == pytest.approx(ops / 2.0e-3 / 1e12)
    assert r["frac"] == pytest.approx(ops / 2.0e-3 / 1.0e12)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    # the a = 0 form counts fewer operations for the same counters
    assert bench.fp64_roofline(st, "schw", 2, 1.0e12, "k")["achieved"] < r["achieved"]


def test_spectrum_error_rule():
    rng = np.random.default_rng(3)
    ref = np.zeros((1, 200, 3))
    ref[..., 2] = rng.integers(100, 10000, (1, 200))
    ref[..., 0] = ref[..., 2] * 2.0
    ref[..., 1] = ref[..., 2] * 4.0 * 1e-6          # tiny Monte Carlo variance: the 1% branch decides
    lum, nb, nok = bench.spectrum_error(ref.copy(), ref)
    assert lum == 0.0 and nb == 200 and nok == 200
    off = ref.copy()
    off[0, 7, 0] *= 1.02                             # 2% off in one bin
    lum, nb, nok = bench.spectrum_error(off, ref)
    assert nok == 199 and lum > 0
    off[0, 7, 1] = (0.02 * ref[0, 7, 0]) ** 2        # ... unless 3 sigma covers it
    lum, nb, nok = bench.spectrum_error(off, ref)
    assert nok == 200
    sparse = ref.copy()
    sparse[0, :50, 2] = 3                            # bins with fewer than 16 superphotons are not compared
    assert bench.spectrum_error(sparse, ref)[1] == 150
