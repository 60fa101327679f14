"""bench.py's per-iteration statistics of a solve's iteration log, on a
hand-built log whose answers are known (no GPU)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

NAMES = ("outer", "inner", "mu", "rho", "E0", "theta", "phi", "alpha_p", "alpha_d",
         "delta_w", "factorizations", "refine_steps", "precision", "accepted",
         "backtracks", "ms")


def _log(rows):
    h = np.zeros((len(rows), len(NAMES)))
    for r, (nf, prec, refine, ms) in enumerate(rows):
        h[r, NAMES.index("factorizations")] = nf
        h[r, NAMES.index("precision")] = prec
        h[r, NAMES.index("refine_steps")] = refine
        h[r, NAMES.index("ms")] = ms
    return h


def test_iteration_stats_split_by_factorizations_and_precision():
    import bench
    # 10 leading iterations that must be skipped (huge times), then 6 with
    # one factorization (6 ms) and 4 with two (10 ms); the first 5 counted
    # ones in FP32 (precision 1, 4 refinement steps), the rest FP64 (0, 0)
    lead = [(1, 1, 0, 1000.0)] * 10
    body = [(1, 1, 4, 6.0)] * 5 + [(1, 0, 0, 6.0)] + [(2, 0, 0, 10.0)] * 4
    s = bench.iteration_stats(NAMES, _log(lead + body), prec_fp32=1, prec_fp64=0)
    assert s["iteration_ms_mean_10_end"] == (6 * 6.0 + 4 * 10.0) / 10
    assert s["iterations_per_s_mean_10_end"] == 1e3 / 7.6
    assert s["iteration_ms_median_10_end"] == 6.0
    assert s["iteration_ms_median_by_factorizations"] == {
        "1": {"iterations": 6, "ms_median": 6.0}, "2": {"iterations": 4, "ms_median": 10.0}}
    p = s["iteration_ms_mean_by_precision"]
    assert p["fp32"] == {"iterations": 5, "ms_mean": 6.0, "refine_steps_mean": 4.0}
    assert p["fp64"] == {"iterations": 5, "ms_mean": (6.0 + 4 * 10.0) / 5,
                         "refine_steps_mean": 0.0}


def test_iteration_stats_short_and_empty_logs():
    import bench
    # fewer than ten iterations: all of them count
    s = bench.iteration_stats(NAMES, _log([(1, 0, 0, 4.0), (3, 0, 1, 8.0)]), 1, 0)
    assert s["iteration_ms_mean_10_end"] == 6.0
    assert set(s["iteration_ms_mean_by_precision"]) == {"fp64"}
    assert bench.iteration_stats(NAMES, np.zeros((0, len(NAMES))), 1, 0) == {}
