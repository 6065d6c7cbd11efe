"""Host-side pieces of bench.py on CPU: the clock record that decides whether
a timed run is kept (throttle reasons, median SM clock), the algorithmic
bytes of the HBM rooflines, and the oracle's closed loop that the CPU
baseline and the reference arm time."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _sampler(lines):
    c = bench.ClockSampler(0)
    c.lines = list(lines)
    return c


def test_clock_summary_reports_median_and_throttle_reasons():
    # index, clocks.sm, clocks.max.sm, power, active, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 2055, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "garbage line",
             "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = _sampler(lines).summary()
    assert s["sm_mhz"] == 2055.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    s = _sampler(lines + ["0, 1500, 2070, 800, 0x8, Active, Not Active, Active, Not Active"]).summary()
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert _sampler([]).summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_hbm_rooflines_use_the_algorithmic_bytes():
    st = {"n_total": 1000, "m_total": 800, "nnz_L": 50000}
    ph = {"ms_eval": 0.01, "ms_assemble": 0.03, "ms_solve": 0.05}
    r = bench.hbm_rooflines(st, ph, latency_bound=True)
    ea, so = r["eval_assembly"], r["solves"]
    assert ea["algorithmic_bytes"] == 8 * (1000 + 5 * 800) + 8 * 50000 + 8 * 1000
    assert so["algorithmic_bytes"] == 16 * 50000
    assert ea["achieved"] == pytest.approx(ea["algorithmic_bytes"] / 0.04e-3 / 1e9)
    assert so["achieved"] == pytest.approx(16 * 50000 / 0.05e-3 / 1e9)
    assert "note" in ea and "note" in so
    if ea["peak"]:
        assert ea["frac"] == pytest.approx(ea["achieved"] / ea["peak"])


def test_oracle_closed_loop_is_bounded_and_converges():
    wl = {"N": 12, "Nf": 5, "T": 20, "seed": 1, "resolves": 5}
    times, iters = bench.run_oracle_loop(wl, budget_s=30.0, max_steps=3)
    assert len(times) == 3 and all(t > 0 for t in times)
    assert all(0 < i < 30 for i in iters)


def test_oracle_batch_loop_restarts_every_instance_from_its_own_solution():
    """The CPU leg of the batch: cold solves, then warm closed-loop re-solves
    of every instance on host threads; one thread and two give the same
    iteration counts (the instances are independent)."""
    import numpy as np
    import paper_2606_04725_gb300.inputs as I
    hz = np.array([20, 24, 16], dtype=np.int32)
    x0s = np.stack([I.distillation_x0(12, 5, seed=30 + i) for i in range(3)])
    sps = np.array([0.78, 0.8, 0.82])
    t2, it2, _ = bench.oracle_batch_loop(hz, x0s, sps, 12, 5, steps=2, threads=2)
    t1, it1, _ = bench.oracle_batch_loop(hz, x0s, sps, 12, 5, steps=2, threads=1)
    assert len(t2) == 2 and all(t > 0 for t in t2)
    assert it1 == it2 and all(len(s) == 3 and all(0 < i < 30 for i in s) for s in it2)


def test_closed_loop_index_points_at_x1_and_u1():
    import numpy as np
    hz = [3, 5]
    N = 4
    ix, iu = bench.closed_loop_index(hz, N)
    n0 = N + 3 * (N + 1)
    assert list(ix) == [4, 5, 6, 7, n0 + 4, n0 + 5, n0 + 6, n0 + 7]
    assert list(iu) == [8, n0 + 8]
    assert np.array_equal(bench.packed_setpoints(hz, [0.9, 0.95]), [0.9] * 3 + [0.95] * 5)
