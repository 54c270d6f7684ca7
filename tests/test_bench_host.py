"""Host-side pieces of bench.py that need no GPU: the algorithmic term counts behind the
roofline figures, the ncu-traffic lookup and the clock-sample parsing."""
import itertools
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def brute_count(rho, d):
    r = int(np.ceil(rho)) + 1
    c = 0
    for o in itertools.product(range(-r, r + 1), repeat=d):
        o2 = sum(k * k for k in o)
        if 0 < o2 < rho * rho:
            c += 1
    return c


@pytest.mark.parametrize("d", [1, 2, 3])
def test_ball_counts_match_brute_force(d):
    n = 64
    rng = np.random.default_rng(d)
    rhos = np.concatenate([rng.uniform(1.0, 6.0, 12), [2.0, 3.0, 4.0, 4.5]])   # ties at integers
    got = bench.ball_counts(rhos / n, n, d)
    want = [brute_count(r, d) for r in rhos]
    assert list(got) == want


def test_ball_counts_of_the_workloads():
    # 1-D delta = 0.05 on 4096 nodes: 204 cells each side; 3-D delta = 4h: 250 (strict ball,
    # the offsets at distance exactly 4 excluded)
    assert bench.ball_counts(np.array([0.05]), 4096, 1)[0] == 408
    assert bench.ball_counts(np.array([4.0 / 256]), 256, 3)[0] == 250
    # 2-D delta = 8h (peridynamic workload): the 197 lattice points with |o| <= 8 (Gauss circle
    # count) minus the origin and the four at distance exactly 8
    assert bench.ball_counts(np.array([8.0 / 512]), 512, 2)[0] == 192 == brute_count(8.0, 2)


def test_traffic_is_looked_up_by_exact_kernel_name():
    r = bench._alu_roof("k_direct2d_x2<16,TY> (direct FP32)", 1e9, 1.0, 80.0, "x")
    assert r["traffic"] == bench.PROFILED_TRAFFIC["k_direct2d_x2"]
    assert bench._alu_roof("k_direct2d_x2s (symmetric)", 1e9, 1.0, 80.0, "x")["traffic"] is None
    assert r["frac"] == pytest.approx(1e9 / 1e-3 / 1e12 / 80.0, rel=1e-3)


def test_clock_summary_parses_samples_and_reasons():
    c = bench.ClockSampler()
    c.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage"]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
