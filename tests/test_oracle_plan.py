"""Pins of oracle/plan.py (run-time balanced windows, Fig. 1b) and of the
oracle's unequal-window support."""
import math

import numpy as np
import pytest

from oracle import OracleREWL, exact_dos as X
from oracle.plan import balanced_windows, bin_costs, check, partition


def test_costs_from_a_pre_run_by_hand():
    # windows [0..5] (first merge after 100 sweeps) and [3..8] (after 400): rho = 10/6 and 20/6
    rho = bin_costs([100, 400], [0, 3], [6, 6], 9)
    want = [10 / 6] * 3 + [(10 / 6 + 20 / 6) / 2] * 3 + [20 / 6] * 3
    assert np.allclose(rho, want, rtol=1e-15)
    with pytest.raises(ValueError):
        bin_costs([100, -1], [0, 3], [6, 6], 9)      # a window without a first merge


def test_partitions_by_hand():
    # uniform cost, B = 20, h = 2, o = 1/2: lam = 40/3 bins -> [0, 13] and [6, 19]
    assert partition([1.0] * 20, 2, 0.5) == ([0, 6], [14, 14])
    # cost 1 below bin 10, 3 from bin 10: U(b) = b, then 10 + 3 (b - 10); T = 40, lam = 80/3
    # window 0 ends at the first b with U(b+1) >= 26.67 -> b = 15; window 1 starts at the
    # last b with U(b) <= 13.33 -> b = 11
    assert partition([1.0] * 10 + [3.0] * 10, 2, 0.5) == ([0, 11], [16, 9])
    assert partition([2.0] * 7, 1, 0.75) == ([0], [7])


def test_windows_carry_equal_cost():
    """On random costs every window's sum of rho equals lam within the cost
    of its two end bins."""
    rng = np.random.default_rng(4)
    for h, o in ((4, 0.75), (9, 0.75), (16, 0.6)):
        rho = list(rng.uniform(0.2, 5.0, size=600))
        starts, widths = partition(rho, h, o)
        T = sum(rho)
        lam = T / (1 + (h - 1) * (1 - o))
        for s, w in zip(starts, widths):
            tot = sum(rho[s:s + w])
            assert abs(tot - lam) <= rho[s] + rho[s + w - 1] + 1e-9


def test_partition_checks():
    check([0, 2, 5], [4, 5, 3], 8)
    for starts, widths in (([0, 2], [4, 5]), ([1, 2], [4, 6]), ([0, 5], [4, 3]), ([0, 0], [4, 8]), ([0, 2], [2, 6])):
        with pytest.raises(ValueError):
            check(starts, widths, 8)


def test_unequal_windows_converge_to_the_exact_dos():
    """Ising L=4 over three unequal windows (bins 0-4, 2-10 and 8-16 of 17):
    the joined ln g equals the exact enumeration within WL accuracy, and each
    walker stays inside its own window.  (WL on a 4 x 4 lattice saturates
    near 0.1 in max |ln g - ln g_exact|; a wrong window bound or join is off
    by O(1).)"""
    R = OracleREWL("ising", 4, 3, 0.75, 2, 0.8, 1e-6, 2, window_starts=[0, 2, 8], window_widths=[5, 9, 9])
    win = R.windows()
    assert list(win["width"]) == [5, 9, 9] and R.w == 9
    for _ in range(3000):
        done = R.run_blocks(10)
        st = R.walkers()
        lo = R.e_min + 4 * np.repeat(win["start"], 2)
        hi = lo + 4 * (np.repeat(win["width"], 2) - 1)
        assert ((st["E"] >= lo) & (st["E"] <= hi)).all()
        if done:
            break
    assert done
    E, g = X.enumerate_dos(4)
    lng = R.joined_lng()
    ex = np.full(len(lng), -np.inf)
    for e, c in zip(E, g):
        ex[(e - R.e_min) // 4] = math.log(c)
    fin = np.isfinite(ex)
    assert np.array_equal(np.isfinite(lng), fin)
    assert np.abs(lng[fin] - ex[fin]).max() < 0.2
    assert (R.windows()["first_iter"] > 0).all()


def test_balanced_plan_from_an_oracle_pre_run():
    R = OracleREWL("potts", 6, 4, 0.75, 2, 0.8, 1e-3, 1, q=5)
    while not (R.windows()["first_iter"] > 0).all():
        R.run_blocks(10)
    win = R.windows()
    starts, widths = balanced_windows(win["first_iter"], win["start"], win["width"], R.n_bins, 4, 0.75)
    check(starts, widths, R.n_bins)
    B = OracleREWL("potts", 6, 4, 0.75, 2, 0.8, 1e-3, 1, q=5, window_starts=starts, window_widths=widths)
    assert list(B.windows()["start"]) == starts and list(B.windows()["width"]) == widths
