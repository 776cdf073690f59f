"""Pins the oracle's joining of window fragments (paper, paragraph after
Eq. (1): join where the inverse temperatures beta = d ln g/dE agree best)."""
import math

import numpy as np

from oracle import exact_dos as X
from oracle.join import join_windows, normalise


def _exact_L8():
    E, g = X.ising_dos_kaufman(8)
    lnx = np.full(65, -np.inf)
    for e, v in zip(E, X.ln_counts(g)):
        lnx[(e + 128) // 4] = v
    return lnx


def _split(lnx, starts, w, offsets):
    tabs = []
    for s, off in zip(starts, offsets):
        t = np.zeros(w)
        for b in range(w):
            v = lnx[s + b]
            t[b] = v + off if np.isfinite(v) else 0.0   # 0 = never visited
        tabs.append(t)
    return tabs


def test_join_recovers_exact_dos_from_shifted_fragments():
    lnx = _exact_L8()
    starts, w = [0, 9, 18, 27], 38
    tabs = _split(lnx, starts, w, [3.0, 17.25, -0.5 + 60.0, 101.0])
    g = normalise(join_windows(tabs, starts, w, 65), 64, 2)
    fin = np.isfinite(lnx)
    assert np.array_equal(np.isfinite(g), fin)
    assert np.abs(g[fin] - lnx[fin]).max() < 1e-9


def test_join_point_is_best_beta_match():
    # two windows, the upper one carries a kink: beta agrees only at one bin
    lnx = _exact_L8()
    starts, w = [0, 20], 45
    tabs = _split(lnx, starts, w, [5.0, 5.0])
    kink = np.zeros(w)
    kink[:12] = 0.3 * (12 - np.arange(12))   # distorts beta of the upper piece below its bin 12
    tabs[1] = np.where(tabs[1] > 0, tabs[1] + kink, 0.0)
    g = join_windows(tabs, starts, w, 65)
    fin = np.isfinite(lnx)
    assert np.array_equal(np.isfinite(g), fin)
    # with the join above the kink the exact shape is kept everywhere
    diff = g[fin] - lnx[fin]
    assert np.abs(diff - diff[0]).max() < 1e-9


def test_normalise_sums_to_total_count():
    lnx = _exact_L8()
    g = normalise(lnx + 12.5, 64, 2)
    fin = np.isfinite(g)
    mx = g[fin].max()
    assert abs(mx + math.log(np.exp(g[fin] - mx).sum()) - 64 * math.log(2)) < 1e-10
    gp = normalise(np.array([1.0, 2.0, -np.inf, 0.5]), 4, 10)
    assert abs(math.log(np.exp(gp[np.isfinite(gp)]).sum()) - 4 * math.log(10)) < 1e-12
