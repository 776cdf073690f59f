"""Pins the oracle's WL walk for the q = 10 Potts model (the paper's Potts
benchmark model) against closed forms of the lowest levels of its density of
states on the periodic 8 x 8 lattice, N = 64 sites, 2N bonds, E = -(number of
satisfied bonds):

* E = -2N: the q uniform states;
* E = -2N + 4: one site changed, q N (q - 1) states;
* E = -2N + 5: unreachable (one changed site breaks 4 bonds, two break 6 or more);
* E = -2N + 6: two neighbouring sites changed to the same new value, q 2N (q - 1);
* E = -2N + 7: two neighbouring sites changed to two different new values,
  q 2N (q - 1)(q - 2).

The oracle runs to ln f < 1e-5 with 4 windows x 2 walkers and four seeds
(about 20 s).  The measured WL errors of the three ratios are at most 0.15 per
seed and 0.03 for the mean over the seeds.  An energy change that miscounts a
bond puts states on E = -2N + 5 or moves whole levels, which fails here."""
import math

import numpy as np

from oracle import OracleREWL

N, Q = 64, 10
EXACT = np.array([math.log(N * (Q - 1)), math.log(2 * N * (Q - 1)), math.log(2 * N * (Q - 1) * (Q - 2))])


def test_potts_q10_L8_low_levels_match_closed_forms():
    errs = []
    for seed in range(4):
        O = OracleREWL("potts", 8, 4, 0.75, 2, 0.8, 1e-5, seed, q=Q)
        while not O.run_blocks(10):
            pass
        g = O.joined_lng()
        at = lambda E: g[(E - O.e_min) // O.e_step]  # noqa: E731
        assert O.e_min == -2 * N and O.e_step == 1
        assert not np.isfinite(at(-2 * N + 5))
        assert all(np.isfinite(at(E)) for E in (-2 * N, -2 * N + 4, -2 * N + 6, -2 * N + 7))
        assert abs(at(-2 * N) - math.log(Q)) < 0.3
        errs.append(np.array([at(-2 * N + 4), at(-2 * N + 6), at(-2 * N + 7)]) - at(-2 * N) - EXACT)
    errs = np.array(errs)
    assert np.abs(errs).max() < 0.3
    assert np.abs(errs.mean(0)).max() < 0.1
