"""Converged accuracy on the GPU against the exact density of states.

Ising 32 x 32, 16 windows at 75% overlap x 4 walkers, flatness 0.8, ln f
from 1 to below 1e-8 (27 iterations in every window), seed 0.  The exact
g(E) is Kaufman's partition function expanded as a polynomial (Beale's
method), stored in tests/golden/ising_L32_exact_dos.txt by
tests/golden/make_golden.py from oracle.exact_dos only.

Criterion: with ln g normalised so that g(E_min) = 2 (the two ground
states), max over E <= 0 of |ln g - ln g_exact| / ln g_exact <= 2e-3.  The
exact DOS is symmetric, so that half determines it; over the full range the
error of a windowed WL run accumulates across the joins toward E_max, where
ln g = ln 2, and a relative measure there is not meaningful.  The run is
deterministic (counter-based draws), so the measured error is a fixed number."""
import math
import os

import numpy as np
import pytest

from paper_1305_5615_gb300 import rewl

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ising_L32_exact_dos.txt")


def _exact_ln(e0, de, n):
    out = np.full(n, -np.inf)
    for line in open(GOLDEN):
        if line.startswith("#"):
            continue
        e, c = line.split()
        c = int(c)
        b = c.bit_length()
        out[(int(e) - e0) // de] = math.log(c) if b < 1000 else math.log(c >> (b - 60)) + (b - 60) * math.log(2.0)
    return out


def test_ising_L32_reaches_exact_dos_within_2e3():
    D = rewl.REWL("ising", 32, 16, 0.75, 4, 0.8, 1e-8, 0)
    assert D.step(0)   # to completion
    st = D.state()
    assert (st["iteration"] == 27).all()
    g, e0, de = D.lng()
    lnx = _exact_ln(e0, de, len(g))
    fin = np.isfinite(lnx)
    assert np.array_equal(np.isfinite(g), fin)   # every reachable level visited, no other
    gn = g - g[0] + lnx[0]                        # g(E_min) = 2
    half = fin & (e0 + de * np.arange(len(g)) <= 0)
    rel = np.abs(gn[half] - lnx[half]) / lnx[half]
    assert rel.max() <= 2e-3, rel.max()
    # normalisation of rewl_get_lng: sum_E g(E) = 2^N
    mx = g[fin].max()
    assert abs(mx + math.log(np.exp(g[fin] - mx).sum()) - 1024 * math.log(2)) < 1e-9
