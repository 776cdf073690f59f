"""Converged accuracy on the GPU against the exact density of states.

Ising 32 x 32, 16 windows at 75% overlap x 4 walkers, flatness 0.8, ln f
from 1 to below 1e-8 (27 iterations in every window), seeds 0..7.  The
exact g(E) is Kaufman's partition function expanded as a polynomial
(Beale's method), stored in tests/golden/ising_L32_exact_dos.txt by
tests/golden/make_golden.py from oracle.exact_dos only.

Measure: max relative error |ln g - ln g_exact| / ln g_exact over each half
of the estimate normalised at its own end -- the lower half (E <= 0) with
g(E_min) = 2, the upper half (E >= 0) with g(E_max) = 2 (the two fully
ordered and the two anti-ordered configurations).  A windowed WL estimate
is not symmetric even though the exact DOS is; each half is scored from the
end where ln g is known, since error accumulates across the joins.

Criterion: the mean ln g of the eight independent runs (the paper's
resampling over independent runs) is within 2e-3 in both halves.  A single
run is not: its largest relative error sits at the lowest levels
(E_min + 8 .. E_min + 20, where ln g is only 7.6 .. 15) and scatters from
run to run by +-0.03 in ln g, i.e. 0.8e-3 .. 5e-3 relative; each run is held
to 6e-3 and its numbers are printed.  The eight seeds run together through
the request server (each result is bit-identical to a solve alone;
tests/test_gpu_serving.py)."""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ising_L32_exact_dos.txt")
SEEDS = list(range(8))


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


def accuracy(g, e0, de, lnx):
    """Max relative error of each half, normalised at its own end, and the
    max absolute deviation after the best shift."""
    fin = np.isfinite(lnx)
    E = e0 + de * np.arange(len(g))
    lo = fin & (E <= 0)
    hi = fin & (E >= 0)
    top = np.nonzero(fin)[0][-1]
    g_lo = g - g[0] + lnx[0]            # g(E_min) = 2
    g_hi = g - g[top] + lnx[top]        # g(E_max) = 2
    rel_lo = float(np.max(np.abs(g_lo[lo] - lnx[lo]) / lnx[lo]))
    rel_hi = float(np.max(np.abs(g_hi[hi] - lnx[hi]) / lnx[hi]))
    d = g[fin] - lnx[fin]
    return rel_lo, rel_hi, float(np.max(np.abs(d - d.mean())))


@pytest.fixture(scope="module")
def solved():
    from paper_1305_5615_gb300 import rewl

    S = rewl.RewlServer(device_bytes=8 << 30, max_running=len(SEEDS))
    ids = [S.submit("ising", 32, 16, 0.75, 4, 0.8, 1e-8, sd) for sd in SEEDS]
    while True:
        st = S.run(1)
        if st["running"] == 0 and st["queued"] == 0:
            break
    out = []
    for rid in ids:
        assert S.poll(rid)["state"] == rewl.REQ_DONE
        out.append(S.result(rid))
    S.close()
    return out


@pytest.mark.gpu
def test_ising_L32_reaches_exact_dos_within_2e3(solved):
    worst_lo = worst_hi = 0.0
    lnx = None
    for sd, (g, e0, de) in zip(SEEDS, solved):
        lnx = _exact_ln(e0, de, len(g))
        fin = np.isfinite(lnx)
        assert np.array_equal(np.isfinite(g), fin), sd   # every reachable level visited, no other
        rel_lo, rel_hi, absd = accuracy(g, e0, de, lnx)
        print("seed %d: max rel. error E<=0 %.3e, E>=0 %.3e; max |d ln g| after best shift %.3f" % (
            sd, rel_lo, rel_hi, absd))
        worst_lo, worst_hi = max(worst_lo, rel_lo), max(worst_hi, rel_hi)
        # normalisation of rewl_get_lng: sum_E g(E) = 2^N
        mx = g[fin].max()
        assert abs(mx + math.log(np.exp(g[fin] - mx).sum()) - 1024 * math.log(2)) < 1e-9
    print("worst single run: E<=0 %.3e, E>=0 %.3e" % (worst_lo, worst_hi))
    g0, e0, de = solved[0]
    mean = np.mean([g for g, _, _ in solved], axis=0)
    m_lo, m_hi, m_abs = accuracy(mean, e0, de, lnx)
    print("mean of the %d runs: E<=0 %.3e, E>=0 %.3e; max |d ln g| after best shift %.3f" % (
        len(SEEDS), m_lo, m_hi, m_abs))
    assert m_lo <= 2e-3 and m_hi <= 2e-3, (m_lo, m_hi)
    assert worst_lo <= 6e-3 and worst_hi <= 6e-3, (worst_lo, worst_hi)


def test_accuracy_measure_on_the_exact_dos():
    """The measure itself: zero on the exact DOS under any constant shift,
    and a perturbation of one level shows up in the half that holds it."""
    e0, de, n = -2048, 4, 1025
    lnx = _exact_ln(e0, de, n)
    g = np.where(np.isfinite(lnx), lnx + 3.25, -np.inf)
    assert max(accuracy(g, e0, de, lnx)) < 1e-13   # rounding of the shift only
    g2 = g.copy()
    g2[100] += 0.5   # E = -1648: lower half only
    rel_lo, rel_hi, _ = accuracy(g2, e0, de, lnx)
    assert rel_lo == pytest.approx(0.5 / lnx[100]) and rel_hi < 1e-13
