"""Pins the oracle's 1/t rule (Belardinelli and Pereyra, PRE 75, 046701
(2007)), which the paper names, in the paragraph that introduces its
replica-exchange scheme, as one of the WL rules the exchange works with.

* schedule: with every energy revisited between checks, the stage-0 halvings,
  the switch to stage 1 and the stage-1 halvings happen at the sweep clocks
  derived by hand from the rule (t = trials per energy level);
* stage 1 keeps ln f a power of two with 1/t <= ln f < 2/t (one check of lag);
* the stage-0 test (every visited bin seen again) on hand-made histograms;
* exactness: every merged ln g is a multiple of 2^-(k + log2 m);
* the defining property of the rule against exact enumeration of the 4 x 4
  Ising lattice: the error of the flatness rule saturates as ln f -> 0, the
  error of the 1/t rule keeps falling.
"""
import math

import numpy as np

from oracle import OracleREWL, exact_dos as X


def _trace(R, n_checks):
    """(sweep clock, ln f, stage, merges) of window 0 after each check."""
    out = []
    spf = 1000
    for _ in range(n_checks):
        R.run_blocks(spf // 100)
        w = R.windows()
        out.append((R.info()["sweep_clock"], float(w["lnf"][0]), int(w["phase"][0]), int(w["iteration"][0])))
        if w["done"][0]:
            break
    return out


def test_schedule_ising_L4_single_window():
    """4 x 4 Ising, one window of w = 17 bins, N = 16, checks every 1000 sweeps:
    t = 16 * clock / 17.  Stage 0 halves ln f = 2^-k at each check while
    t >= 2^(k+1), i.e. at clocks 1000 ... 13000 (k -> 1 ... 13); at clock 14000
    t = 13176 < 2^14, so the window merges, keeps ln f = 2^-13 and enters
    stage 1.  Stage 1 halves at the first check with t >= 2^(k+1):
    clock >= 17 * 2^14 / 16 = 17408 -> 18000, then >= 34816 -> 35000,
    >= 69632 -> 70000, >= 139264 -> 140000."""
    R = OracleREWL("ising", 4, 1, 0.75, 1, 0.8, 2.0 ** -16, 0, wl_rule="1/t")
    assert (R.w, R.N) == (17, 16)
    tr = _trace(R, 200)
    changes = [tr[0]] + [b for a, b in zip(tr, tr[1:]) if (a[1], a[2]) != (b[1], b[2])]
    want = [(1000 * n, 2.0 ** -n, 0, n) for n in range(1, 14)] + [(14000, 2.0 ** -13, 1, 14)] + [
        (18000, 2.0 ** -14, 1, 15), (35000, 2.0 ** -15, 1, 16), (70000, 2.0 ** -16, 1, 17),
        (140000, 2.0 ** -17, 1, 18)]
    assert changes == want
    assert R.windows()["done"][0] == 1 and tr[-1][0] == 140000


def test_stage_one_follows_one_over_t_from_above():
    """Six windows x 2 walkers of a 6 x 6 Ising lattice: in stage 1 every
    window keeps 1 <= ln f * t < 2 (t + check period) / t at each check."""
    R = OracleREWL("ising", 6, 3, 0.75, 2, 0.8, 2.0 ** -15, 3, wl_rule="1/t")
    N, w = R.N, R.w
    seen_stage1 = False
    for _ in range(400):
        done = R.run_blocks(10)
        win = R.windows()
        clock = R.info()["sweep_clock"]
        t = clock * N / w
        for a in range(R.h):
            if win["phase"][a] == 1 and not win["done"][a]:
                seen_stage1 = True
                lnf = win["lnf"][a]
                assert math.frexp(lnf)[0] == 0.5                      # a power of two
                assert lnf * t >= 1.0
                assert lnf * t < 2.0 * (clock + 1000) / clock
        if done:
            break
    assert seen_stage1 and done


def test_stage_zero_test_on_hand_made_histograms():
    R = OracleREWL("ising", 4, 1, 0.75, 1, 0.8, 1e-4, 0, wl_rule="1/t")
    w = R.w
    lng = np.zeros(w)
    lng[2:9] = 1.5                  # visited bins 2..8; the others never visited
    R.set_walker_lng(0, lng)
    H = np.zeros(w, np.uint32)
    H[2:9] = 1
    R.set_walker_H(0, H)
    assert R.walker_all_seen(0)
    H[5] = 0                        # one visited bin not seen again
    R.set_walker_H(0, H)
    assert not R.walker_all_seen(0)
    H[5] = 7
    H[12] = 0                       # unvisited bins do not count
    R.set_walker_H(0, H)
    assert R.walker_all_seen(0)
    R.set_walker_lng(0, np.zeros(w))
    assert not R.walker_all_seen(0)  # nothing visited yet


def test_merged_ln_g_stays_exact():
    R = OracleREWL("potts", 4, 2, 0.75, 4, 0.8, 2.0 ** -12, 5, q=3, wl_rule="1/t")
    for _ in range(3000):
        done = R.run_blocks(10)
        win = R.windows()
        lng = R.walkers()["lng"]
        for a in range(R.h):
            k = -math.frexp(win["lnf"][a])[1] + 1
            scaled = lng[a * 4:(a + 1) * 4] * 2.0 ** (k + 2)     # m = 4
            assert np.array_equal(scaled, np.floor(scaled))
        if done:
            break
    assert done


def _max_err(R, E, g):
    lng = R.joined_lng()
    ex = np.full(len(lng), -np.inf)
    for e, c in zip(E, g):
        ex[(e - R.e_min) // R.e_step] = math.log(c)
    fin = np.isfinite(ex)
    assert np.array_equal(np.isfinite(lng), fin)
    return float(np.abs(lng[fin] - ex[fin]).max())


def test_one_over_t_error_keeps_falling_where_flatness_saturates():
    """4 x 4 Ising, one walker, seeds 0..3, run to ln f = 2^-20.  Measured
    mean max |ln g - ln g_exact|: flatness rule 0.093 at 2^-14 and 0.071 at
    2^-20 (saturated); 1/t rule 0.068 at 2^-14 and 0.0076 at 2^-20.  Bounds:
    the 1/t error at 2^-20 below 0.02 and below a third of the flatness
    rule's, and below half its own at 2^-14."""
    E, g = X.enumerate_dos(4)
    res = {}
    for rule in ("flat", "1/t"):
        R = [OracleREWL("ising", 4, 1, 0.75, 1, 0.8, 2.0 ** -20, s, wl_rule=rule) for s in range(4)]
        errs = {}
        for k in (14, 20):
            e = []
            for r in R:
                while r.windows()["lnf"][0] >= 2.0 ** -k and not r.run_blocks(10):
                    pass
                e.append(_max_err(r, E, g))
            errs[k] = float(np.mean(e))
        res[rule] = errs
    assert res["1/t"][20] < 0.02
    assert res["1/t"][20] < res["flat"][20] / 3
    assert res["1/t"][20] < res["1/t"][14] / 2
