"""Pins the REWL oracle against what the paper and the mathematics fix.

* window partition: hand-derived widths and starts (paper, Fig. 1a: equal
  windows, overlap o = 75%);
* state invariants: incremental energy = recomputed energy; walkers stay in
  their windows; in the first iteration ln g = H * ln f0 exactly; H sums equal
  the attempts since the last reset; after a merge all walkers of a window
  share one ln g (paper, paragraph after Eq. (1));
* flatness: the min >= flatness * mean rule on hand-made histograms;
* Eq. (1): with ln g frozen (ln f = 0) the WL moves plus exchanges must sample
  the product distribution g(E_i)/g_i(E_i) * g(E_j)/g_j(E_j) -- detailed
  balance of the exchange (checked against exact enumeration);
* convergence: the joined, normalised ln g equals the exact DOS within the
  statistical error for Ising, +-J and Potts lattices.
"""
import math

import numpy as np
import pytest

from oracle import OracleREWL, exact_dos as X


def _exact_ln(E_exact, g_exact, e_min, e_step, n_bins):
    out = np.full(n_bins, -np.inf)
    ln = X.ln_counts(g_exact)
    for e, v in zip(E_exact, ln):
        out[(e - e_min) // e_step] = v
    return out


# ---------------------------------------------------------------- partition
def test_partition_ising_L8_four_windows():
    R = OracleREWL("ising", 8, 4, 0.75, 2, 0.8, 1e-6, 0)
    assert (R.n_bins, R.w) == (65, 38)
    assert list(R.windows()["start"]) == [0, 9, 18, 27]
    assert R.windows()["start"][-1] + R.w - 1 == R.n_bins - 1


def test_partition_ising_L32_sixteen_windows():
    R = OracleREWL("ising", 32, 16, 0.75, 1, 0.8, 1e-8, 0)
    st = R.windows()["start"]
    assert (R.n_bins, R.w) == (1025, 216)
    assert st[0] == 0 and st[-1] + R.w - 1 == 1024
    # starts are k*(B-w)/(h-1) = k*809/15 rounded half up
    assert list(st[:4]) == [0, 54, 108, 162] and st[8] == 431
    ov = [(st[k] + R.w - st[k + 1]) / R.w for k in range(15)]
    assert min(ov) >= 0.75 - 1.0 / R.w


def test_partition_potts_L32_thirtytwo_windows():
    R = OracleREWL("potts", 32, 32, 0.75, 1, 0.8, 1e-8, 0, q=10)
    assert (R.n_bins, R.w) == (2049, 235)
    assert R.e_min == -2048 and R.e_max == 0 and R.e_step == 1


def test_single_window_covers_range():
    R = OracleREWL("ising", 4, 1, 0.75, 2, 0.8, 1e-3, 3)
    assert R.w == R.n_bins == 17 and list(R.windows()["start"]) == [0]


# --------------------------------------------------------------- invariants
def test_state_invariants_during_first_iteration():
    R = OracleREWL("ising", 8, 4, 0.75, 2, 0.8, 1e-6, 5, sweeps_per_flat_check=100000)
    R.run_blocks(7)
    st = R.walkers()
    win = R.windows()
    assert R.info()["sweep_clock"] == 700
    for W in range(8):
        a = W // 2
        assert st["E"][W] == R.energy(st["spins"][W])
        lo = R.e_min + win["start"][a] * R.e_step
        assert lo <= st["E"][W] <= lo + (R.w - 1) * R.e_step
        # iteration 0, ln f0 = 1: every visit adds exactly 1.0
        assert np.array_equal(st["lng"][W], st["H"][W].astype(np.float64))
        assert int(st["H"][W].sum()) == 700 * R.N


def test_merge_shares_ln_g_and_resets_H():
    R = OracleREWL("ising", 4, 2, 0.75, 4, 0.8, 1e-4, 11, sweeps_per_exchange=10, sweeps_per_flat_check=100)
    it0 = R.windows()["iteration"].copy()
    for _ in range(400):
        R.run_blocks(10)   # ends on a flatness check
        win = R.windows()
        if (win["iteration"] > it0).any():
            break
    a = int(np.argmax(win["iteration"] > it0))
    st = R.walkers()
    lng = st["lng"][a * 4:(a + 1) * 4]
    assert all(np.array_equal(lng[0], lng[k]) for k in range(4))
    assert not st["H"][a * 4:(a + 1) * 4].any()
    assert win["lnf"][a] == 0.5 ** win["iteration"][a]


def test_merge_value_is_the_walker_order_mean():
    """The merged ln g is the mean of the window's m estimators (merge
    paragraph: the estimators are averaged), summed in walker order and
    divided by m, bit for bit.  ln g is frozen (ln f = 0 in every window) at
    four distinct hand-made tables per window and H at a large flat level, so
    the first check finds every walker flat and merges: copying one walker's
    table, dropping a walker, averaging another window's walkers or summing in
    another order all change the bits."""
    m = 4
    R = OracleREWL("ising", 4, 2, 0.75, m, 0.8, 1e-4, 17, sweeps_per_exchange=10, sweeps_per_flat_check=100)
    rng = np.random.default_rng(5)
    win = R.windows()
    tables = {}
    for a in range(R.h):
        R.set_window_lnf(a, 0.0)
        for k in range(m):
            W = a * m + k
            t = np.zeros(R.w)
            # distinct per walker, positive on the window's bins (all count as visited), not dyadic
            t[:win["width"][a]] = rng.uniform(1.0, 50.0, size=win["width"][a]) * (1.0 + 0.37 * k) + 0.1 * a
            tables[W] = t
            R.set_walker_lng(W, t)
            R.set_walker_H(W, np.full(R.w, 10 ** 6, np.uint32))
    R.run_blocks(10)  # 100 sweeps: one flatness check
    win = R.windows()
    assert (win["iteration"] == 1).all()
    st = R.walkers()
    for a in range(R.h):
        s = tables[a * m].copy()
        for k in range(1, m):
            s = s + tables[a * m + k]
        mean = s / float(m)
        for k in range(m):
            assert np.array_equal(st["lng"][a * m + k].view(np.uint64), mean.view(np.uint64)), (a, k)
        # a plausible mistake changes the value: one walker's table, or a sum without walker m-1
        assert not np.array_equal(mean, tables[a * m])
        assert not np.array_equal(mean, (s - tables[a * m + m - 1]) / float(m - 1))
    assert not st["H"].any()


def test_phase_schedule_counts_exchanges():
    R = OracleREWL("ising", 8, 4, 0.75, 2, 0.8, 1e-6, 2, sweeps_per_exchange=50, sweeps_per_flat_check=1000)
    R.run_blocks(6)
    c = R.counters()
    # rounds 0,2,4 pair windows (0,1),(2,3); rounds 1,3,5 pair (1,2); m = 2 pairs each
    assert list(c["x_tried"]) == [6, 6, 6, 0]
    assert R.info()["xround"] == 6


# ---------------------------------------------------------------- flatness
def test_flatness_rule():
    R = OracleREWL("ising", 8, 4, 0.75, 2, 0.8, 1e-6, 0, sweeps_per_flat_check=100000)
    lng = np.zeros(R.w)
    lng[:10] = 1.0
    R.set_walker_lng(0, lng)
    H = np.zeros(R.w, np.uint32)
    H[:10] = 100
    R.set_walker_H(0, H)
    assert R.walker_is_flat(0)
    H[3] = 78      # 78*10 = 780 < 0.8*978 = 782.4
    R.set_walker_H(0, H)
    assert not R.walker_is_flat(0)
    H[3] = 79      # 790 >= 0.8*979 = 783.2
    R.set_walker_H(0, H)
    assert R.walker_is_flat(0)
    H[20] = 0      # bins never visited (ln g = 0) do not count
    lng[3] = 0.0
    H[3] = 0
    R.set_walker_lng(0, lng)
    R.set_walker_H(0, H)
    assert R.walker_is_flat(0)
    R.set_walker_lng(0, np.zeros(R.w))
    assert not R.walker_is_flat(0)   # nothing visited is not flat


def test_flatness_on_the_exact_four_fifths_boundary():
    """Flatness 0.8 is tested in FP64 as min H * n >= 0.8 * sum H.  On the
    exact rational boundary 5 min H n = 4 sum H it agrees with the exact test
    (flat), and one count below the boundary it is not flat."""
    R = OracleREWL("ising", 8, 4, 0.75, 2, 0.8, 1e-6, 0, sweeps_per_flat_check=100000)
    lng = np.zeros(R.w)
    lng[:10] = 1.0
    R.set_walker_lng(0, lng)
    # n = 10 visited bins, min H = 80, sum H = 5 * 80 * 10 / 4 = 1000
    H = np.zeros(R.w, np.uint32)
    H[:10] = [80, 80, 80, 80, 80, 120, 120, 120, 120, 120]
    assert 5 * 80 * 10 == 4 * int(H.sum())
    R.set_walker_H(0, H)
    assert R.walker_is_flat(0)
    H[9] += 1          # sum 1001: 5 * 80 * 10 < 4 * 1001
    R.set_walker_H(0, H)
    assert not R.walker_is_flat(0)
    # larger counts, still on the boundary: min H = 4k, n = 8, sum H = 40k
    lng[:] = 0.0
    lng[:8] = 2.0
    R.set_walker_lng(0, lng)
    for kk in (1, 7, 12345, 999983):
        H = np.zeros(R.w, np.uint32)
        H[:8] = 4 * kk
        H[0] += 8 * kk   # sum = 32k + 8k = 40k = 5 * (4k) * 8 / 4
        R.set_walker_H(0, H)
        assert 5 * int(H[:8].min()) * 8 == 4 * int(H.sum())
        assert R.walker_is_flat(0), kk
        H[1] += 1
        R.set_walker_H(0, H)
        assert not R.walker_is_flat(0), kk


# ----------------------------------------------------- Eq. (1): detailed balance
def _frozen_pair_histograms(oracle_cls, n_blocks, seed):
    R = oracle_cls("ising", 4, 2, 0.75, 1, 0.8, 1e-8, seed, sweeps_per_exchange=1,
                   sweeps_per_flat_check=1000000000)
    E_ex, g_ex = X.enumerate_dos(4)
    lnx = _exact_ln(E_ex, g_ex, R.e_min, R.e_step, R.n_bins)
    st = R.windows()["start"]
    lng_tables = []
    for a, tilt in ((0, -0.25), (1, 0.25)):   # both windows favour the overlap
        loc = np.zeros(R.w)
        for b in range(R.w):
            gb = st[a] + b
            e = R.e_min + gb * R.e_step
            base = lnx[gb] if np.isfinite(lnx[gb]) else 0.0
            loc[b] = base + tilt * e / 4.0 + 40.0
        R.set_walker_lng(a, loc)
        R.set_window_lnf(a, 0.0)
        lng_tables.append(loc)
    hist = np.zeros((R.w, R.w))
    for _ in range(n_blocks):
        R.run_blocks(1)
        E = R.walkers()["E"]
        hist[(E[0] - R.e_min) // R.e_step - st[0], (E[1] - R.e_min) // R.e_step - st[1]] += 1
    # expected: independent product of g(E)/g_a(E) restricted to each window
    p = []
    for a in range(2):
        v = np.zeros(R.w)
        for b in range(R.w):
            gb = st[a] + b
            if np.isfinite(lnx[gb]):
                v[b] = math.exp(lnx[gb] - lng_tables[a][b])
        p.append(v / v.sum())
    return hist / hist.sum(), np.outer(p[0], p[1]), R.counters()


def test_exchange_detailed_balance_eq1():
    emp, exp, c = _frozen_pair_histograms(OracleREWL, 100000, 3)
    acc = c["x_accepted"][0] / c["x_tried"][0]
    assert 0.05 < acc < 0.95, acc         # the exchange is exercised
    mask = exp > 0.01
    # marginals and joint agree within sampling noise (correlated samples)
    assert np.abs(emp.sum(1) - exp.sum(1)).max() < 0.012
    assert np.abs(emp.sum(0) - exp.sum(0)).max() < 0.012
    assert np.abs(emp[mask] - exp[mask]).max() < 0.012


# ------------------------------------------------------------- convergence
def _max_abs_error(R, E_ex, g_ex):
    g = R.joined_lng()
    lnx = _exact_ln(E_ex, g_ex, R.e_min, R.e_step, R.n_bins)
    fin = np.isfinite(lnx)
    assert np.array_equal(np.isfinite(g), fin)   # visited bins = reachable bins
    return np.abs(g[fin] - lnx[fin]).max()


def _run(R, limit=20000):
    for _ in range(limit):
        if R.run_blocks(10):
            return
    raise AssertionError("did not converge")


def test_converges_ising_L4():
    R = OracleREWL("ising", 4, 2, 0.75, 2, 0.8, 1e-6, 1)
    _run(R)
    assert _max_abs_error(R, *X.enumerate_dos(4)) < 0.08


def test_converges_ising_L8_four_windows():
    R = OracleREWL("ising", 8, 4, 0.75, 2, 0.8, 1e-6, 0)
    _run(R)
    assert (R.windows()["iteration"] == 20).all()
    assert _max_abs_error(R, *X.ising_dos_kaufman(8)) < 0.2


def test_converges_ea_L4_given_couplings():
    J = np.random.default_rng(21).choice([-1, 1], size=32).astype(np.int8)
    R = OracleREWL("ea", 4, 2, 0.75, 2, 0.8, 1e-6, 4, couplings=J)
    E_ex, g_ex = X.enumerate_dos(4, "ea", couplings=J)
    # the grid reaches from the descent's lowest energy on down to -2N (nothing locked out)
    assert R.e_min <= min(E_ex) and R.e_max == -R.e_min and R.e_min >= -2 * R.N and (min(E_ex) - R.e_min) % 4 == 0
    _run(R)
    assert _max_abs_error(R, E_ex, g_ex) < 0.08


def test_converges_ea_L8_drawn_couplings():
    """+-J 8 x 8 with couplings drawn from the seed, four windows over the range
    the descent lays out (reaching on to -2N): the walk finds every reachable
    level, the ground state included, and nothing else, and ln g matches the
    transfer-matrix DOS of the same couplings (measured max error 0.085)."""
    R = OracleREWL("ea", 8, 4, 0.75, 2, 0.8, 1e-6, 5)
    E_ex, g_ex = X.transfer_dos(8, "ea", couplings=R.couplings())
    assert R.e_min == -2 * R.N < min(E_ex)
    _run(R)
    assert _max_abs_error(R, E_ex, g_ex) < 0.2


def test_converges_potts_q3_L4():
    R = OracleREWL("potts", 4, 2, 0.75, 2, 0.8, 1e-6, 2, q=3)
    _run(R)
    assert _max_abs_error(R, *X.transfer_dos(4, "potts", 3)) < 0.12


def test_couplings_drawn_from_seed_are_balanced():
    R = OracleREWL("ea", 16, 2, 0.75, 1, 0.8, 1e-3, 99)
    J = R.couplings()
    assert set(np.unique(J)) == {-1, 1}
    assert abs((J < 0).mean() - 0.5) < 0.05
    assert R.e_max == -R.e_min and (R.e_min + 2 * R.N - 2 * int((J < 0).sum())) % 4 == 0


def test_invalid_arguments():
    with pytest.raises(RuntimeError):
        OracleREWL("ising", 8, 4, 1.5, 2, 0.8, 1e-6, 0)
    with pytest.raises(RuntimeError):
        OracleREWL("potts", 8, 4, 0.75, 2, 0.8, 1e-6, 0, q=17)
    with pytest.raises(RuntimeError):
        OracleREWL("ising", 8, 4, 0.75, 2, 0.8, 1e-6, 0, couplings=np.ones(128, np.int8))
    with pytest.raises(RuntimeError):
        OracleREWL("ising", 8, 4, 0.75, 2, 0.8, 1e-6, 0, sweeps_per_exchange=30, sweeps_per_flat_check=100)


def test_threaded_block_sweeps_equal_the_single_threaded_run():
    """The oracle's threaded driver (disjoint walker ranges of each block swept
    on several host threads, then the block's exchange and flatness check on
    one) gives the same state, bit for bit, as orc_run_blocks."""
    A = OracleREWL("ising", 8, 4, 0.75, 2, 0.8, 1e-6, 23, sweeps_per_exchange=50, sweeps_per_flat_check=200)
    B = OracleREWL("ising", 8, 4, 0.75, 2, 0.8, 1e-6, 23, sweeps_per_exchange=50, sweeps_per_flat_check=200)
    for _ in range(5):
        A.run_blocks(8)
        B.run_blocks(8, threads=3)
    wa, wb = A.walkers(), B.walkers()
    for k in wa:
        assert np.array_equal(wa[k].view(np.uint8), wb[k].view(np.uint8)), k
    for k, v in A.windows().items():
        assert np.array_equal(v, B.windows()[k]), k
    for k, v in A.counters().items():
        assert np.array_equal(v, B.counters()[k]), k
    assert A.info() == B.info()
    assert (A.windows()["iteration"] > 0).any()   # flatness checks and merges happened
