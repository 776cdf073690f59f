"""Pins of the oracle's 3D +-J model (the paper's 12 x 12 x 12 spin glass):
its energy against an independent numpy sum over the 3N bonds of the cube,
converged densities of states against exact enumeration, the closed-form
low-energy degeneracies of the 3D ferromagnet (all J = +1), and the coupling
draws and energy grid."""
import math

import numpy as np

from oracle import OracleREWL, exact_dos as X


def _numpy_energy(spins, J, L):
    right, down, back = X._bonds3(L)
    s = 1 - 2 * spins.astype(np.int64)
    J = J.reshape(-1, 3).astype(np.int64)
    return int(-(J[:, 0] * s * s[right]).sum() - (J[:, 1] * s * s[down]).sum() - (J[:, 2] * s * s[back]).sum())


def test_energy_is_the_sum_over_the_cube_bonds():
    R = OracleREWL("ea3d", 4, 2, 0.75, 1, 0.8, 1e-3, 5)
    J = R.couplings()
    assert J.shape == (3 * 64,) and set(np.unique(J)) == {-1, 1}
    rng = np.random.default_rng(2)
    for _ in range(20):
        s = rng.integers(0, 2, size=64).astype(np.uint8)
        assert R.energy(s) == _numpy_energy(s, J, 4)
    R.run_blocks(3)
    st = R.walkers()
    for W in range(2):
        assert st["E"][W] == _numpy_energy(st["spins"][W], J, 4)


def _converged_error(R, E, g):
    for _ in range(50000):
        if R.run_blocks(10):
            break
    lng = R.joined_lng()
    ex = np.full(len(lng), -np.inf)
    for e, c in zip(E, g):
        ex[(e - R.e_min) // R.e_step] = math.log(c)
    fin = np.isfinite(ex)
    assert np.array_equal(np.isfinite(lng), fin)
    return float(np.abs(lng[fin] - ex[fin]).max())


def test_L2_glass_and_ferromagnet_converge_to_enumeration():
    J = np.random.default_rng(0).choice([-1, 1], size=24).astype(np.int8)
    R = OracleREWL("ea3d", 2, 1, 0.75, 2, 0.8, 1e-6, 3, couplings=J)
    # WL on 8 spins saturates near 0.1 in max |ln g - ln g_exact|; a wrong bond is off by O(1)
    assert _converged_error(R, *X.enumerate_dos(2, "ea3d", couplings=J)) < 0.15
    F = OracleREWL("ea3d", 2, 2, 0.75, 2, 0.8, 1e-6, 4, couplings=np.ones(24, np.int8))
    assert _converged_error(F, *X.enumerate_dos(2, "ea3d")) < 0.15


def test_ferromagnet_L4_low_energy_degeneracies():
    """4 x 4 x 4 cube, J = +1: E0 = -3N = -192 (g = 2); one flipped spin breaks
    6 bonds (E0 + 12, g = 2N); two neighbours break 10 (E0 + 20, g = 2 * 3N);
    two apart break 12 (E0 + 24, g = 2 (N(N-1)/2 - 3N)); nothing at E0 + 4,
    E0 + 8, E0 + 16.  (WL to ln f = 1e-5 on this lattice: ratios within about
    0.1 over seeds; a wrong coordination moves whole levels.)"""
    R = OracleREWL("ea3d", 4, 4, 0.75, 2, 0.8, 1e-5, 7, couplings=np.ones(192, np.int8))
    assert R.e_min == -192
    for _ in range(50000):
        if R.run_blocks(10):
            break
    lng = R.joined_lng()
    g0 = lng[0]
    assert abs(g0 - math.log(2)) < 0.3                  # normalised to sum g = 2^64
    assert abs(lng[3] - g0 - math.log(64)) < 0.2
    assert abs(lng[5] - g0 - math.log(192)) < 0.2
    assert abs(lng[6] - g0 - math.log(64 * 63 // 2 - 192)) < 0.2
    assert not np.isfinite(lng[1]) and not np.isfinite(lng[2]) and not np.isfinite(lng[4])


def test_drawn_couplings_and_the_energy_grid():
    R = OracleREWL("ea3d", 8, 2, 0.75, 1, 0.8, 1e-3, 99)
    J = R.couplings()
    assert abs((J < 0).mean() - 0.5) < 0.05
    n_neg = int((J < 0).sum())
    assert R.e_max == -R.e_min and R.e_min >= -3 * R.N and (R.e_min + 3 * R.N - 2 * n_neg) % 4 == 0
    win = R.windows()
    assert win["start"][0] == 0 and win["start"][-1] + win["width"][-1] == R.n_bins
