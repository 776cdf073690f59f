"""Ising 256 x 256 (the largest 2D lattice the paper runs): bit-exact parity
with the oracle on eight windows x one walker for one block (100 sweeps of
65 536 trials per walker), and properties that hold at any size: reported
energy = energy recomputed from the configuration, walkers inside their
windows, sum H = trials, and ln g = H in the first iteration (ln f = 1)."""
import numpy as np
import pytest

from paper_1305_5615_gb300 import rewl
from parity_util import compare_states, make_pair, run_both

pytestmark = pytest.mark.gpu


def test_L256_eight_windows_bit_exact():
    O, D = make_pair("ising", 256, 8, 0.75, 1, 0.8, 1e-6, 4)
    assert (D.info["n_bins"], D.info["window_bins"]) == (65537, 23832)
    assert compare_states(O, D, "entry") == 0
    run_both(O, D, 1)
    assert compare_states(O, D, "1 block") == 0


def _ising_energy(words, L):
    spins = rewl.unpack_lattice(words, L, rewl.ISING).reshape(-1, L, L).astype(np.int32)
    s = 1 - 2 * spins
    return -(s * np.roll(s, -1, axis=2)).sum((1, 2)) - (s * np.roll(s, -1, axis=1)).sum((1, 2))


def test_L256_sixty_four_windows_properties():
    D = rewl.REWL("ising", 256, 64, 0.75, 4, 0.8, 1e-6, 0)
    info = D.info
    w = info["window_bins"]
    D.step(100)
    st = D.state()
    E = st["E"]
    assert np.array_equal(E, _ising_energy(st["lattice"], 256))
    a = np.arange(256) // 4
    lo = info["e_min"] + st["win_start"][a] * 4
    assert np.all((E >= lo) & (E <= lo + 4 * (w - 1)))
    assert np.all(st["H"].sum(1, dtype=np.int64) == 100 * 65536)
    assert np.array_equal(st["lng"], st["H"].astype(np.float64))
    assert st["near_ties"].sum() == 0
