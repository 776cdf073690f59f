"""Ising 128 x 128: bit-exact parity with the oracle on a few walkers, and the
full 128 windows x 32 walkers (4096 walkers, 501-bin windows) checked through
properties that hold at any size (the oracle would need minutes per block):
every reported energy equals the energy recomputed from the configuration,
every walker stays in its window, sum H = its trials, and in the first
iteration (ln f = 1) ln g = H exactly."""
import numpy as np
import pytest

from paper_1305_5615_gb300 import rewl
from parity_util import compare_states, make_pair, run_both

pytestmark = pytest.mark.gpu


def test_L128_four_windows_bit_exact():
    O, D = make_pair("ising", 128, 4, 0.75, 1, 0.8, 1e-6, 3)
    assert D.info["window_bins"] == 9363
    assert compare_states(O, D, "entry") == 0
    run_both(O, D, 2)
    assert compare_states(O, D, "2 blocks") == 0


def _ising_energy(words, L):
    spins = rewl.unpack_lattice(words, L, rewl.ISING).reshape(-1, L, L).astype(np.int32)
    s = 1 - 2 * spins
    return -(s * np.roll(s, -1, axis=2)).sum((1, 2)) - (s * np.roll(s, -1, axis=1)).sum((1, 2))


def test_L128_full_size_properties():
    D = rewl.REWL("ising", 128, 128, 0.75, 32, 0.8, 1e-6, 0)
    info = D.info
    assert (info["n_bins"], info["window_bins"]) == (16385, 501)
    D.step(100)
    st = D.state()
    E = st["E"]
    assert np.array_equal(E, _ising_energy(st["lattice"], 128))
    a = np.arange(4096) // 32
    lo = info["e_min"] + st["win_start"][a] * 4
    assert np.all((E >= lo) & (E <= lo + 4 * (501 - 1)))
    assert np.all(st["H"].sum(1, dtype=np.int64) == 100 * 128 * 128)
    assert np.array_equal(st["lng"], st["H"].astype(np.float64))
    assert st["near_ties"].sum() == 0
