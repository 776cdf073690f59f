"""Pins the exact density-of-states routes of oracle/exact_dos.py against each
other and against closed-form counts.  Enumeration is the definition; the
transfer matrix and the Kaufman/Beale polynomial must reproduce it exactly."""
import math
import os

import numpy as np
import pytest

from oracle import exact_dos as X

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_ising_enumeration_transfer_kaufman_L4():
    a = X.enumerate_dos(4)
    assert a == X.transfer_dos(4)
    assert a == X.ising_dos_kaufman(4)


def test_ising_transfer_kaufman_L6():
    assert X.transfer_dos(6) == X.ising_dos_kaufman(6)


@pytest.mark.slow
def test_ising_transfer_kaufman_L8():
    assert X.transfer_dos(8) == X.ising_dos_kaufman(8)


@pytest.mark.parametrize("L", [4, 8, 16])
def test_ising_closed_form_counts(L):
    N = L * L
    E, g = X.ising_dos_kaufman(L)
    d = dict(zip(E, g))
    assert sum(g) == 2 ** N
    assert d[-2 * N] == 2 and d[2 * N] == 2              # two ground states, two Neel states
    assert (-2 * N + 4) not in d                         # one flip costs 8
    assert d[-2 * N + 8] == 2 * N                        # one flipped spin, either ground state
    assert d[-2 * N + 12] == 4 * N                       # an adjacent flipped pair (2 orientations)
    for e, c in d.items():
        assert d[-e] == c                                # g(E) = g(-E) on the bipartite torus
        assert (e + 2 * N) % 4 == 0


def test_ising_L32_golden_file():
    """The stored L = 32 table was written by tests/golden/make_golden.py from
    oracle.exact_dos only; re-check its exact identities."""
    path = os.path.join(GOLDEN, "ising_L32_exact_dos.txt")
    E, g = [], []
    for line in open(path):
        if line.startswith("#"):
            continue
        e, c = line.split()
        E.append(int(e))
        g.append(int(c))
    N = 1024
    assert sum(g) == 2 ** N
    d = dict(zip(E, g))
    assert d[-2 * N] == 2 and d[-2 * N + 8] == 2 * N and d[-2 * N + 12] == 4 * N
    assert all(d[-e] == c for e, c in d.items())


def test_potts_enumeration_vs_transfer():
    assert X.enumerate_dos(3, "potts", 3) == X.transfer_dos(3, "potts", 3)
    assert X.enumerate_dos(4, "potts", 2) == X.transfer_dos(4, "potts", 2)


def test_potts_q2_is_ising():
    # q = 2 Potts: E_potts = (E_ising - 2N) / 2
    Ep, gp = X.transfer_dos(4, "potts", 2)
    Ei, gi = X.enumerate_dos(4)
    assert dict(zip(Ep, gp)) == {(e - 32) // 2: c for e, c in zip(Ei, gi)}


@pytest.mark.slow
def test_potts_q10_L4_closed_forms():
    q, L = 10, 4
    N = L * L
    E, g = X.transfer_dos(L, "potts", q)
    d = dict(zip(E, g))
    assert sum(g) == q ** N
    assert d[-2 * N] == q
    for e in (-2 * N + 1, -2 * N + 2, -2 * N + 3):
        assert e not in d
    assert d[-2 * N + 4] == q * N * (q - 1)                # one spin changed
    assert d[-2 * N + 6] == q * 2 * N * (q - 1)            # adjacent pair, same new value
    assert d[-2 * N + 7] == q * 2 * N * (q - 1) * (q - 2)  # adjacent pair, two new values


def test_ea_enumeration_vs_transfer():
    rng = np.random.default_rng(7)
    for _ in range(2):
        J = rng.choice([-1, 1], size=32).astype(np.int8)
        a = X.enumerate_dos(4, "ea", couplings=J)
        assert a == X.transfer_dos(4, "ea", couplings=J)
        d = dict(zip(*a))
        assert sum(d.values()) == 2 ** 16
        assert all(d[-e] == c for e, c in d.items())    # bipartite symmetry holds for any couplings
        nneg = int((J < 0).sum())
        assert all((e + 32 - 2 * nneg) % 4 == 0 for e in d)


def test_ea_all_ferro_is_ising():
    J = np.ones(32, np.int8)
    assert X.enumerate_dos(4, "ea", couplings=J) == X.enumerate_dos(4)


def test_ln_counts_large():
    c = 3 * 2 ** 1500
    assert abs(X.ln_counts([c])[0] - (math.log(3) + 1500 * math.log(2))) < 1e-9
