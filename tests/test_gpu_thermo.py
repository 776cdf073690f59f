"""rewl_thermo (canonical thermodynamics from ln g) on the GPU against the
oracle's numpy version, on the exact 32 x 32 Ising DOS and on a GPU Potts
solve."""
import os

import numpy as np
import pytest

from oracle.thermo import thermodynamics
from paper_1305_5615_gb300 import rewl

pytestmark = pytest.mark.gpu


def _golden():
    E, c = [], []
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "ising_L32_exact_dos.txt")):
        if not line.startswith("#"):
            a, b = line.split()
            E.append(int(a))
            c.append(int(b))
    lng = np.full(1025, -np.inf)
    for e, cc in zip(E, c):
        b = cc.bit_length()
        lng[(e + 2048) // 4] = np.log(float(cc)) if b < 1000 else np.log(float(cc >> (b - 60))) + (b - 60) * np.log(2)
    return lng


def test_thermo_matches_oracle_on_exact_ising_dos():
    lng = _golden()
    T = np.concatenate([np.linspace(0.3, 6.0, 300), [1e4]])
    got = rewl.rewl_thermo(lng, -2048, 4, T)
    ref = thermodynamics(lng, -2048, 4, T)
    assert np.allclose(got, ref, rtol=1e-10, atol=1e-9)
    Tc = 2.0 / np.log(1.0 + np.sqrt(2.0))
    assert abs(T[np.argmax(got[:-1, 2])] - Tc) < 0.05


def test_thermo_on_a_potts_solve():
    D = rewl.REWL("potts", 8, 4, 0.75, 2, 0.8, 1e-4, 5, q=10)
    assert D.step(0)
    g, e0, de = D.lng()
    T = np.linspace(0.4, 1.2, 81)
    assert np.allclose(rewl.rewl_thermo(g, e0, de, T), thermodynamics(g, e0, de, T), rtol=1e-10, atol=1e-9)
    with pytest.raises(rewl.RewlError):
        rewl.rewl_thermo(g, e0, de, [0.0])


def test_jackknife_matches_oracle_and_closed_forms():
    from oracle.thermo import jackknife

    lng = _golden()
    fin = np.isfinite(lng)
    rng = np.random.default_rng(3)
    runs = np.repeat(lng[None, :], 12, axis=0)
    runs[:, fin] += rng.normal(0.0, 0.02, size=(12, int(fin.sum())))
    runs[5, 7] = -np.inf            # a bin missing from one run is left out of every table
    T = np.linspace(1.5, 3.5, 41)
    est, err = rewl.rewl_thermo_jackknife(runs, -2048, 4, T)
    e_ref, r_ref = jackknife(runs, -2048, 4, T)
    assert np.allclose(est, e_ref, rtol=1e-10, atol=1e-9)
    assert np.allclose(err, r_ref, rtol=1e-7, atol=1e-9)
    # constant shifts: U and C exact, ln Z error = standard error of the shifts' mean
    c = rng.normal(0.0, 1.0, size=6)
    est, err = rewl.rewl_thermo_jackknife(lng[None, :] + c[:, None], -2048, 4, T)
    sem = np.sqrt(((c - c.mean()) ** 2).sum() / (6 * 5))
    assert np.allclose(err[:, 0], sem, rtol=1e-8) and np.allclose(err[:, 1:3], 0.0, atol=1e-6)
    with pytest.raises(rewl.RewlError):
        rewl.rewl_thermo_jackknife(runs[:1], -2048, 4, T)


def test_jackknife_over_independent_potts_solves():
    from oracle.thermo import jackknife

    runs = []
    for seed in range(4):
        D = rewl.REWL("potts", 8, 4, 0.75, 2, 0.8, 1e-4, 20 + seed, q=10)
        assert D.step(0)
        g, e0, de = D.lng()
        runs.append(g)
        D.close()
    T = np.linspace(0.5, 1.0, 26)
    est, err = rewl.rewl_thermo_jackknife(np.array(runs), e0, de, T)
    e_ref, r_ref = jackknife(np.array(runs), e0, de, T)
    assert np.allclose(est, e_ref, rtol=1e-10, atol=1e-9) and np.allclose(err, r_ref, rtol=1e-7, atol=1e-9)
    assert (err[:, 2] > 0).all()
