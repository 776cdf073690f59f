"""Pins of oracle/thermo.py (canonical thermodynamics from a DOS)."""
import math

import numpy as np

from oracle import exact_dos as X
from oracle.thermo import thermodynamics


def _dos_arrays(E, g, step):
    e0 = min(E)
    n = (max(E) - e0) // step + 1
    lng = np.full(n, -np.inf)
    for e, c in zip(E, X.ln_counts(g)):
        lng[(e - e0) // step] = c
    return lng, e0


def test_matches_direct_state_enumeration_ising_L4():
    N, L = 16, 4
    E, g = X.enumerate_dos(L)
    lng, e0 = _dos_arrays(E, g, 4)
    # Z by summing exp(-E/T) over all 2^16 states directly
    idx = np.arange(1 << N)
    right = np.array([(i // L) * L + (i % L + 1) % L for i in range(N)])
    down = np.array([((i // L + 1) % L) * L + i % L for i in range(N)])
    s = 1 - 2 * ((idx[:, None] >> np.arange(N)) & 1)
    Es = -(s * s[:, right]).sum(1) - (s * s[:, down]).sum(1)
    Ts = [0.7, 1.5, 2.269, 3.5, 10.0]
    th = thermodynamics(lng, e0, 4, Ts)
    for k, T in enumerate(Ts):
        w = np.exp(-(Es - Es.min()) / T)
        lnZ = math.log(w.sum()) - Es.min() / T
        U = (w * Es).sum() / w.sum()
        C = ((w * Es ** 2).sum() / w.sum() - U ** 2) / T ** 2
        assert abs(th[k, 0] - lnZ) < 1e-10 and abs(th[k, 1] - U) < 1e-9 and abs(th[k, 2] - C) < 1e-8


def test_identities_and_limits():
    E, g = X.ising_dos_kaufman(16)
    lng, e0 = _dos_arrays(E, g, 4)
    T = np.array([2.0, 2.2, 2.5])
    h = 1e-5
    th = thermodynamics(lng, e0, 4, T)
    beta = 1.0 / T
    lz_p = thermodynamics(lng, e0, 4, 1.0 / (beta + h))[:, 0]
    lz_m = thermodynamics(lng, e0, 4, 1.0 / (beta - h))[:, 0]
    assert np.allclose(th[:, 1], -(lz_p - lz_m) / (2 * h), rtol=1e-7)          # U = -d ln Z / d beta
    u_p = thermodynamics(lng, e0, 4, T + h)[:, 1]
    u_m = thermodynamics(lng, e0, 4, T - h)[:, 1]
    assert np.allclose(th[:, 2], (u_p - u_m) / (2 * h), rtol=1e-6)              # C = dU/dT
    lo, hi = thermodynamics(lng, e0, 4, [0.05, 1e6])
    assert abs(lo[1] - (-512)) < 1e-6 and abs(lo[0] - (512 / 0.05 + math.log(2))) < 1e-6   # ground state
    assert abs(hi[1]) < 1e-2 and abs(hi[0] - 256 * math.log(2)) < 1e-3                    # all 2^N states


def _golden_L32():
    import os

    E, g = [], []
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "ising_L32_exact_dos.txt")):
        if not line.startswith("#"):
            a, b = line.split()
            E.append(int(a))
            g.append(int(b))
    return E, g


def test_specific_heat_peak_near_exact_critical_points():
    E, g = _golden_L32()
    lng, e0 = _dos_arrays(E, g, 4)
    T = np.linspace(2.1, 2.5, 401)
    C = thermodynamics(lng, e0, 4, T)[:, 2]
    Tc = 2.0 / math.log(1.0 + math.sqrt(2.0))
    assert abs(T[np.argmax(C)] - Tc) < 0.05          # finite-size shift of a few per cent at L = 32
    Ep, gp = X.transfer_dos(4, "potts", 3)
    lngp, e0p = _dos_arrays(Ep, gp, 1)
    Cp = thermodynamics(lngp, e0p, 1, np.linspace(0.5, 1.5, 201))[:, 2]
    assert np.all(np.isfinite(Cp)) and Cp.max() > 0


# ------------------------------------------------------------- jackknife
def test_jackknife_closed_forms_for_shifted_runs():
    """Runs ln g + c_i: U and C do not depend on a constant shift, so their
    jackknife errors vanish; ln Z_(i) = ln Z + mean_{j != i} c_j is linear in
    the shifts, so its jackknife error is the standard error of the mean of
    the c_i, sqrt(sum (c - cbar)^2 / (R (R - 1))); F = -T ln Z and
    S = U/T + ln Z carry T times and once that error."""
    from oracle.thermo import jackknife

    E, g = X.enumerate_dos(4)
    lng, e0 = _dos_arrays(E, g, 4)
    c = np.array([0.3, -1.1, 0.45, 2.0, -0.7, 0.05])
    R = len(c)
    runs = lng[None, :] + c[:, None]
    Ts = np.array([1.0, 2.269, 5.0])
    est, err = jackknife(runs, e0, 4, Ts)
    sem = math.sqrt(((c - c.mean()) ** 2).sum() / (R * (R - 1)))
    ref = thermodynamics(lng + c.mean(), e0, 4, Ts)
    assert np.allclose(est, ref, rtol=1e-12, atol=1e-12)
    assert np.allclose(err[:, 1], 0.0, atol=1e-9) and np.allclose(err[:, 2], 0.0, atol=1e-9)
    assert np.allclose(err[:, 0], sem, rtol=1e-9)
    assert np.allclose(err[:, 3], Ts * sem, rtol=1e-9)
    assert np.allclose(err[:, 4], sem, rtol=1e-9)
    est1, err1 = jackknife(np.repeat(lng[None, :], 4, axis=0), e0, 4, Ts)
    assert np.array_equal(err1, np.zeros_like(err1))
    assert np.allclose(est1, thermodynamics(lng, e0, 4, Ts), rtol=1e-14, atol=0)


def test_jackknife_error_matches_the_spread_over_experiments():
    """Exact 4 x 4 Ising DOS plus independent N(0, 0.05^2) noise per bin and
    run; 300 experiments of R = 16 runs.  The mean jackknife error of U and C
    at T = 2.269 must match the standard deviation of their estimates over
    the experiments within 20%."""
    from oracle.thermo import jackknife

    E, g = X.enumerate_dos(4)
    lng, e0 = _dos_arrays(E, g, 4)
    fin = np.isfinite(lng)
    rng = np.random.default_rng(1)
    ests, errs = [], []
    for _ in range(300):
        runs = np.repeat(lng[None, :], 16, axis=0)
        runs[:, fin] += rng.normal(0.0, 0.05, size=(16, int(fin.sum())))
        est, err = jackknife(runs, e0, 4, [2.269])
        ests.append(est[0])
        errs.append(err[0])
    ests, errs = np.array(ests), np.array(errs)
    for q in (1, 2):
        ratio = errs[:, q].mean() / ests[:, q].std(ddof=1)
        assert 0.8 < ratio < 1.2, (q, ratio)
