"""Canonical thermodynamics from a density of states (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper, opening paragraph: Wang-Landau sampling gives thermodynamic quantities,
the free energy included, at any temperature from one simulation.  With
k_B = 1, beta = 1/T and w(E) = g(E) exp(-beta E):
    ln Z = ln sum_E w(E),  U = <E>,  C = beta^2 <(E - U)^2>,
    F = -T ln Z,  S = (U - F) / T.
Written plainly with numpy in FP64 (largest term factored out of the sum).

Parity: pinned by tests/test_oracle_thermo.py against direct enumeration of
all states, thermodynamic identities (U = -d ln Z / d beta, C = dU/dT), the
limits T -> 0 and T -> infinity, and the location of the specific-heat peak
near the exact critical temperatures (Ising 2/ln(1+sqrt 2); Potts q=10
1/ln(1+sqrt 10) = 0.701232, the value the paper quotes).  ``jackknife`` is
pinned by closed forms (runs that differ by constant shifts: U and C exact,
the ln Z error equal to the standard error of the shifts' mean) and by a
Monte Carlo check of the error it reports against the true spread of the
estimate over repeated experiments.
"""
import numpy as np


def thermodynamics(lng, e_min, e_step, temperatures):
    lng = np.asarray(lng, dtype=np.float64)
    E = e_min + e_step * np.arange(len(lng), dtype=np.float64)
    fin = np.isfinite(lng)
    lng, E = lng[fin], E[fin]
    out = []
    for T in np.asarray(temperatures, dtype=np.float64):
        beta = 1.0 / T
        x = lng - beta * E
        mx = x.max()
        w = np.exp(x - mx)
        z = w.sum()
        U = (w * E).sum() / z
        C = beta * beta * (w * (E - U) ** 2).sum() / z
        lnZ = mx + np.log(z)
        F = -T * lnZ
        out.append((lnZ, U, C, F, (U - F) / T))
    return np.array(out)


def jackknife(lng_runs, e_min, e_step, temperatures):
    """Resampling errors over R independent runs (paper, join paragraph:
    statistical errors by resampling; the jackknife of Newman and Barkema,
    "Monte Carlo Methods in Statistical Physics", section 3.4.3).

    lng_runs: R normalised ln g tables of one problem (R >= 2); a bin counts
    only where every run has a finite value.  For each temperature the
    quantities of ``thermodynamics`` are computed from the mean ln g over all
    runs (the estimate) and from each leave-one-out mean ln g_(i); the
    jackknife error is sqrt((R-1)/R * sum_i (Q_(i) - mean_i Q_(i))^2).
    Returns (estimate, error), each [n_T][5]."""
    runs = np.asarray(lng_runs, dtype=np.float64)
    R = runs.shape[0]
    fin = np.isfinite(runs).all(axis=0)
    mean = np.full(runs.shape[1], -np.inf)
    total = runs[0, fin].copy()
    for i in range(1, R):          # summed in run order
        total = total + runs[i, fin]
    mean[fin] = total / R
    est = thermodynamics(mean, e_min, e_step, temperatures)
    loo = []
    for i in range(R):
        t = np.full(runs.shape[1], -np.inf)
        t[fin] = (total - runs[i, fin]) / (R - 1)
        loo.append(thermodynamics(t, e_min, e_step, temperatures))
    loo = np.array(loo)
    err = np.sqrt((R - 1) / R * ((loo - loo.mean(axis=0)) ** 2).sum(axis=0))
    return est, err
