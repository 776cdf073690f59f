"""Run-time balanced window partition (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper, Fig. 1b and the paragraph on the speed-up: besides equal windows
(Fig. 1a) the energy range can be split so that the walkers of every window
complete the first WL iteration after the same number of sweeps; the paper
estimates such a split from the first-iteration data of a short pre-run with
equal windows, using that the growth of WL histograms is known.  It gives no
formula.  Reading used here:

* the first iteration of a window behaves like a diffusive walk over its
  bins: its duration is tau = (sum over its bins of rho(b))^2 with a local
  cost rho(b) per bin;
* from the pre-run, window a (first merge after tau_a sweeps, width w_a)
  gives rho_a = sqrt(tau_a) / w_a, and rho(b) is the mean of rho_a over the
  pre-run windows that contain bin b (summed in window order);
* with U(b) = rho(0) + ... + rho(b-1) (U(0) = 0, summed in bin order) the
  balanced windows are the equal-width partition of Fig. 1a laid out in U
  instead of in bins: length lam = U(B) / (1 + (h-1)(1-o)), window k covers
  [u_k, u_k + lam] with u_k = k (U(B) - lam) / (h-1); its first bin is the
  last b with U(b) <= u_k, its last bin the first b with U(b+1) >= u_k + lam
  (first window from bin 0, last to bin B-1);
* the result must pass the checks of any explicit partition (widths >= 3,
  starts and ends strictly increasing, neighbours share >= 1 bin).

Parity: pinned by tests/test_oracle_plan.py -- equal costs give back the
equal partition; hand-computed partitions for piecewise costs; the balance
property (equal sum of rho per window up to one bin) on random costs.
"""
import math


def bin_costs(first_iter_sweeps, starts, widths, n_bins):
    """rho(b) from a pre-run with the given windows and first-merge clocks."""
    h = len(starts)
    rho_w = []
    for a in range(h):
        tau = int(first_iter_sweeps[a])
        if tau <= 0:
            raise ValueError("window %d has not finished its first iteration" % a)
        rho_w.append(math.sqrt(float(tau)) / float(widths[a]))
    rho = []
    for b in range(n_bins):
        s, n = 0.0, 0
        for a in range(h):
            if starts[a] <= b < starts[a] + widths[a]:
                s = s + rho_w[a]
                n += 1
        if n == 0:
            raise ValueError("bin %d is in no window" % b)
        rho.append(s / float(n))
    return rho


def partition(rho, h, overlap):
    """Windows with equal sums of rho (overlap o in that measure): (starts, widths)."""
    B = len(rho)
    U = [0.0]
    for b in range(B):
        U.append(U[-1] + rho[b])
    if h == 1:
        return [0], [B]
    T = U[B]
    lam = T / (1.0 + float(h - 1) * (1.0 - overlap))
    starts, ends = [], []
    for k in range(h):
        u_lo = (float(k) * (T - lam)) / float(h - 1)
        u_hi = u_lo + lam
        if k == 0:
            s = 0
        else:
            s = 0
            for b in range(B):
                if U[b] <= u_lo:
                    s = b
        if k == h - 1:
            e = B - 1
        else:
            e = B - 1
            for b in range(B):
                if U[b + 1] >= u_hi:
                    e = b
                    break
        starts.append(s)
        ends.append(e)
    widths = [e - s + 1 for s, e in zip(starts, ends)]
    check(starts, widths, B)
    return starts, widths


def check(starts, widths, B):
    h = len(starts)
    if starts[0] != 0 or starts[-1] + widths[-1] != B:
        raise ValueError("partition does not cover the range")
    for k in range(h):
        if widths[k] < 3:
            raise ValueError("window %d narrower than 3 bins" % k)
        if k > 0:
            if starts[k] <= starts[k - 1] or starts[k] + widths[k] <= starts[k - 1] + widths[k - 1]:
                raise ValueError("windows %d and %d not ordered" % (k - 1, k))
            if starts[k] > starts[k - 1] + widths[k - 1] - 1:
                raise ValueError("windows %d and %d do not overlap" % (k - 1, k))


def balanced_windows(first_iter_sweeps, pre_starts, pre_widths, n_bins, h, overlap):
    return partition(bin_costs(first_iter_sweeps, pre_starts, pre_widths, n_bins), h, overlap)
