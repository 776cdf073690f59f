"""Joining of overlapping ln g fragments (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper, paragraph after Eq. (1): at the end of the simulation the h x m
overlapping fragments of g(E) are joined into one g(E) over the whole range;
the joining point of two overlapping pieces is where the inverse
microcanonical temperatures beta = d ln g / dE of the two pieces agree best.

Reading used (the paper gives no formula): beta at bin b is the central
difference (ln g[b+1] - ln g[b-1]) / (2 dE), defined where b-1, b, b+1 are all
visited in the piece; the joining bin is the overlap bin with the smallest
|beta_a - beta_{a+1}|, ties to the lowest bin.  Window a+1 is shifted to agree
with window a there; below the joining bin the lower window is used, above it
the upper one.  The result is normalised so that sum_E g(E) = 2^N (Ising,
+-J) or q^N (Potts).  Bins never visited are -inf.

Parity: pinned by tests/test_oracle_join.py (exact ln g split into windows
with per-window offsets is recovered exactly; normalisation identity).
"""
import math

import numpy as np


def join_windows(lng_windows, starts, w, n_bins):
    """lng_windows[a][b] is window a's ln g at its local bin b (0 = never
    visited); starts[a] its first global bin; w the width of every window, or
    a sequence of per-window widths (unequal, run-time balanced windows).
    Returns the joined, not yet normalised ln g over n_bins global bins (-inf
    where not visited)."""
    h = len(starts)
    widths = [int(w)] * h if np.ndim(w) == 0 else [int(x) for x in w]
    out = np.full(n_bins, -np.inf)
    first = np.asarray(lng_windows[0], dtype=np.float64)
    for b in range(widths[0]):
        if first[b] > 0.0:
            out[starts[0] + b] = first[b]
    shift_prev = 0.0
    for a in range(h - 1):
        A = np.asarray(lng_windows[a], dtype=np.float64)
        B = np.asarray(lng_windows[a + 1], dtype=np.float64)
        sa, sb = int(starts[a]), int(starts[a + 1])
        lo, hi = sb, sa + widths[a] - 1  # global overlap [lo, hi]
        best, best_b = None, None
        for g in range(lo + 1, hi):      # interior overlap bins
            ia, ib = g - sa, g - sb
            if not (A[ia - 1] > 0 and A[ia] > 0 and A[ia + 1] > 0 and B[ib - 1] > 0 and B[ib] > 0 and B[ib + 1] > 0):
                continue
            dA = A[ia + 1] - A[ia - 1]
            dB = B[ib + 1] - B[ib - 1]
            diff = abs(dA - dB)
            if best is None or diff < best:
                best, best_b = diff, g
        if best_b is None:               # no 3-bin stretch: any bin visited in both pieces
            for g in range(lo, hi + 1):
                if A[g - sa] > 0 and B[g - sb] > 0:
                    best_b = g
                    break
        if best_b is None:
            raise ValueError("windows %d and %d share no visited bin" % (a, a + 1))
        shift = (A[best_b - sa] + shift_prev) - B[best_b - sb]
        for g in range(best_b + 1, sb + widths[a + 1]):
            v = B[g - sb]
            out[g] = v + shift if v > 0 else -np.inf
        shift_prev = shift
    return out


def normalise(lng, N, q):
    """Shift ln g so that sum_E g(E) = q^N (q = 2 for Ising and +-J)."""
    lng = np.asarray(lng, dtype=np.float64)
    fin = np.isfinite(lng)
    mx = lng[fin].max()
    lse = mx + math.log(np.exp(lng[fin] - mx).sum())
    out = lng.copy()
    out[fin] = lng[fin] + (N * math.log(q) - lse)
    return out
