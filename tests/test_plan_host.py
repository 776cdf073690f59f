"""The library's window planner (rewl_plan_windows, host arithmetic only --
no device is touched) against the oracle's independent planner
(oracle/plan.py, pinned in tests/test_oracle_plan.py): the same partition,
integer for integer, on hand cases and on random pre-run data."""
import numpy as np
import pytest

from oracle.plan import balanced_windows
from paper_1305_5615_gb300 import rewl


def _equal(B, h, o):
    w = int(np.ceil(B / (1 + (h - 1) * (1 - o))))
    starts = [(2 * k * (B - w) + (h - 1)) // (2 * (h - 1)) for k in range(h)] if h > 1 else [0]
    return starts, [w] * h


def test_hand_cases():
    st, wd = rewl.rewl_plan_windows([100, 400], [0, 3], [6, 6], 9, 2, 0.5)
    assert (list(st), list(wd)) == balanced_windows([100, 400], [0, 3], [6, 6], 9, 2, 0.5)
    st, wd = rewl.rewl_plan_windows([50], [0], [40], 40, 1, 0.75)
    assert (list(st), list(wd)) == ([0], [40])


def test_random_pre_runs_match_the_oracle():
    rng = np.random.default_rng(7)
    for _ in range(40):
        B = int(rng.integers(60, 2100))
        h0 = int(rng.integers(2, 17))
        o = float(rng.choice([0.6, 0.75, 0.8]))
        ps, pw = _equal(B, h0, o)
        tau = rng.integers(1000, 10 ** 7, size=h0)
        h = int(rng.integers(2, 17))
        try:
            want = balanced_windows(tau, ps, pw, B, h, o)
        except ValueError:
            with pytest.raises(rewl.RewlError):
                rewl.rewl_plan_windows(tau, ps, pw, B, h, o)
            continue
        st, wd = rewl.rewl_plan_windows(tau, ps, pw, B, h, o)
        assert (list(st), list(wd)) == want


def test_rejects_unfinished_pre_runs():
    with pytest.raises(rewl.RewlError):
        rewl.rewl_plan_windows([100, -1], [0, 3], [6, 6], 9, 2, 0.5)
