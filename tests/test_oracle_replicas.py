"""Pins of the oracle's replica round-trip log (Fig. 3 follows replicas through
the windows): the counters equal a recount, by the definition, from the
replica-to-walker map recorded after every exchange round."""
import numpy as np

from oracle import OracleREWL


def _recount(history, m, h):
    """history[t][W] = replica held by walker W after round t.  A round trip:
    lowest window, then the highest, then the lowest again."""
    n = h * m
    state = np.zeros(n, np.int64)
    trips = np.zeros(n, np.int64)
    state[history[0][:m]] = 1
    for ids in history[1:]:
        for W, r in enumerate(ids):
            a = W // m
            if a == 0:
                if state[r] == 2:
                    trips[r] += 1
                state[r] = 1
            elif a == h - 1 and state[r] == 1:
                state[r] = 2
    return state, trips


def test_round_trips_match_a_recount_of_the_history():
    for model, L, h, m, q in (("ising", 8, 3, 2, 2), ("potts", 6, 4, 3, 3), ("ising", 8, 2, 4, 2)):
        R = OracleREWL(model, L, h, 0.75, m, 0.8, 1e-8, 3, q=q, sweeps_per_exchange=10, sweeps_per_flat_check=100)
        hist = [R.replicas()["rep_id"].copy()]
        for _ in range(400):
            R.run_blocks(1)
            hist.append(R.replicas()["rep_id"].copy())
        rep = R.replicas()
        assert sorted(rep["rep_id"]) == list(range(h * m))          # a permutation at every time
        state, trips = _recount(hist, m, h)
        assert np.array_equal(rep["rep_state"], state) and np.array_equal(rep["rep_trips"], trips)
        assert trips.sum() > 0, model                               # replicas do travel
