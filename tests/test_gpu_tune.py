"""rewl_autotune: every candidate launch shape runs, the fastest is returned,
and a solve with the chosen shape matches the oracle bit for bit (the shapes
change speed only)."""
import pytest

from paper_1305_5615_gb300 import rewl
from parity_util import compare_states, make_pair, run_both

pytestmark = pytest.mark.gpu


def test_autotune_picks_a_shape_that_computes_the_same_bits():
    kw, res = rewl.rewl_autotune("ising", 16, 4, 0.75, 2, 0.8, 1e-6, 3, sweeps=200)
    assert len(res) == 6 and all(r["status"] == 0 for r in res)
    assert all(r["ms_per_launch"] > 0 and r["attempts_per_s"] > 0 for r in res)
    fastest = min(res, key=lambda r: r["ms_per_launch"])
    assert (kw["sweep_variant"], kw["lanes_per_walker"]) == (fastest["sweep_variant"], fastest["lanes_per_walker"])
    O, _ = make_pair("ising", 16, 4, 0.75, 2, 0.8, 1e-6, 3)
    D = rewl.REWL("ising", 16, 4, 0.75, 2, 0.8, 1e-6, 3, **kw)
    run_both(O, D, 5)
    assert compare_states(O, D, "autotuned") == 0
    with pytest.raises(rewl.RewlError):
        rewl.rewl_autotune("ising", 16, 4, 0.75, 2, 0.8, 1e-6, 3, sweeps=150)   # not whole blocks
