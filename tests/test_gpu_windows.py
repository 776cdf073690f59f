"""Unequal windows (Fig. 1b) on the GPU: explicit partitions bit-exact against
the oracle to convergence; the run-time balanced pipeline -- equal pre-run,
plan, balanced run -- identical on both sides; malformed tables rejected."""
import numpy as np
import pytest

from oracle.plan import balanced_windows
from paper_1305_5615_gb300 import rewl
from parity_util import compare_states, make_pair, run_both

pytestmark = pytest.mark.gpu


def test_explicit_unequal_windows_ising_L8_to_convergence():
    # 65 bins: widths 20, 30, 28, 25 (the equal partition has 38 each)
    st, wd = [0, 14, 30, 40], [20, 30, 28, 25]
    O, D = make_pair("ising", 8, 4, 0.75, 2, 0.8, 1e-4, 3, window_starts=st, window_widths=wd)
    assert D.info["window_bins"] == 30
    assert compare_states(O, D, "entry") == 0
    for _ in range(1000):
        done_o, done_d = run_both(O, D, 20)
        assert compare_states(O, D, "unequal L=8") == 0
        assert done_o == done_d
        if done_o:
            break
    assert done_o
    g, e0, de = D.lng()
    assert np.array_equal(np.isfinite(g), np.isfinite(O.joined_lng()))
    assert np.allclose(g[np.isfinite(g)], O.joined_lng()[np.isfinite(g)], rtol=0, atol=1e-9)


@pytest.mark.parametrize("model,L,q,h,m", [("potts", 8, 10, 4, 2), ("ea", 8, 2, 4, 2), ("ising", 16, 2, 6, 2)])
def test_balanced_pipeline_matches_the_oracle(model, L, q, h, m):
    O, D = make_pair(model, L, h, 0.75, m, 0.8, 1e-3, 60 + L, q=q)
    for _ in range(2000):
        run_both(O, D, 10)
        assert compare_states(O, D, "pre-run") == 0
        if (D.state()["first_iter"] > 0).all():
            break
    sd = D.state()
    assert (sd["first_iter"] > 0).all()
    ps, pw = rewl.rewl_plan_windows(sd["first_iter"], sd["win_start"], sd["win_width"], D.info["n_bins"], h, 0.75)
    assert (list(ps), list(pw)) == balanced_windows(sd["first_iter"], sd["win_start"], sd["win_width"],
                                                    D.info["n_bins"], h, 0.75)
    O2, D2 = make_pair(model, L, h, 0.75, m, 0.8, 1e-3, 60 + L, q=q, window_starts=ps, window_widths=pw)
    assert compare_states(O2, D2, "balanced entry") == 0
    for _ in range(5):
        run_both(O2, D2, 10)
        assert compare_states(O2, D2, "balanced run") == 0


def test_malformed_tables_are_rejected():
    bad = [([0, 14, 30, 40], [20, 30, 28, 24]),   # does not reach the last bin
           ([1, 14, 30, 40], [20, 30, 28, 25]),   # does not start at bin 0
           ([0, 25, 30, 40], [20, 30, 28, 25]),   # windows 0 and 1 do not overlap
           ([0, 14, 30, 40], [20, 2, 28, 25]),    # narrower than 3 bins
           ([0, 30, 14, 40], [20, 28, 30, 25])]   # not ordered
    for st, wd in bad:
        with pytest.raises(rewl.RewlError) as e:
            rewl.REWL("ising", 8, 4, 0.75, 2, 0.8, 1e-4, 3, window_starts=st, window_widths=wd)
        assert e.value.status == 1
