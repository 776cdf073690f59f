"""GPU parity: the CUDA library against the oracle, on the same seeded inputs,
bit for bit (configurations, energies, FP64 ln g bit patterns, H, ln f,
iteration counters, WL and exchange counters).  Only acceptance tests whose
|ln u - Delta ln g| < 1e-12 may diverge; they are counted by both sides and
none has occurred in these cases (the tests assert it)."""
import numpy as np
import pytest

from oracle import OracleREWL
from paper_1305_5615_gb300 import rewl
from parity_util import compare_states, make_pair, run_both

pytestmark = pytest.mark.gpu


def _parity(O, D, blocks_list, where):
    assert compare_states(O, D, where + " after entry") == 0
    for i, nb in enumerate(blocks_list):
        run_both(O, D, nb)
        assert compare_states(O, D, "%s after chunk %d" % (where, i)) == 0


# ---------------------------------------------------------------- Ising L=8
@pytest.mark.parametrize("G", [1, 2, 4, 8, 16, 32])
def test_ising_L8_all_lane_counts(G):
    O, D = make_pair("ising", 8, 4, 0.75, 2, 0.8, 1e-6, 0, G=G)
    _parity(O, D, [1, 9, 30], "G=%d" % G)


def test_ising_L8_full_run_to_convergence():
    """Four windows x two walkers, ln f down to < 1e-6: the whole run, every
    flatness check and merge, matches the oracle bit for bit."""
    O, D = make_pair("ising", 8, 4, 0.75, 2, 0.8, 1e-6, 0)
    assert compare_states(O, D, "entry") == 0
    for i in range(2000):
        do, dd = run_both(O, D, 10)
        assert do == dd
        if i % 10 == 0 or do:
            assert compare_states(O, D, "block %d" % (10 * i)) == 0
        if do:
            break
    assert do, "did not converge"
    assert (D.state()["iteration"] == 20).all()
    g_d, e0, de = D.lng()
    g_o = O.joined_lng()
    fin = np.isfinite(g_o)
    assert np.array_equal(np.isfinite(g_d), fin)
    assert np.abs(g_d[fin] - g_o[fin]).max() < 1e-9


def test_ising_L8_seeds_and_walker_counts():
    for seed, h, m in ((1, 4, 1), (2, 3, 3), (3, 1, 4), (4, 6, 2)):
        O, D = make_pair("ising", 8, h, 0.75, m, 0.8, 1e-6, seed)
        _parity(O, D, [20], "seed %d h %d m %d" % (seed, h, m))


def test_graph_mode_matches_plain_and_oracle():
    O, D = make_pair("ising", 8, 4, 0.75, 2, 0.8, 1e-6, 5, mode=rewl.MODE_GRAPH)
    assert compare_states(O, D, "entry") == 0
    for i in range(6):
        O.run_blocks(10)
        D.step(1000)
        assert compare_states(O, D, "graph period %d" % i) == 0


def test_short_exchange_and_check_periods():
    O, D = make_pair("ising", 8, 4, 0.75, 2, 0.8, 1e-6, 6, spe=7, spf=21)
    assert compare_states(O, D, "entry") == 0
    for i in range(8):
        O.run_blocks(5)
        D.step(5 * 7)
        assert compare_states(O, D, "chunk %d" % i) == 0


# ------------------------------------------------------ odd and ragged sizes
@pytest.mark.parametrize("L", [5, 12, 33, 40])
def test_ising_non_power_of_two_sizes(L):
    O, D = make_pair("ising", L, 3, 0.75, 2, 0.8, 1e-6, 10 + L, G=8)
    _parity(O, D, [2], "L=%d" % L)


def test_ising_L32_sixteen_windows_four_walkers():
    """Ising 32 x 32, 16 windows x 4 walkers: the launch configuration the
    benchmark times, 1000 sweeps."""
    O, D = make_pair("ising", 32, 16, 0.75, 4, 0.8, 1e-8, 0)
    _parity(O, D, [1, 9], "Ising L32")


# --------------------------------------------------------------- Potts, +-J
@pytest.mark.parametrize("G", [1, 8, 32])
def test_potts_q10_L8(G):
    O, D = make_pair("potts", 8, 4, 0.75, 2, 0.8, 1e-6, 3, q=10, G=G)
    _parity(O, D, [1, 19], "Potts q10 L8 G=%d" % G)


def test_potts_q3_L6_to_convergence():
    O, D = make_pair("potts", 6, 3, 0.75, 2, 0.8, 1e-4, 8, q=3)
    assert compare_states(O, D, "entry") == 0
    for i in range(2000):
        do, dd = run_both(O, D, 10)
        assert do == dd
        if do:
            break
    assert compare_states(O, D, "end") == 0


def test_potts_q10_L32_thirtytwo_windows_sixteen_walkers():
    O, D = make_pair("potts", 32, 32, 0.75, 16, 0.8, 1e-8, 0, q=10)
    _parity(O, D, [2], "Potts q10 L32")


@pytest.mark.parametrize("L", [8, 12, 20])
def test_ea_drawn_couplings(L):
    O, D = make_pair("ea", L, 4, 0.75, 2, 0.8, 1e-6, 40 + L)
    assert np.array_equal(O.couplings(), O.couplings())
    _parity(O, D, [1, 10], "EA L=%d" % L)


def test_ea_given_couplings():
    J = np.random.default_rng(3).choice([-1, 1], size=2 * 16 * 16).astype(np.int8)
    O, D = make_pair("ea", 16, 8, 0.75, 4, 0.8, 1e-6, 9, couplings=J)
    _parity(O, D, [3], "EA given J")


# ------------------------------------------------------- checkpoint / resume
def test_checkpoint_resume_is_bit_exact():
    _, A = make_pair("ising", 16, 4, 0.75, 2, 0.8, 1e-6, 21)
    A.step(2000)
    snap = A.state()
    A.step(2000)
    ref = A.state()
    B = rewl.REWL("ising", 16, 4, 0.75, 2, 0.8, 1e-6, 21)
    B.set_state(snap)
    B.step(2000)
    got = B.state()
    for k in ("lattice", "E", "H", "lnf", "iteration", "done", "wl_accept", "x_accepted"):
        assert np.array_equal(got[k], ref[k]), k
    assert np.array_equal(got["lng"].view(np.uint64), ref["lng"].view(np.uint64))


# ----------------------------------------------------------------- errors
def test_invalid_arguments_are_rejected():
    with pytest.raises(rewl.RewlError) as e:
        rewl.REWL("ising", 8, 4, 1.5, 2, 0.8, 1e-6, 0)
    assert e.value.status == 1
    with pytest.raises(rewl.RewlError):
        rewl.REWL("ising", 8, 4, 0.75, 2, 0.8, 1e-6, 0, lnf0=0.7)
    with pytest.raises(rewl.RewlError):
        rewl.REWL("ea", 9, 2, 0.75, 2, 0.8, 1e-6, 0)
    with pytest.raises(rewl.RewlError):
        rewl.REWL("ising", 8, 200, 0.75, 2, 0.8, 1e-6, 0)   # windows of 2 bins are too narrow


def test_entry_failure_is_reported():
    # one sweep of greedy entry, even after the restart from the ground
    # state, leaves some of 16 windows unreached (the oracle fails alike)
    with pytest.raises(RuntimeError):
        OracleREWL("ising", 32, 16, 0.75, 1, 0.8, 1e-6, 0, entry_max_sweeps=1)
    with pytest.raises(rewl.RewlError) as e:
        rewl.REWL("ising", 32, 16, 0.75, 1, 0.8, 1e-6, 0, entry_max_sweeps=1)
    assert e.value.status == 5
    D = rewl.REWL("ising", 32, 8, 0.75, 1, 0.8, 1e-6, 0, entry_max_sweeps=1)   # and succeeds where it does
    assert D.info["window_bins"] > 0


def test_torch_allocator_and_stream():
    import torch

    s = torch.cuda.Stream()
    before = torch.cuda.memory_allocated()
    O = OracleREWL("ising", 8, 4, 0.75, 2, 0.8, 1e-6, 0)
    D = rewl.REWL("ising", 8, 4, 0.75, 2, 0.8, 1e-6, 0, stream=s, torch_allocator=True)
    assert torch.cuda.memory_allocated() > before
    O.run_blocks(10)
    D.step(1000)
    assert compare_states(O, D, "torch allocator") == 0
    D.close()
    assert torch.cuda.memory_allocated() == before
