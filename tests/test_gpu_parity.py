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


# ------------------------------------------ the warp-specialised ring variant
@pytest.mark.parametrize("model,L,q,h,m", [("ising", 8, 2, 4, 2), ("ising", 5, 2, 3, 2), ("potts", 8, 10, 4, 2),
                                           ("ea", 8, 2, 4, 2), ("ising", 32, 2, 16, 4)])
def test_ring_variant_matches_oracle(model, L, q, h, m):
    """sweep_variant 2: draws from a producer warp through a shared-memory ring
    (L=5: 2500 trials per launch, a ragged last group of 4)."""
    O = OracleREWL(model, L, h, 0.75, m, 0.8, 1e-6, 71 + L, q=q)
    D = rewl.REWL(model, L, h, 0.75, m, 0.8, 1e-6, 71 + L, q=q, sweep_variant=2)
    assert (D.info["lanes_per_walker"], D.info["walkers_per_block"], D.info["sweep_variant"]) == (32, 1, 2)
    _parity(O, D, [1, 12], "ring %s L=%d" % (model, L))


def test_ring_variant_full_run_and_served_shapes():
    O, _ = make_pair("ising", 8, 4, 0.75, 2, 0.8, 1e-6, 0)
    D = rewl.REWL("ising", 8, 4, 0.75, 2, 0.8, 1e-6, 0, sweep_variant=2)
    for _ in range(10000):
        done_o, done_d = run_both(O, D, 10)
        assert compare_states(O, D, "ring full run") == 0
        assert done_o == done_d
        if done_o:
            break
    assert done_o
    with pytest.raises(rewl.RewlError):
        rewl.REWL("ising", 8, 4, 0.75, 2, 0.8, 1e-6, 0, sweep_variant=2, lanes_per_walker=8)
    # the automatic choice: the ring form for few walkers, the chain form for many or forced lanes
    assert rewl.REWL("ising", 8, 4, 0.75, 2, 0.8, 1e-6, 0).info["sweep_variant"] == 2
    assert rewl.REWL("ising", 8, 4, 0.75, 2, 0.8, 1e-6, 0, lanes_per_walker=8).info["sweep_variant"] == 0
    assert rewl.REWL("potts", 16, 32, 0.75, 64, 0.8, 1e-6, 0, q=3).info["sweep_variant"] == 0


# ------------------------------------------------- the staged sweep variant
@pytest.mark.parametrize("model,L,q,G", [("ising", 8, 2, 32), ("ising", 12, 2, 8), ("potts", 8, 10, 32), ("ea", 8, 2, 16)])
def test_staged_variant_matches_oracle(model, L, q, G):
    O = OracleREWL(model, L, 4, 0.75, 2, 0.8, 1e-6, 31 + L, q=q)
    D = rewl.REWL(model, L, 4, 0.75, 2, 0.8, 1e-6, 31 + L, q=q, lanes_per_walker=G, sweep_variant=1)
    _parity(O, D, [1, 12], "staged %s L=%d G=%d" % (model, L, G))


# -------------------------------------------- failures made on the host side
def test_timeout_then_resume_is_bit_exact():
    _, A = make_pair("ising", 16, 4, 0.75, 2, 0.8, 1e-6, 23)
    A.step(3000)
    ref = A.state()
    B = rewl.REWL("ising", 16, 4, 0.75, 2, 0.8, 1e-6, 23, timeout_ms=1)
    with pytest.raises(rewl.RewlError) as e:
        B.step(3000)
    assert e.value.status == 4                         # REWL_ETIMEOUT, at a block boundary
    done_sweeps = rewl.rewl_get_info(B._h)["sweep_clock"]
    assert 0 < done_sweeps < 3000 and done_sweeps % 100 == 0
    B.params.timeout_ms = 0
    C = rewl.REWL("ising", 16, 4, 0.75, 2, 0.8, 1e-6, 23)
    C.set_state(B.state())                               # resume the interrupted solve elsewhere
    C.step(3000 - done_sweeps)
    got = C.state()
    for k in ("lattice", "E", "H", "lnf", "iteration"):
        assert np.array_equal(got[k], ref[k]), k
    assert np.array_equal(got["lng"].view(np.uint64), ref["lng"].view(np.uint64))


def test_allocation_failure_is_reported_and_nothing_leaks():
    import ctypes
    import torch

    calls = {"n": 0}
    live = {}

    def alloc(nbytes, stream, user):
        calls["n"] += 1
        if calls["n"] > 6:           # refuse from the 7th allocation on
            return None
        p = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream)
        live[p] = True
        return p

    def free(ptr, stream, user):
        live.pop(ptr, None)
        torch.cuda.caching_allocator_delete(ptr)

    A, F = rewl.ALLOC_FN(alloc), rewl.FREE_FN(free)
    p = rewl.rewl_params_default()
    p.alloc, p.free = A, F
    with pytest.raises(rewl.RewlError) as e:
        rewl.rewl_create(rewl.rewl_model(0, 2), rewl.rewl_lattice(2, 8, 8, 1), None, 4, 0.75, 2, 0.8, 1e-6, 0, p)
    assert e.value.status == 2                           # REWL_ENOMEM
    assert not live                                       # every granted block was returned
    assert "allocation" in rewl.rewl_last_error()


# ------------------------------------- draws prepared ahead on a second stream
def test_prefetched_draws_match_in_kernel_draws_and_the_oracle():
    """Ising L=32, 16 windows x 4 walkers: with the next block's draws prepared
    on a second stream the states equal those of the in-kernel draws and of the
    oracle; a rewind through rewl_set_state (stale prepared buffers) and a
    replay give the same bits again."""
    O = OracleREWL("ising", 32, 16, 0.75, 4, 0.8, 1e-8, 5)
    A = rewl.REWL("ising", 32, 16, 0.75, 4, 0.8, 1e-8, 5, prefetch_draws=1, sweep_variant=0)
    B = rewl.REWL("ising", 32, 16, 0.75, 4, 0.8, 1e-8, 5, prefetch_draws=0, sweep_variant=0)
    assert A.info["prefetch_draws"] == 1 and B.info["prefetch_draws"] == 0
    A.step(1000)
    B.step(1000)
    sa, sb = A.state(), B.state()
    for k in ("lattice", "E", "H", "lnf", "iteration"):
        assert np.array_equal(sa[k], sb[k]), k
    assert np.array_equal(sa["lng"].view(np.uint64), sb["lng"].view(np.uint64))
    O.run_blocks(10)    # the oracle to the same clock
    assert compare_states(O, A, "prefetched 1000 sweeps") == 0
    A.step(300)
    A.set_state(sa)     # rewind: the prepared buffers now hold draws of later blocks
    A.step(300)
    B.step(300)
    sa, sb = A.state(), B.state()
    for k in ("lattice", "E", "H", "lnf", "iteration"):
        assert np.array_equal(sa[k], sb[k]), k
    assert np.array_equal(sa["lng"].view(np.uint64), sb["lng"].view(np.uint64))


def test_ring_hand_off_wait_runs_out_and_reports_a_timeout():
    """The ring form's bounded hand-off waits: with a bound of a few cycles
    the first wait that finds its slot not ready gives up, both warps of every
    walker's CTA stop, and rewl_step reports REWL_ETIMEOUT from the error word
    at its flatness check; the context stays usable (a fresh solve then
    matches the oracle)."""
    D = rewl.REWL("ising", 32, 16, 0.75, 4, 0.8, 1e-8, 0, wait_cycles=4)
    assert D.info["sweep_variant"] == 2   # the ring form
    with pytest.raises(rewl.RewlError) as e:
        D.step(1000)
    assert e.value.status == 4            # REWL_ETIMEOUT
    assert "bounded" in rewl.rewl_last_error()
    D.close()
    O, D2 = make_pair("ising", 32, 16, 0.75, 4, 0.8, 1e-8, 0)
    _parity(O, D2, [1], "after a timed-out launch")
