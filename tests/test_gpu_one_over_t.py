"""The 1/t rule (REWL_RULE_ONE_OVER_T) on the GPU: bit-exact against the
oracle's 1/t rule (pinned in tests/test_oracle_one_over_t.py) -- lattices,
energies, ln g, H, ln f, stage and counters -- through both stages and to
convergence; in the served form, each result equal to its result alone; and
checkpoint / resume across the stage change."""
import numpy as np
import pytest

from paper_1305_5615_gb300 import rewl
from parity_util import compare_states, make_pair, run_both

pytestmark = pytest.mark.gpu


def _to_end(O, D, step_blocks, where):
    ties = 0
    for _ in range(100000):
        done_o, done_d = run_both(O, D, step_blocks)
        ties += compare_states(O, D, where)
        if ties:
            return ties
        assert done_o == done_d, where
        if done_o:
            return 0
    raise AssertionError("no convergence")


def test_ising_L8_four_windows_to_convergence():
    """t = 64 * clock / 38: stage 0 ends near the 15th check (2^-14), stage 1
    halves at t = 2^15, 2^16, 2^17 -- the run ends near 78000 sweeps."""
    O, D = make_pair("ising", 8, 4, 0.75, 2, 0.8, 2.0 ** -16, 7, wl_rule="1/t")
    assert compare_states(O, D, "entry") == 0
    assert _to_end(O, D, 100, "ising L=8 1/t") == 0
    st = D.state()
    assert (st["stage"] == 1).all() and (st["lnf"] == 2.0 ** -17).all()


@pytest.mark.parametrize("model,L,q,h,m", [("potts", 6, 3, 3, 2), ("ea", 8, 2, 4, 2), ("ising", 16, 2, 8, 4)])
def test_models_through_the_stage_change(model, L, q, h, m):
    O, D = make_pair(model, L, h, 0.75, m, 0.8, 2.0 ** -20, 40 + L, q=q, wl_rule="1/t")
    seen = False
    for _ in range(40):
        run_both(O, D, 10)
        assert compare_states(O, D, "%s L=%d" % (model, L)) == 0
        seen = seen or bool((D.state()["stage"] == 1).any())
        if seen and D.state()["sweep_clock"] >= 20000:
            break
    assert seen


def test_checkpoint_resume_across_the_stage_change():
    _, A = make_pair("ising", 8, 4, 0.75, 2, 0.8, 2.0 ** -16, 9, wl_rule="1/t")
    A.step(9000)
    mid = A.state()
    assert (mid["stage"] == 0).all()
    A.step(12000)
    ref = A.state()
    assert (ref["stage"] == 1).any()
    B = rewl.REWL("ising", 8, 4, 0.75, 2, 0.8, 2.0 ** -16, 9, wl_rule="1/t")
    B.set_state(mid)
    B.step(12000)
    got = B.state()
    for k in ("lattice", "E", "H", "lnf", "iteration", "stage"):
        assert np.array_equal(got[k], ref[k]), k
    assert np.array_equal(got["lng"].view(np.uint64), ref["lng"].view(np.uint64))
    bad = dict(mid)
    bad["stage"] = np.full_like(mid["stage"], 2)
    with pytest.raises(rewl.RewlError):
        B.set_state(bad)


def test_served_results_equal_results_alone():
    reqs = [("ising", 8, 4, 2, 2, 11), ("potts", 6, 3, 2, 3, 12), ("ea", 8, 4, 2, 2, 13)]
    alone = []
    for model, L, h, m, q, seed in reqs:
        D = rewl.REWL(model, L, h, 0.75, m, 0.8, 2.0 ** -16, seed, q=q, wl_rule="1/t")
        assert D.step(0)
        alone.append(D.lng()[0])
        D.close()
    S = rewl.RewlServer(device_bytes=1 << 30, max_running=3, wl_rule="1/t")
    ids = [S.submit(model, L, h, 0.75, m, 0.8, 2.0 ** -16, seed, q=q) for model, L, h, m, q, seed in reqs]
    for _ in range(100000):
        st = S.run(50)
        if st["running"] == 0 and st["queued"] == 0:
            break
    assert st["finished"] == 3
    for rid, g in zip(ids, alone):
        assert np.array_equal(S.result(rid)[0].view(np.uint64), g.view(np.uint64))
