"""The 3D +-J glass (REWL_EA_PM_J_3D, the paper's 12^3 spin glass) on the GPU:
bit-exact against the oracle's 3D model (pinned in tests/test_oracle_3d.py)
for every sweep form, drawn and given couplings, up to the paper's size; a
full run to convergence; and a 3D request in the served form."""
import numpy as np
import pytest

from paper_1305_5615_gb300 import rewl
from parity_util import compare_states, make_pair, run_both

pytestmark = pytest.mark.gpu


def _parity(O, D, chunks, where):
    assert compare_states(O, D, where + " entry") == 0
    for nb in chunks:
        run_both(O, D, nb)
        assert compare_states(O, D, where) == 0


@pytest.mark.parametrize("G,variant", [(0, -1), (8, -1), (32, 1), (4, -1)])
def test_L4_all_sweep_forms(G, variant):
    O, D = make_pair("ea3d", 4, 4, 0.75, 2, 0.8, 1e-6, 5, G=G)
    if variant == 1:
        D = rewl.REWL("ea3d", 4, 4, 0.75, 2, 0.8, 1e-6, 5, lanes_per_walker=G, sweep_variant=1)
    _parity(O, D, [1, 9], "3D L=4 G=%d variant %d" % (G, variant))


@pytest.mark.parametrize("L,h,m", [(6, 4, 2), (8, 8, 2), (12, 8, 2)])
def test_larger_cubes(L, h, m):
    O, D = make_pair("ea3d", L, h, 0.75, m, 0.8, 1e-6, 40 + L)
    assert D.info["N"] == L ** 3
    _parity(O, D, [1], "3D L=%d" % L)


def test_given_couplings_full_run():
    J = np.random.default_rng(3).choice([-1, 1], size=3 * 64).astype(np.int8)
    O, D = make_pair("ea3d", 4, 3, 0.75, 2, 0.8, 1e-4, 6, couplings=J)
    assert np.array_equal(O.couplings(), J)
    for _ in range(10000):
        done_o, done_d = run_both(O, D, 10)
        assert compare_states(O, D, "3D full run") == 0
        assert done_o == done_d
        if done_o:
            break
    assert done_o
    g, e0, de = D.lng()
    go = O.joined_lng()
    fin = np.isfinite(go)
    assert np.array_equal(np.isfinite(g), fin) and np.allclose(g[fin], go[fin], rtol=0, atol=1e-9)


def test_served_3d_request_equals_alone():
    D = rewl.REWL("ea3d", 4, 3, 0.75, 2, 0.8, 1e-3, 8)
    assert D.step(0)
    g = D.lng()[0]
    S = rewl.RewlServer(device_bytes=1 << 30, max_running=3)
    a = S.submit("ea3d", 4, 3, 0.75, 2, 0.8, 1e-3, 8)
    b = S.submit("ea", 8, 4, 0.75, 2, 0.8, 1e-3, 9)
    for _ in range(100000):
        st = S.run(20)
        if st["running"] == 0 and st["queued"] == 0:
            break
    assert st["finished"] == 2
    assert np.array_equal(S.result(a)[0].view(np.uint64), g.view(np.uint64))
