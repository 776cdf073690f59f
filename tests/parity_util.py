"""Helpers shared by the GPU parity tests: build the same solve on the oracle
and on the CUDA library, and compare their full states bit for bit."""
import numpy as np

from oracle import OracleREWL
from paper_1305_5615_gb300 import rewl


def make_pair(model, L, h, o, m, flatness, lnf_final, seed, q=2, couplings=None, spe=100, spf=1000, lnf0=1.0,
              G=0, wpb=0, mode=rewl.MODE_PLAIN, entry_max_sweeps=1000, discovery_sweeps=200, wl_rule="flat",
              window_starts=None, window_widths=None, **gpu_kw):
    O = OracleREWL(model, L, h, o, m, flatness, lnf_final, seed, q=q, couplings=couplings, sweeps_per_exchange=spe,
                   sweeps_per_flat_check=spf, lnf0=lnf0, entry_max_sweeps=entry_max_sweeps,
                   discovery_sweeps=discovery_sweeps, wl_rule=wl_rule, window_starts=window_starts,
                   window_widths=window_widths)
    D = rewl.REWL(model, L, h, o, m, flatness, lnf_final, seed, q=q, couplings=couplings, sweeps_per_exchange=spe,
                  sweeps_per_flat_check=spf, lnf0=lnf0, entry_max_sweeps=entry_max_sweeps,
                  discovery_sweeps=discovery_sweeps, lanes_per_walker=G, walkers_per_block=wpb, mode=mode,
                  wl_rule=wl_rule, window_starts=window_starts, window_widths=window_widths, **gpu_kw)
    return O, D


def compare_states(O, D, where=""):
    """Bit-exact comparison of configurations, energies, ln g, H, ln f,
    iteration counters, done flags and the WL / exchange counters.  Returns
    the number of near-tie acceptance tests (|ln u - Delta ln g| < 1e-12) the
    oracle met; those are the only places the two may legitimately diverge."""
    so, wo, co = O.walkers(), O.windows(), O.counters()
    sg = D.state()
    ties = int(co["near_ties"].sum())
    if ties:
        return ties
    model = D.info["model"]
    spins = rewl.unpack_lattice(sg["lattice"], D.info["L"], model)
    assert D.info["window_bins"] == O.w and D.info["n_bins"] == O.n_bins and D.info["e_min"] == O.e_min, where
    assert np.array_equal(sg["win_start"], wo["start"]), where
    assert np.array_equal(sg["win_width"], wo["width"]), where
    assert np.array_equal(sg["first_iter"], wo["first_iter"]), where
    bad = np.nonzero((spins != so["spins"]).any(1))[0]
    assert bad.size == 0, "%s: configurations differ for walkers %s" % (where, bad[:8])
    assert np.array_equal(sg["E"], so["E"]), where
    assert np.array_equal(sg["H"], so["H"]), "%s: H differs for walkers %s" % (
        where, np.nonzero((sg["H"] != so["H"]).any(1))[0][:8])
    lb_g, lb_o = sg["lng"].view(np.uint64), so["lng"].view(np.uint64)
    assert np.array_equal(lb_g, lb_o), "%s: ln g bits differ for walkers %s (max |d| %g)" % (
        where, np.nonzero((lb_g != lb_o).any(1))[0][:8], np.abs(sg["lng"] - so["lng"]).max())
    assert np.array_equal(sg["lnf"].view(np.uint64), wo["lnf"].view(np.uint64)), where
    assert np.array_equal(sg["iteration"], wo["iteration"]), where
    assert np.array_equal(sg["done"] != 0, wo["done"] != 0), where
    assert np.array_equal(sg["stage"], wo["phase"]), where
    assert np.array_equal(sg["wl_accept"], co["wl_accept"]), where
    assert np.array_equal(sg["near_ties"], co["near_ties"]), where
    assert np.array_equal(sg["x_tried"], co["x_tried"]), where
    assert np.array_equal(sg["x_accepted"], co["x_accepted"]), where
    rp = O.replicas()
    for k in ("rep_id", "rep_state", "rep_trips"):
        assert np.array_equal(sg[k], rp[k]), (where, k)
    assert sg["sweep_clock"] == O.info()["sweep_clock"], where
    return 0


def run_both(O, D, n_blocks, spe=100):
    done_o = O.run_blocks(n_blocks)
    done_d = D.step(n_blocks * spe)
    return done_o, done_d
