"""rewl_sweep_noalloc: the sweep for callers that cannot let the library
allocate device memory (they hold the state in their own buffers and the
library takes its working memory from a fixed array compiled into it).

The entry point is called through the C ABI on device buffers owned by the
test.  With one window there is no exchange pair, so one 100-sweep block of
rewl_step is one sweep launch and the two are compared directly; with
several windows (nonzero window starts) the result is compared with the
oracle's sweeps of the same trial range (its block sweeps, no exchange).
Two calls in a row must both match bit for bit (the bar every parity test
here uses).  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1305_5615_gb300 import rewl

pytestmark = pytest.mark.gpu


def _to_dev(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).view(dtype)).cuda()


def _coupling_bits(J, L):
    """+-J couplings (site-major [2 i] right, [2 i + 1] down, i = y L + x) as
    the two bit planes [right|down][L][ceil(L/32)], bit set = J = -1."""
    Wr1 = (L + 31) // 32
    out = np.zeros((2, L, Wr1), np.uint32)
    for i in range(L * L):
        y, x = divmod(i, L)
        for plane in range(2):
            if J[2 * i + plane] < 0:
                out[plane, y, x // 32] |= np.uint32(1 << (x % 32))
    return out.reshape(-1)


def _desc(info, L, windows, m, seed, sweeps, G, status=None):
    return rewl.rewl_sweep_desc(model=info["model"], q=info["q"], L=L, windows=windows, walkers_per_window=m,
                                window_bins=info["window_bins"], e_min=info["e_min"], e_step=info["e_step"],
                                seed=seed, first_sweep=0, sweeps=sweeps, lanes_per_walker=G, status=status)


def _device_state(torch, st):
    return (_to_dev(torch, st["lattice"], np.int32), _to_dev(torch, st["E"], np.int32),
            _to_dev(torch, st["lng"], np.float64), _to_dev(torch, st["H"], np.int32),
            _to_dev(torch, st["win_start"], np.int32), _to_dev(torch, st["lnf"], np.float64))


@pytest.mark.parametrize("model,L,q,G,couplings", [("ising", 16, 2, 0, False), ("potts", 12, 10, 0, False),
                                                   ("ea", 16, 2, 8, True)])
def test_sweep_noalloc_matches_rewl_step_twice(model, L, q, G, couplings):
    import torch

    from oracle import OracleREWL

    D = rewl.REWL(model, L, 1, 0.75, 4, 0.8, 1e-6, 7, q=q)
    info = D.info
    lat, E, lng, H, win, lnf = _device_state(torch, D.state())
    Jb = None
    if couplings:   # the couplings the solve drew from its seed (the oracle draws the same)
        Jb = _to_dev(torch, _coupling_bits(OracleREWL(model, L, 1, 0.75, 4, 0.8, 1e-6, 7).couplings(), L), np.int32)
    status = torch.full((4,), -1, dtype=torch.int32, device="cuda")
    desc = _desc(info, L, 1, 4, 7, 100, G, status.data_ptr())
    for call in range(2):
        desc.first_sweep = 100 * call
        rewl.rewl_sweep_noalloc(desc, lat.data_ptr(), E.data_ptr(), lng.data_ptr(), H.data_ptr(),
                                Jb.data_ptr() if Jb is not None else None, win.data_ptr(), lnf.data_ptr(), None)
        torch.cuda.synchronize()
        D.step(100)
        ref = D.state()
        assert (status.cpu().numpy() == 0).all(), call
        assert np.array_equal(lat.cpu().numpy().view(np.uint32), ref["lattice"]), call
        assert np.array_equal(E.cpu().numpy(), ref["E"]), call
        assert np.array_equal(H.cpu().numpy().view(np.uint32), ref["H"]), call
        assert np.array_equal(lng.cpu().numpy().view(np.uint64), ref["lng"].view(np.uint64)), call
        assert ref["H"].sum() == 4 * 100 * (call + 1) * L * L


@pytest.mark.parametrize("G", [1, 8, 32])
def test_sweep_noalloc_several_windows_matches_the_oracle_sweeps(G):
    """Four windows x 2 walkers (window starts 0, 37, 73, 110 of 257 bins):
    per-window indexing of win_start and lnf, for 1, 8 and 32 lanes per
    walker.  Call 1 (sweeps 0..99) against the oracle's block of 100 sweeps,
    call 2 (sweeps 100..199) against a block of 200 from the same start."""
    import torch

    from oracle import OracleREWL

    args = ("ising", 16, 4, 0.75, 2, 0.8, 1e-6, 11)
    D = rewl.REWL(*args)
    info = D.info
    st = D.state()
    assert list(st["win_start"]) == [0, 37, 73, 110] and (st["win_width"] == info["window_bins"]).all()
    lat, E, lng, H, win, lnf = _device_state(torch, st)
    desc = _desc(info, 16, 4, 2, 11, 100, G)
    for call, spe in ((0, 100), (1, 200)):
        desc.first_sweep = 100 * call
        rewl.rewl_sweep_noalloc(desc, lat.data_ptr(), E.data_ptr(), lng.data_ptr(), H.data_ptr(), None,
                                win.data_ptr(), lnf.data_ptr(), None)
        torch.cuda.synchronize()
        O = OracleREWL(*args, sweeps_per_exchange=spe, sweeps_per_flat_check=1000)
        O.block_sweeps()
        so = O.walkers()
        spins = rewl.unpack_lattice(lat.cpu().numpy().view(np.uint32), 16, rewl.ISING)
        assert np.array_equal(spins, so["spins"]), call
        assert np.array_equal(E.cpu().numpy(), so["E"]), call
        assert np.array_equal(H.cpu().numpy().view(np.uint32), so["H"]), call
        assert np.array_equal(lng.cpu().numpy().view(np.uint64), so["lng"].view(np.uint64)), call


def test_sweep_noalloc_reports_walkers_it_cannot_run():
    """A walker whose E lies outside its window, and the walkers of a window
    whose ln f is not a usable power of two, are skipped and reported in the
    caller's status array; the others run as usual."""
    import torch

    D = rewl.REWL("ising", 16, 2, 0.75, 2, 0.8, 1e-6, 3)
    info = D.info
    st = D.state()
    lat, E, lng, H, win, lnf = _device_state(torch, st)
    bad_E = st["E"].copy()
    lo0 = info["e_min"] + int(st["win_start"][0]) * info["e_step"]
    bad_E[1] = lo0 + info["window_bins"] * info["e_step"] + 8     # above window 0
    E.copy_(torch.from_numpy(bad_E))
    lnf_h = st["lnf"].copy()
    lnf_h[1] = 0.75                                                # window 1: not a power of two
    lnf.copy_(torch.from_numpy(lnf_h))
    status = torch.full((4,), -1, dtype=torch.int32, device="cuda")
    before = (lat.clone(), lng.clone(), H.clone())
    rewl.rewl_sweep_noalloc(_desc(info, 16, 2, 2, 3, 10, 0, status.data_ptr()), lat.data_ptr(), E.data_ptr(),
                            lng.data_ptr(), H.data_ptr(), None, win.data_ptr(), lnf.data_ptr(), None)
    torch.cuda.synchronize()
    assert list(status.cpu().numpy()) == [0, 1, 1, 1]              # REWL_EINVAL for walkers 1, 2, 3
    Wd = info["lattice_words"]
    w = info["window_bins"]
    for W in (1, 2, 3):   # skipped: state unchanged
        assert torch.equal(lat[W * Wd:(W + 1) * Wd], before[0][W * Wd:(W + 1) * Wd])
        assert torch.equal(lng[W * w:(W + 1) * w], before[1][W * w:(W + 1) * w])
        assert torch.equal(H[W * w:(W + 1) * w], before[2][W * w:(W + 1) * w])
    assert int(H[:w].sum()) == 10 * 256                            # walker 0 ran its 10 sweeps


def test_sweep_noalloc_rejects_more_walkers_than_its_array_holds():
    desc = rewl.rewl_sweep_desc(model=0, q=2, L=8, windows=2, walkers_per_window=4096, window_bins=40, e_min=-128,
                                e_step=4, seed=0, first_sweep=0, sweeps=1, lanes_per_walker=0)
    with pytest.raises(rewl.RewlError) as e:
        rewl.rewl_sweep_noalloc(desc, 16, 16, 16, 16, None, 16, 16, None)   # never dereferenced: rejected first
    assert e.value.status == 1
    assert "4096" in rewl.rewl_last_error()
