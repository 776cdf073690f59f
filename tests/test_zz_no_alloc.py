"""rewl_sweep_noalloc: the sweep for callers that cannot let the library
allocate device memory (they hold the state in their own buffers and the
library takes its working memory from a fixed array compiled into it).

The entry point is called through the C ABI on device buffers owned by the
test, and its result is compared with rewl_step on the same solve: with one
window there is no exchange pair, so one 100-sweep block of rewl_step is one
sweep launch.  Two calls in a row must both match bit for bit (the bar every
parity test here uses).  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1305_5615_gb300 import rewl

pytestmark = pytest.mark.gpu


def _to_dev(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).view(dtype)).cuda()


@pytest.mark.parametrize("model,L,q", [("ising", 16, 2), ("potts", 12, 10)])
def test_sweep_noalloc_matches_rewl_step_twice(model, L, q):
    import torch

    D = rewl.REWL(model, L, 1, 0.75, 4, 0.8, 1e-6, 7, q=q)
    info = D.info
    st = D.state()
    lat = _to_dev(torch, st["lattice"], np.int32)
    E = _to_dev(torch, st["E"], np.int32)
    lng = _to_dev(torch, st["lng"], np.float64)
    H = _to_dev(torch, st["H"], np.int32)
    win = _to_dev(torch, st["win_start"], np.int32)
    lnf = _to_dev(torch, st["lnf"], np.float64)
    desc = rewl.rewl_sweep_desc(model=info["model"], q=info["q"], L=L, windows=1, walkers_per_window=4,
                                window_bins=info["window_bins"], e_min=info["e_min"], e_step=info["e_step"],
                                seed=7, first_sweep=0, sweeps=100, lanes_per_walker=0)
    for call in range(2):
        desc.first_sweep = 100 * call
        rewl.rewl_sweep_noalloc(desc, lat.data_ptr(), E.data_ptr(), lng.data_ptr(), H.data_ptr(), None,
                                win.data_ptr(), lnf.data_ptr(), None)
        torch.cuda.synchronize()
        D.step(100)
        ref = D.state()
        assert np.array_equal(lat.cpu().numpy().view(np.uint32), ref["lattice"]), call
        assert np.array_equal(E.cpu().numpy(), ref["E"]), call
        assert np.array_equal(H.cpu().numpy().view(np.uint32), ref["H"]), call
        assert np.array_equal(lng.cpu().numpy().view(np.uint64), ref["lng"].view(np.uint64)), call
        assert ref["H"].sum() == 4 * 100 * (call + 1) * L * L


def test_sweep_noalloc_rejects_more_walkers_than_its_array_holds():
    desc = rewl.rewl_sweep_desc(model=0, q=2, L=8, windows=2, walkers_per_window=4096, window_bins=40, e_min=-128,
                                e_step=4, seed=0, first_sweep=0, sweeps=1, lanes_per_walker=0)
    with pytest.raises(rewl.RewlError) as e:
        rewl.rewl_sweep_noalloc(desc, 16, 16, 16, 16, None, 16, 16, None)   # never dereferenced: rejected first
    assert e.value.status == 1
    assert "4096" in rewl.rewl_last_error()
