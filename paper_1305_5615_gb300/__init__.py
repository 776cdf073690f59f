"""GB300-native replica-exchange Wang-Landau (REWL) sampling.

The method is that of Vogel, Li, Wuest and Landau (PRL 110, 210603, 2013):
overlapping energy windows, several independent Wang-Landau walkers per
window, configuration swaps between neighbouring windows (Eq. (1)), merging
of the walkers' ln g when a window's histograms are flat, and joining of the
fragments at the end.  Every phase runs as hand-written CUDA for sm_103a in
``librewl.so`` behind the C ABI of ``include/rewl.h``; ``rewl`` is its thin
Python binding.
"""
from .rewl import REWL, rewl_create, rewl_destroy, rewl_get_info, rewl_get_lng, rewl_get_state  # noqa: F401
from .rewl import rewl_get_window_lng, rewl_params_default, rewl_set_state, rewl_step  # noqa: F401
from .rewl import rewl_last_error, rewl_status_str, RewlError, unpack_lattice, RewlServer  # noqa: F401
