"""Thin ctypes binding of the REWL C ABI (include/rewl.h).

Argument marshalling only: every step of the method runs in the CUDA library
``librewl.so``.  The functions keep the C names (``rewl_create``,
``rewl_step``, ``rewl_get_lng``, ...).  ``REWL`` is a small convenience class
over one handle.  PyTorch is optional and only supplies the CUDA stream and,
with ``torch_allocator=True``, the device memory (its caching allocator).
There is no CPU fallback: without the built library every call raises.
"""
import ctypes
import os

import numpy as np

from . import _build

ISING, POTTS, EA_PM_J, EA_PM_J_3D = 0, 1, 2, 3
MODE_PLAIN, MODE_GRAPH = 0, 1
MODELS = {"ising": ISING, "potts": POTTS, "ea": EA_PM_J, "pmj": EA_PM_J, "ea3d": EA_PM_J_3D}
RULE_FLAT, RULE_ONE_OVER_T = 0, 1
WL_RULES = {"flat": RULE_FLAT, "1/t": RULE_ONE_OVER_T}

STATUS = {0: "REWL_OK", 1: "REWL_EINVAL", 2: "REWL_ENOMEM", 3: "REWL_ECUDA", 4: "REWL_ETIMEOUT", 5: "REWL_EENTRY",
          6: "REWL_EOVERFLOW", 7: "REWL_EBUSY", 8: "REWL_ENOTFOUND", 9: "REWL_ENODEV"}

EXPORTED = ["rewl_params_default", "rewl_create", "rewl_step", "rewl_get_lng", "rewl_get_window_lng",
            "rewl_get_info", "rewl_get_state", "rewl_set_state", "rewl_destroy", "rewl_status_str",
            "rewl_last_error", "rewl_sweep_noalloc", "rewl_server_create", "rewl_server_submit", "rewl_server_run",
            "rewl_server_poll", "rewl_server_result", "rewl_server_cancel", "rewl_server_destroy", "rewl_thermo",
            "rewl_thermo_jackknife", "rewl_plan_windows", "rewl_autotune"]
REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED, REQ_CANCELLED = range(5)


class RewlError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        super().__init__("%s failed: %s%s" % (where, STATUS.get(status, status), (" (%s)" % detail) if detail else ""))


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class rewl_model(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("q", ctypes.c_int32)]


class rewl_lattice(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("Lx", ctypes.c_int32), ("Ly", ctypes.c_int32), ("periodic", ctypes.c_int32)]


class rewl_params(ctypes.Structure):
    _fields_ = [("sweeps_per_exchange", ctypes.c_int32), ("sweeps_per_flat_check", ctypes.c_int32),
                ("lnf0", ctypes.c_double), ("entry_max_sweeps", ctypes.c_int32), ("discovery_sweeps", ctypes.c_int32),
                ("timeout_ms", ctypes.c_int64), ("stream", ctypes.c_void_p), ("lanes_per_walker", ctypes.c_int32),
                ("walkers_per_block", ctypes.c_int32), ("mode", ctypes.c_int32), ("alloc", ALLOC_FN),
                ("free", FREE_FN), ("alloc_user", ctypes.c_void_p), ("profile", ctypes.c_int32),
                ("sweep_variant", ctypes.c_int32), ("prefetch_draws", ctypes.c_int32), ("wl_rule", ctypes.c_int32),
                ("window_starts", ctypes.c_void_p), ("window_widths", ctypes.c_void_p),
                ("wait_cycles", ctypes.c_int64), ("server_walker_target", ctypes.c_int32)]


class rewl_info(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("model", "q", "L", "N", "windows", "walkers_per_window", "window_bins", "n_bins", "e_min", "e_max",
                 "e_step", "lattice_words", "lanes_per_walker", "walkers_per_block", "mode", "windows_done")] + \
               [("sweep_clock", ctypes.c_int64), ("exchange_rounds", ctypes.c_int64), ("attempts", ctypes.c_int64),
                ("sweep_launches", ctypes.c_int64), ("sweep_ms", ctypes.c_double), ("h2d_bytes", ctypes.c_int64),
                ("d2h_bytes", ctypes.c_int64), ("prefetch_draws", ctypes.c_int32), ("sweep_variant", ctypes.c_int32)]


class rewl_sweep_desc(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("q", ctypes.c_int32), ("L", ctypes.c_int32), ("windows", ctypes.c_int32),
                ("walkers_per_window", ctypes.c_int32), ("window_bins", ctypes.c_int32), ("e_min", ctypes.c_int32),
                ("e_step", ctypes.c_int32), ("seed", ctypes.c_uint64), ("first_sweep", ctypes.c_uint64),
                ("sweeps", ctypes.c_int32), ("lanes_per_walker", ctypes.c_int32), ("status", ctypes.c_void_p)]


class rewl_request(ctypes.Structure):
    _fields_ = [("model", rewl_model), ("lattice", rewl_lattice), ("couplings", ctypes.c_void_p),
                ("windows", ctypes.c_int32), ("overlap", ctypes.c_double), ("walkers_per_window", ctypes.c_int32),
                ("flatness", ctypes.c_double), ("lnf_final", ctypes.c_double), ("seed", ctypes.c_uint64)]


class rewl_request_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("error", ctypes.c_int32), ("queued_ms", ctypes.c_double),
                ("run_ms", ctypes.c_double), ("latency_ms", ctypes.c_double), ("sweeps", ctypes.c_int64),
                ("attempts", ctypes.c_int64), ("device_bytes", ctypes.c_int64)]


class rewl_server_stats(ctypes.Structure):
    _fields_ = [("running", ctypes.c_int32), ("queued", ctypes.c_int32), ("finished", ctypes.c_int32),
                ("failed", ctypes.c_int32), ("rounds", ctypes.c_int64), ("attempts", ctypes.c_int64),
                ("device_bytes_in_use", ctypes.c_int64)]


class rewl_tune_result(ctypes.Structure):
    _fields_ = [("sweep_variant", ctypes.c_int32), ("lanes_per_walker", ctypes.c_int32),
                ("walkers_per_block", ctypes.c_int32), ("status", ctypes.c_int32), ("ms_per_launch", ctypes.c_double),
                ("attempts_per_s", ctypes.c_double)]


class rewl_state(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in
                ("lattice", "E", "lng", "H", "win_start", "lnf", "iteration", "done", "wl_accept", "near_ties",
                 "exact_tests", "x_tried", "x_accepted")] + \
               [("sweep_clock", ctypes.c_int64), ("exchange_rounds", ctypes.c_int64), ("stage", ctypes.c_void_p),
                ("win_width", ctypes.c_void_p), ("first_iter", ctypes.c_void_p), ("rep_id", ctypes.c_void_p),
                ("rep_state", ctypes.c_void_p), ("rep_trips", ctypes.c_void_p)]


_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load librewl.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError("librewl.so is not built; run __graft_entry__.build()")
    L = ctypes.CDLL(_build.LIB)
    P = ctypes.c_void_p
    L.rewl_params_default.argtypes = [ctypes.POINTER(rewl_params)]
    L.rewl_params_default.restype = None
    L.rewl_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(rewl_model), ctypes.POINTER(rewl_lattice), P,
                              ctypes.c_int32, ctypes.c_double, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                              ctypes.c_uint64, ctypes.POINTER(rewl_params)]
    L.rewl_create.restype = ctypes.c_int
    L.rewl_step.argtypes = [P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)]
    L.rewl_step.restype = ctypes.c_int
    L.rewl_get_lng.argtypes = [P, P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                               ctypes.POINTER(ctypes.c_int32)]
    L.rewl_get_lng.restype = ctypes.c_int
    L.rewl_get_window_lng.argtypes = [P, ctypes.c_int32, ctypes.c_int32, P, ctypes.c_int32,
                                      ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
    L.rewl_get_window_lng.restype = ctypes.c_int
    L.rewl_get_info.argtypes = [P, ctypes.POINTER(rewl_info)]
    L.rewl_get_info.restype = ctypes.c_int
    L.rewl_get_state.argtypes = [P, ctypes.POINTER(rewl_state)]
    L.rewl_get_state.restype = ctypes.c_int
    L.rewl_set_state.argtypes = [P, ctypes.POINTER(rewl_state)]
    L.rewl_set_state.restype = ctypes.c_int
    L.rewl_destroy.argtypes = [P]
    L.rewl_destroy.restype = None
    L.rewl_status_str.argtypes = [ctypes.c_int]
    L.rewl_status_str.restype = ctypes.c_char_p
    L.rewl_last_error.argtypes = []
    L.rewl_last_error.restype = ctypes.c_char_p
    L.rewl_sweep_noalloc.argtypes = [ctypes.POINTER(rewl_sweep_desc)] + [P] * 8
    L.rewl_sweep_noalloc.restype = ctypes.c_int
    L.rewl_server_create.argtypes = [ctypes.POINTER(P), ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(rewl_params)]
    L.rewl_server_create.restype = ctypes.c_int
    L.rewl_server_submit.argtypes = [P, ctypes.POINTER(rewl_request), ctypes.POINTER(ctypes.c_uint64)]
    L.rewl_server_submit.restype = ctypes.c_int
    L.rewl_server_run.argtypes = [P, ctypes.c_int32, ctypes.POINTER(rewl_server_stats)]
    L.rewl_server_run.restype = ctypes.c_int
    L.rewl_server_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(rewl_request_info)]
    L.rewl_server_poll.restype = ctypes.c_int
    L.rewl_server_result.argtypes = [P, ctypes.c_uint64, P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
    L.rewl_server_result.restype = ctypes.c_int
    L.rewl_server_cancel.argtypes = [P, ctypes.c_uint64]
    L.rewl_server_cancel.restype = ctypes.c_int
    L.rewl_server_destroy.argtypes = [P]
    L.rewl_server_destroy.restype = None
    L.rewl_thermo.argtypes = [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, ctypes.c_int32, P]
    L.rewl_thermo_jackknife.argtypes = [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P,
                                        ctypes.c_int32, P, P]
    L.rewl_thermo_jackknife.restype = ctypes.c_int
    L.rewl_plan_windows.argtypes = [P, P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, P, P]
    L.rewl_plan_windows.restype = ctypes.c_int
    L.rewl_autotune.argtypes = [P, P, P, ctypes.c_int32, ctypes.c_double, ctypes.c_int32, ctypes.c_double,
                                ctypes.c_double, ctypes.c_uint64, P, ctypes.c_int32, P, ctypes.c_int32,
                                ctypes.POINTER(ctypes.c_int32), P]
    L.rewl_autotune.restype = ctypes.c_int
    L.rewl_thermo.restype = ctypes.c_int
    _lib = L
    return L


def _check(st, where):
    if st != 0:
        raise RewlError(st, where, load().rewl_last_error().decode())


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


# ---------------------------------------------------------------- C names
def rewl_params_default():
    p = rewl_params()
    load().rewl_params_default(ctypes.byref(p))
    return p


def rewl_create(model, lattice, couplings, windows, overlap, walkers_per_window, flatness, lnf_final, seed,
                params=None):
    h = ctypes.c_void_p()
    cpl = None if couplings is None else np.ascontiguousarray(couplings, dtype=np.int8)
    if cpl is not None and cpl.size != lattice.dim * lattice.Lx ** lattice.dim:
        raise ValueError("couplings: %d values for %d sites in %d dimensions" %
                         (cpl.size, lattice.Lx ** lattice.dim, lattice.dim))
    st = load().rewl_create(ctypes.byref(h), ctypes.byref(model), ctypes.byref(lattice), _p(cpl), windows, overlap,
                            walkers_per_window, flatness, lnf_final, ctypes.c_uint64(seed),
                            ctypes.byref(params) if params is not None else None)
    _check(st, "rewl_create")
    return h


def rewl_step(h, max_sweeps):
    done = ctypes.c_int32(0)
    _check(load().rewl_step(h, max_sweeps, ctypes.byref(done)), "rewl_step")
    return bool(done.value)


def rewl_get_info(h):
    i = rewl_info()
    _check(load().rewl_get_info(h, ctypes.byref(i)), "rewl_get_info")
    return {k: getattr(i, k) for k, _ in rewl_info._fields_}


def rewl_get_lng(h, capacity):
    out = np.empty(capacity, np.float64)
    n, e0, de = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().rewl_get_lng(h, _p(out), capacity, ctypes.byref(n), ctypes.byref(e0), ctypes.byref(de)),
           "rewl_get_lng")
    return out[:n.value], e0.value, de.value


def rewl_get_window_lng(h, window, walker, capacity):
    out = np.empty(capacity, np.float64)
    lo, n = ctypes.c_int32(), ctypes.c_int32()
    _check(load().rewl_get_window_lng(h, window, walker, _p(out), capacity, ctypes.byref(lo), ctypes.byref(n)),
           "rewl_get_window_lng")
    return out[:n.value], lo.value


def rewl_get_state(h, info):
    nW = info["windows"] * info["walkers_per_window"]
    w, hw = info["window_bins"], info["windows"]
    a = {"lattice": np.zeros((nW, info["lattice_words"]), np.uint32), "E": np.zeros(nW, np.int32),
         "lng": np.zeros((nW, w), np.float64), "H": np.zeros((nW, w), np.uint32),
         "win_start": np.zeros(hw, np.int32), "lnf": np.zeros(hw, np.float64), "iteration": np.zeros(hw, np.int32),
         "done": np.zeros(hw, np.int32), "wl_accept": np.zeros(nW, np.uint64), "near_ties": np.zeros(nW, np.uint64),
         "exact_tests": np.zeros(nW, np.uint64), "x_tried": np.zeros(hw, np.uint64),
         "x_accepted": np.zeros(hw, np.uint64), "stage": np.zeros(hw, np.int32), "win_width": np.zeros(hw, np.int32),
         "first_iter": np.zeros(hw, np.int64), "rep_id": np.zeros(nW, np.int32), "rep_state": np.zeros(nW, np.int32),
         "rep_trips": np.zeros(nW, np.int64)}
    s = rewl_state(**{k: _p(v) for k, v in a.items()})
    _check(load().rewl_get_state(h, ctypes.byref(s)), "rewl_get_state")
    a["sweep_clock"], a["exchange_rounds"] = s.sweep_clock, s.exchange_rounds
    return a


def rewl_set_state(h, state):
    keys = [k for k, _ in rewl_state._fields_ if k not in ("sweep_clock", "exchange_rounds", "win_width")]
    arrs = {k: (np.ascontiguousarray(state[k]) if state.get(k) is not None else None) for k in keys}
    s = rewl_state(**{k: _p(v) for k, v in arrs.items()})
    s.sweep_clock, s.exchange_rounds = int(state["sweep_clock"]), int(state["exchange_rounds"])
    _check(load().rewl_set_state(h, ctypes.byref(s)), "rewl_set_state")


def rewl_destroy(h):
    load().rewl_destroy(h)


def rewl_sweep_noalloc(desc, lattice, E, lng, H, coupling_bits, win_start, lnf, stream=None):
    """WL sweeps on caller-owned device buffers (integer device addresses, e.g.
    torch tensor .data_ptr()); the library allocates nothing for this call."""
    ptrs = [ctypes.c_void_p(p) if p else None for p in (lattice, E, lng, H, coupling_bits, win_start, lnf, stream)]
    _check(load().rewl_sweep_noalloc(ctypes.byref(desc), *ptrs), "rewl_sweep_noalloc")


def rewl_thermo(lng, e_min, e_step, temperatures):
    """Canonical ln Z, U, C, F, S (columns) at each temperature, from ln g."""
    g = np.ascontiguousarray(lng, dtype=np.float64)
    T = np.ascontiguousarray(temperatures, dtype=np.float64)
    out = np.zeros((len(T), 5), np.float64)
    _check(load().rewl_thermo(_p(g), len(g), e_min, e_step, _p(T), len(T), _p(out)), "rewl_thermo")
    return out


def rewl_autotune(model, L, windows, overlap, walkers_per_window, flatness, lnf_final, seed, q=2, couplings=None,
                  sweeps=200, sweeps_per_exchange=100, sweeps_per_flat_check=1000):
    """Times the sweep launch shapes on this problem (rewl_autotune): returns
    (the keyword arguments of the fastest for REWL(), the list of results)."""
    if isinstance(model, str):
        model = MODELS[model]
    p = rewl_params_default()
    p.sweeps_per_exchange, p.sweeps_per_flat_check = sweeps_per_exchange, sweeps_per_flat_check
    cpl = None if couplings is None else np.ascontiguousarray(couplings, dtype=np.int8)
    res = (rewl_tune_result * 8)()
    n = ctypes.c_int32()
    best = rewl_params()
    dim = 3 if model == EA_PM_J_3D else 2
    _check(load().rewl_autotune(ctypes.byref(rewl_model(model, q)), ctypes.byref(rewl_lattice(dim, L, L, 1)), _p(cpl),
                                windows, overlap, walkers_per_window, flatness, lnf_final, ctypes.c_uint64(seed),
                                ctypes.byref(p), sweeps, res, 8, ctypes.byref(n), ctypes.byref(best)), "rewl_autotune")
    out = [{k: getattr(res[i], k) for k, _ in rewl_tune_result._fields_} for i in range(n.value)]
    kw = {"sweep_variant": best.sweep_variant, "lanes_per_walker": best.lanes_per_walker,
          "walkers_per_block": best.walkers_per_block}
    return kw, out


def rewl_plan_windows(first_iter_sweeps, pre_starts, pre_widths, n_bins, windows, overlap):
    """Run-time balanced partition (Fig. 1b) from a pre-run: (starts, widths)."""
    f = np.ascontiguousarray(first_iter_sweeps, dtype=np.int64)
    ps = np.ascontiguousarray(pre_starts, dtype=np.int32)
    pw = np.ascontiguousarray(pre_widths, dtype=np.int32)
    st = np.zeros(windows, np.int32)
    wd = np.zeros(windows, np.int32)
    _check(load().rewl_plan_windows(_p(f), _p(ps), _p(pw), len(ps), int(n_bins), int(windows), float(overlap), _p(st),
                                    _p(wd)), "rewl_plan_windows")
    return st, wd


def rewl_thermo_jackknife(lng_runs, e_min, e_step, temperatures):
    """rewl_thermo's quantities of the mean ln g over runs, with jackknife
    errors over the runs: (estimate, error), each [n_T][5]."""
    g = np.ascontiguousarray(lng_runs, dtype=np.float64)
    T = np.ascontiguousarray(temperatures, dtype=np.float64)
    est = np.zeros((len(T), 5), np.float64)
    err = np.zeros((len(T), 5), np.float64)
    _check(load().rewl_thermo_jackknife(_p(g), g.shape[0], g.shape[1], e_min, e_step, _p(T), len(T), _p(est), _p(err)),
           "rewl_thermo_jackknife")
    return est, err


def rewl_status_str(status):
    return load().rewl_status_str(status).decode()


def rewl_last_error():
    return load().rewl_last_error().decode()


# ---------------------------------------------------------------- wrapper
def _torch_allocator():
    import torch

    def alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream)
        except Exception:
            return None

    def free(ptr, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    return ALLOC_FN(alloc), FREE_FN(free)


class REWL:
    """One REWL solve on the GPU.  Arguments mirror ``rewl_create``."""

    def __init__(self, model, L, windows, overlap, walkers_per_window, flatness, lnf_final, seed, q=2,
                 couplings=None, sweeps_per_exchange=100, sweeps_per_flat_check=1000, lnf0=1.0,
                 entry_max_sweeps=1000, discovery_sweeps=200, timeout_ms=0, lanes_per_walker=0,
                 walkers_per_block=0, mode=MODE_PLAIN, stream=None, torch_allocator=False, profile=False,
                 sweep_variant=-1, prefetch_draws=0, wl_rule=0, window_starts=None, window_widths=None,
                 wait_cycles=0):
        if isinstance(model, str):
            model = MODELS[model]
        p = rewl_params_default()
        p.sweeps_per_exchange, p.sweeps_per_flat_check, p.lnf0 = sweeps_per_exchange, sweeps_per_flat_check, lnf0
        p.entry_max_sweeps, p.discovery_sweeps, p.timeout_ms = entry_max_sweeps, discovery_sweeps, timeout_ms
        p.lanes_per_walker, p.walkers_per_block, p.mode = lanes_per_walker, walkers_per_block, mode
        p.profile = 1 if profile else 0
        p.sweep_variant = sweep_variant
        p.prefetch_draws = prefetch_draws
        p.wait_cycles = int(wait_cycles)
        p.wl_rule = WL_RULES[wl_rule] if isinstance(wl_rule, str) else wl_rule
        if window_starts is not None:
            self._win = (np.ascontiguousarray(window_starts, dtype=np.int32),
                         np.ascontiguousarray(window_widths, dtype=np.int32))
            p.window_starts, p.window_widths = self._win[0].ctypes.data, self._win[1].ctypes.data
        if stream is not None:
            p.stream = ctypes.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
        self._keep = None
        if torch_allocator:
            self._keep = _torch_allocator()
            p.alloc, p.free = self._keep
        self.params = p
        self._h = None
        dim = 3 if model == EA_PM_J_3D else 2
        self._h = rewl_create(rewl_model(model, q), rewl_lattice(dim, L, L, 1), couplings, windows, overlap,
                              walkers_per_window, flatness, lnf_final, seed, p)
        self.info = rewl_get_info(self._h)

    def close(self):
        if self._h:
            rewl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, max_sweeps):
        done = rewl_step(self._h, max_sweeps)
        self.info = rewl_get_info(self._h)
        return done

    def lng(self):
        return rewl_get_lng(self._h, self.info["n_bins"])

    def window_lng(self, window, walker=-1):
        return rewl_get_window_lng(self._h, window, walker, self.info["window_bins"])

    def state(self):
        return rewl_get_state(self._h, rewl_get_info(self._h))

    def set_state(self, state):
        rewl_set_state(self._h, state)
        self.info = rewl_get_info(self._h)


class RewlServer:
    """Served form: many REWL requests admitted by slots and device memory and
    run together (rewl_server_* of include/rewl.h)."""

    def __init__(self, device_bytes, max_running, sweeps_per_exchange=100, sweeps_per_flat_check=1000, lnf0=1.0,
                 entry_max_sweeps=1000, discovery_sweeps=200, stream=None, wl_rule=0, timeout_ms=0,
                 walker_target=0):
        L = load()
        p = rewl_params_default()
        p.sweeps_per_exchange, p.sweeps_per_flat_check, p.lnf0 = sweeps_per_exchange, sweeps_per_flat_check, lnf0
        p.entry_max_sweeps, p.discovery_sweeps = entry_max_sweeps, discovery_sweeps
        p.wl_rule = WL_RULES[wl_rule] if isinstance(wl_rule, str) else wl_rule
        p.timeout_ms = timeout_ms
        p.server_walker_target = int(walker_target)
        if stream is not None:
            p.stream = ctypes.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
        self._h = None
        h = ctypes.c_void_p()
        _check(L.rewl_server_create(ctypes.byref(h), int(device_bytes), int(max_running), ctypes.byref(p)),
               "rewl_server_create")
        self._h = h
        self._keep = {}

    def close(self):
        if self._h:
            load().rewl_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, model, L, windows, overlap, walkers_per_window, flatness, lnf_final, seed, q=2, couplings=None):
        if isinstance(model, str):
            model = MODELS[model]
        cpl = None if couplings is None else np.ascontiguousarray(couplings, dtype=np.int8)
        if cpl is not None and cpl.size != (3 * L ** 3 if model == EA_PM_J_3D else 2 * L * L):
            raise ValueError("couplings: wrong number of values")
        r = rewl_request(rewl_model(model, q), rewl_lattice(3 if model == EA_PM_J_3D else 2, L, L, 1), _p(cpl),
                         windows, overlap,
                         walkers_per_window, flatness, lnf_final, seed)
        rid = ctypes.c_uint64()
        _check(load().rewl_server_submit(self._h, ctypes.byref(r), ctypes.byref(rid)), "rewl_server_submit")
        return rid.value

    def run(self, max_rounds):
        st = rewl_server_stats()
        _check(load().rewl_server_run(self._h, int(max_rounds), ctypes.byref(st)), "rewl_server_run")
        return {k: getattr(st, k) for k, _ in rewl_server_stats._fields_}

    def poll(self, rid):
        i = rewl_request_info()
        _check(load().rewl_server_poll(self._h, rid, ctypes.byref(i)), "rewl_server_poll")
        return {k: getattr(i, k) for k, _ in rewl_request_info._fields_}

    def result(self, rid, capacity=1 << 16):
        out = np.empty(capacity, np.float64)
        n, e0, de = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(load().rewl_server_result(self._h, rid, _p(out), capacity, ctypes.byref(n), ctypes.byref(e0),
                                         ctypes.byref(de)), "rewl_server_result")
        return out[:n.value], e0.value, de.value

    def cancel(self, rid):
        _check(load().rewl_server_cancel(self._h, rid), "rewl_server_cancel")


def unpack_lattice(words, L, model):
    """Packed configurations [walkers][lattice_words] -> site values [walkers][N]
    (site i = y*L + x; on the cube i = (z*L + y)*L + x, row z*L + y), following
    the layout documented in include/rewl.h."""
    words = np.asarray(words, dtype=np.uint32)
    n = words.shape[0]
    rows = L * L if model == EA_PM_J_3D else L
    out = np.zeros((n, rows * L), np.uint8)
    if model == POTTS:
        Wr = (L + 7) // 8
        for y in range(rows):
            for x in range(L):
                out[:, y * L + x] = (words[:, y * Wr + x // 8] >> (4 * (x % 8))) & 15
    else:
        Wr = (L + 31) // 32
        for y in range(rows):
            for x in range(L):
                out[:, y * L + x] = (words[:, y * Wr + x // 32] >> (x % 32)) & 1
    return out
