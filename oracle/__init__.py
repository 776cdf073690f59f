"""Plain CPU oracle for replica-exchange Wang-Landau (REWL) sampling.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  It shares
no code with the CUDA library (``paper_1305_5615_gb300``) and imports nothing
from it; both sides only receive the same seeded inputs.

Contents
  * ``rewl_oracle.c``  -- single-threaded REWL exactly as the paper states it
    (WL walk, windows, exchange Eq. (1), flatness, merging, termination), with
    its own Philox4x32-10 written from Salmon et al. (SC'11).
  * ``join.py``        -- joining of the window fragments where the inverse
    microcanonical temperatures agree best, and normalisation.
  * ``exact_dos.py``   -- exact densities of states (enumeration, transfer
    matrix, Kaufman/Beale closed form) that pin the oracle's converged output.

Parity status of each function is listed at the top of its module.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

ISING, POTTS, EA, EA3 = 0, 1, 2, 3
MODEL_NAMES = {"ising": ISING, "potts": POTTS, "ea": EA, "ea3d": EA3}
WL_RULES = {"flat": 0, "1/t": 1}


def build(force=False):
    """Compile the oracle with plain gcc.  -ffp-contract=off keeps every FP64
    operation a separate IEEE operation on x86-64 and aarch64 alike."""
    src = os.path.join(_HERE, "rewl_oracle.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "rewl_oracle.h"))):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-Wall", "-Wno-unused-function", "-o", tmp, src, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("sweeps_per_exchange", ctypes.c_int), ("sweeps_per_flat_check", ctypes.c_int),
                ("lnf0", ctypes.c_double), ("entry_max_sweeps", ctypes.c_int),
                ("discovery_sweeps", ctypes.c_int), ("wl_rule", ctypes.c_int),
                ("window_starts", ctypes.c_void_p), ("window_widths", ctypes.c_void_p)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.c_int, ctypes.c_int, P, ctypes.c_int,
                                 ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                 ctypes.POINTER(_Params)]
        L.orc_create.restype = ctypes.c_int
        L.orc_destroy.argtypes = [P]
        L.orc_run_blocks.argtypes = [P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int)]
        L.orc_run_blocks.restype = ctypes.c_int
        L.orc_active_windows.argtypes = [P]
        L.orc_active_windows.restype = ctypes.c_int
        L.orc_block_sweeps.argtypes = [P, ctypes.c_int, ctypes.c_int]
        L.orc_block_finish.argtypes = [P]
        L.orc_info.argtypes = [P, P]
        L.orc_get_windows.argtypes = [P, P, P, P, P]
        L.orc_get_phase.argtypes = [P, P]
        L.orc_get_window_layout.argtypes = [P, P, P]
        L.orc_get_replicas.argtypes = [P, P, P, P]
        L.orc_walker_all_seen.argtypes = [P, ctypes.c_int]
        L.orc_walker_all_seen.restype = ctypes.c_int
        L.orc_get_walkers.argtypes = [P, P, P, P, P]
        L.orc_get_couplings.argtypes = [P, P]
        L.orc_get_counters.argtypes = [P, P, P, P, P]
        L.orc_set_walker_lng.argtypes = [P, ctypes.c_int, P]
        L.orc_set_window_lnf.argtypes = [P, ctypes.c_int, ctypes.c_double]
        L.orc_set_walker_H.argtypes = [P, ctypes.c_int, P]
        L.orc_philox4x32_10.argtypes = [P, P, P]
        L.orc_walker_is_flat.argtypes = [P, ctypes.c_int]
        L.orc_walker_is_flat.restype = ctypes.c_int
        L.orc_energy.argtypes = [P, P]
        L.orc_energy.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def philox4x32_10(ctr, key):
    """Philox4x32-10 of one 128-bit counter and 64-bit key (oracle copy)."""
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


class OracleREWL:
    """One REWL solve on the CPU oracle.  Arguments mirror ``rewl_create``."""

    def __init__(self, model, L, windows, overlap, walkers_per_window, flatness, lnf_final, seed, q=2,
                 couplings=None, sweeps_per_exchange=100, sweeps_per_flat_check=1000, lnf0=1.0,
                 entry_max_sweeps=1000, discovery_sweeps=200, wl_rule=0, window_starts=None, window_widths=None):
        if isinstance(model, str):
            model = MODEL_NAMES[model]
        if isinstance(wl_rule, str):
            wl_rule = WL_RULES[wl_rule]
        self._lib = lib()
        p = _Params(sweeps_per_exchange, sweeps_per_flat_check, lnf0, entry_max_sweeps, discovery_sweeps, wl_rule)
        if window_starts is not None:
            self._ws = np.ascontiguousarray(window_starts, dtype=np.int32)
            self._ww = np.ascontiguousarray(window_widths, dtype=np.int32)
            assert self._ws.shape == (windows,) and self._ww.shape == (windows,)
            p.window_starts, p.window_widths = self._ws.ctypes.data, self._ww.ctypes.data
        h = ctypes.c_void_p()
        cpl = None
        if couplings is not None:
            cpl = np.ascontiguousarray(couplings, dtype=np.int8)
        st = self._lib.orc_create(ctypes.byref(h), model, q, L, _ptr(cpl), windows, overlap, walkers_per_window,
                                  flatness, lnf_final, ctypes.c_uint64(seed), ctypes.byref(p))
        if st != 0:
            raise RuntimeError("orc_create failed with status %d" % st)
        self._h = h
        self.model, self.q, self.L = model, (q if model == POTTS else 2), L
        info = self.info()
        self.N, self.h, self.m, self.w = info["N"], info["h"], info["m"], info["w"]
        self.n_bins, self.e_min, self.e_max, self.e_step = info["n_bins"], info["e_min"], info["e_max"], info["e_step"]

    def close(self):
        if getattr(self, "_h", None):
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def run_blocks(self, n_blocks, threads=1):
        """Runs n_blocks blocks (sweeps, exchange round, flatness check when
        due).  threads > 1 sweeps disjoint walker ranges of each block on that
        many host threads (orc_block_sweeps; the walkers of a block are
        independent, so the trials and results are the same), then finishes
        the block on this thread.  Returns True when every window is done."""
        if threads <= 1:
            done = ctypes.c_int(0)
            st = self._lib.orc_run_blocks(self._h, n_blocks, ctypes.byref(done))
            if st != 0:
                raise RuntimeError("orc_run_blocks failed with status %d" % st)
            return bool(done.value)
        import concurrent.futures

        n = self.h * self.m
        cuts = [n * i // threads for i in range(threads + 1)]
        ranges = [(cuts[i], cuts[i + 1]) for i in range(threads) if cuts[i + 1] > cuts[i]]
        with concurrent.futures.ThreadPoolExecutor(max_workers=len(ranges)) as ex:
            for _ in range(n_blocks):
                if self._lib.orc_active_windows(self._h) == 0:
                    break
                list(ex.map(lambda r: self._lib.orc_block_sweeps(self._h, r[0], r[1]), ranges))
                self._lib.orc_block_finish(self._h)
        return self._lib.orc_active_windows(self._h) == 0

    def block_sweeps(self):
        """The WL sweeps of one block (sweeps_per_exchange sweeps of every
        walker of the windows not done) and nothing else: no clock advance, no
        exchange, no flatness check."""
        self._lib.orc_block_sweeps(self._h, 0, self.h * self.m)

    def info(self):
        a = np.zeros(16, dtype=np.int64)
        self._lib.orc_info(self._h, _ptr(a))
        keys = ["model", "q", "L", "N", "h", "m", "w", "n_bins", "e_min", "e_max", "e_step", "sweep_clock", "xround"]
        return {k: int(a[i]) for i, k in enumerate(keys)}

    def windows(self):
        h = self.h
        start = np.zeros(h, np.int32)
        lnf = np.zeros(h, np.float64)
        it = np.zeros(h, np.int32)
        done = np.zeros(h, np.int32)
        phase = np.zeros(h, np.int32)
        width = np.zeros(h, np.int32)
        first = np.zeros(h, np.int64)
        self._lib.orc_get_windows(self._h, _ptr(start), _ptr(lnf), _ptr(it), _ptr(done))
        self._lib.orc_get_phase(self._h, _ptr(phase))
        self._lib.orc_get_window_layout(self._h, _ptr(width), _ptr(first))
        return {"start": start, "lnf": lnf, "iteration": it, "done": done, "phase": phase, "width": width,
                "first_iter": first}

    def walkers(self):
        n = self.h * self.m
        spins = np.zeros((n, self.N), np.uint8)
        E = np.zeros(n, np.int32)
        lng = np.zeros((n, self.w), np.float64)
        H = np.zeros((n, self.w), np.uint32)
        self._lib.orc_get_walkers(self._h, _ptr(spins), _ptr(E), _ptr(lng), _ptr(H))
        return {"spins": spins, "E": E, "lng": lng, "H": H}

    def couplings(self):
        J = np.zeros((3 if self.model == EA3 else 2) * self.N, np.int8)
        self._lib.orc_get_couplings(self._h, _ptr(J))
        return J

    def counters(self):
        n = self.h * self.m
        acc = np.zeros(n, np.uint64)
        ties = np.zeros(n, np.uint64)
        xt = np.zeros(self.h, np.uint64)
        xa = np.zeros(self.h, np.uint64)
        self._lib.orc_get_counters(self._h, _ptr(acc), _ptr(ties), _ptr(xt), _ptr(xa))
        return {"wl_accept": acc, "near_ties": ties, "x_tried": xt, "x_accepted": xa}

    def energy(self, spins):
        s = np.ascontiguousarray(spins, dtype=np.uint8)
        return int(self._lib.orc_energy(self._h, _ptr(s)))

    def replicas(self):
        """rep_id[W] (the replica walker W holds), rep_state and rep_trips per replica."""
        n = self.h * self.m
        rid, rst, rtr = np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n, np.int64)
        self._lib.orc_get_replicas(self._h, _ptr(rid), _ptr(rst), _ptr(rtr))
        return {"rep_id": rid, "rep_state": rst, "rep_trips": rtr}

    def walker_all_seen(self, W):
        return bool(self._lib.orc_walker_all_seen(self._h, W))

    def walker_is_flat(self, W):
        return bool(self._lib.orc_walker_is_flat(self._h, W))

    def set_walker_lng(self, W, lng):
        a = np.ascontiguousarray(lng, dtype=np.float64)
        assert a.shape == (self.w,)
        self._lib.orc_set_walker_lng(self._h, W, _ptr(a))

    def set_walker_H(self, W, H):
        a = np.ascontiguousarray(H, dtype=np.uint32)
        assert a.shape == (self.w,)
        self._lib.orc_set_walker_H(self._h, W, _ptr(a))

    def set_window_lnf(self, a, lnf):
        self._lib.orc_set_window_lnf(self._h, a, lnf)

    def window_lng(self):
        """Per-window ln g: the mean over the window's walkers, summed in walker
        order (identical to every walker's table right after a merge)."""
        lng = self.walkers()["lng"].reshape(self.h, self.m, self.w)
        out = lng[:, 0, :].copy()
        for k in range(1, self.m):
            out = out + lng[:, k, :]
        return out / float(self.m)

    def joined_lng(self):
        from .join import join_windows, normalise
        win = self.windows()
        g = join_windows(self.window_lng(), win["start"], win["width"], self.n_bins)
        return normalise(g, self.N, self.q)
