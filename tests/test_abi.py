"""CPU checks of the boundary: the library builds for sm_103a, loads, and
exports every entry point that include/rewl.h declares.  No compute call is
made (there is no GPU here)."""
import os
import re

import pytest

from paper_1305_5615_gb300 import rewl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rewl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rewl_[a-z_]+)\s*\(", src)) - {"rewl_alloc_fn", "rewl_free_fn"})


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("rewl_create", "rewl_step", "rewl_get_lng", "rewl_destroy"):
        assert n in names


def test_library_loads_and_exports_every_declared_symbol():
    lib = rewl.load()
    for n in declared_functions():
        assert hasattr(lib, n), n
    assert sorted(rewl.EXPORTED) == declared_functions()


def test_status_strings_need_no_gpu():
    assert rewl.rewl_status_str(0) == "ok"
    assert "window" in rewl.rewl_status_str(5)
    p = rewl.rewl_params_default()
    assert (p.sweeps_per_exchange, p.sweeps_per_flat_check, p.lnf0) == (100, 1000, 1.0)


def test_create_fails_cleanly_without_a_suitable_device():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(rewl.RewlError) as e:
        rewl.REWL("ising", 8, 4, 0.75, 2, 0.8, 1e-6, 0)
    assert e.value.status in (3, 9)


STRUCTS = ("rewl_model", "rewl_lattice", "rewl_params", "rewl_info", "rewl_sweep_desc", "rewl_request",
           "rewl_request_info", "rewl_server_stats", "rewl_state", "rewl_tune_result")


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets
    that a C compiler gives the header's struct (gcc, plain C)."""
    import ctypes
    import shutil
    import subprocess

    if not shutil.which("gcc"):
        pytest.skip("no gcc")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "rewl.h"', "int main(void) {"]
    for name in STRUCTS:
        cls = getattr(rewl, name)
        lines.append('  printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for f, _ in cls._fields_:
            lines.append('  printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n") if l)
    for name in STRUCTS:
        cls = getattr(rewl, name)
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got["%s.%s" % (name, f)]) == getattr(cls, f).offset, (name, f)


def test_binding_marshals_every_option_without_a_device():
    """Every keyword of the Python classes reaches the C call (which then fails
    cleanly without a GPU) -- no error in the argument marshalling itself."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(rewl.RewlError):
        rewl.REWL("ising", 8, 4, 0.75, 2, 0.8, 1e-6, 0, q=2, couplings=None, sweeps_per_exchange=100,
                  sweeps_per_flat_check=1000, lnf0=1.0, entry_max_sweeps=1000, discovery_sweeps=200,
                  lanes_per_walker=32, walkers_per_block=1, mode=rewl.MODE_PLAIN, profile=True, sweep_variant=2,
                  prefetch_draws=0, wl_rule="1/t", window_starts=[0, 10, 20, 30], window_widths=[20, 20, 20, 35],
                  wait_cycles=1 << 20)
    with pytest.raises(rewl.RewlError):
        rewl.RewlServer(device_bytes=1 << 30, max_running=4, sweeps_per_exchange=100, sweeps_per_flat_check=1000,
                        lnf0=1.0, entry_max_sweeps=1000, discovery_sweeps=200, wl_rule="1/t", timeout_ms=1000,
                        walker_target=0)
