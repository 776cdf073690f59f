"""Microbenchmarks of the GB300 rates that bound the REWL sweep kernel
(rates.cu): FP64 add, log / logf and Philox throughput, shared-memory and
shuffle latency, and the latency of the sequential WL step on its own.

    python -m paper_1305_5615_gb300.ubench     # build (nvcc, sm_103a) and run on the current GPU
"""
import os
import subprocess

from .. import _build

HERE = os.path.dirname(os.path.abspath(__file__))
EXE = os.path.join(_build.OUT_DIR, "ubench_rates")


def build():
    """Compiles rates.cu into an executable next to the library's objects."""
    os.makedirs(_build.OUT_DIR, exist_ok=True)
    src = os.path.join(HERE, "rates.cu")
    deps = [src, os.path.join(_build.CSRC, "rewl_device.cuh"), os.path.join(_build.CSRC, "rewl_layout.h")]
    if _build._stale(EXE, deps):
        cmd = [_build.nvcc()] + _build.ARCH + ["-O3", "-lineinfo", "-std=c++17", "-I" + _build.CSRC,
                                               "-I" + os.path.join(os.path.dirname(_build.HERE), "include"),
                                               "-o", EXE + ".tmp", src]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for rates.cu:\n%s%s" % (r.stdout, r.stderr))
        os.replace(EXE + ".tmp", EXE)
    return EXE


def run():
    """Builds if needed, runs on the current GPU and returns the printed table."""
    r = subprocess.run([build()], capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        raise RuntimeError("ubench_rates failed:\n%s%s" % (r.stdout, r.stderr))
    return r.stdout
