"""Microbenchmarks of the GB300 rates that bound the REWL sweep kernel
(rates.cu): integer issue rates of the instruction mixes a trial needs (the
Philox round's 32x32->64 multiply with a three-input XOR, the 32-bit
multiply, add and XOR), FP64 add, log / logf and Philox throughput,
shared-memory and shuffle latency, and the latency of the sequential WL step
on its own.  Measurement tooling beside bench.py, not part of the library:
bench.py's roofline reads the committed summary in profiles/.

    python -m ubench     # build (nvcc, sm_103a) and run on the current GPU
"""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.join(ROOT, "ubench")
CSRC = os.path.join(ROOT, "paper_1305_5615_gb300", "csrc")
OUT_DIR = os.path.join(HERE, "_build")
EXE = os.path.join(OUT_DIR, "ubench_rates")


def build():
    """Compiles rates.cu into an executable under ubench/_build."""
    import sys

    sys.path.insert(0, ROOT)
    from paper_1305_5615_gb300 import _build

    os.makedirs(OUT_DIR, exist_ok=True)
    src = os.path.join(HERE, "rates.cu")
    deps = [src, os.path.join(CSRC, "rewl_device.cuh"), os.path.join(CSRC, "rewl_layout.h")]
    if _build._stale(EXE, deps):
        cmd = [_build.nvcc()] + _build.ARCH + ["-O3", "-lineinfo", "-std=c++17", "-I" + CSRC,
                                               "-I" + os.path.join(ROOT, "include"), "-o", EXE + ".tmp", src]
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
