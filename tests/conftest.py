import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a); runs the CUDA library")
    config.addinivalue_line("markers", "slow: CPU test that takes more than ~20 s")


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "curand_philox4x32_x.h")):
            return os.path.join(d, "include")
    return None


@pytest.fixture(scope="session")
def curand_philox(tmp_path_factory):
    """NVIDIA's own Philox4x32-10 (curand header, host code path), compiled
    from the toolkit header by the host C++ compiler."""
    import ctypes

    inc = _cuda_include()
    if inc is None:
        pytest.skip("CUDA headers not found")
    out = tmp_path_factory.mktemp("curandref") / "libcurandref.so"
    src = os.path.join(ROOT, "tests", "helpers", "curand_philox_host.cpp")
    subprocess.check_call(["g++", "-O1", "-fPIC", "-shared", "-I", inc, "-o", str(out), src])
    lib = ctypes.CDLL(str(out))
    lib.curand_philox_ref.argtypes = [ctypes.c_void_p] * 3
    return lib
