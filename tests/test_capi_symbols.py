"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point that include/mgmlmc.h declares (no GPU work)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(mgmlmc_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2211_15383_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["mgmlmc_create", "mgmlmc_set_gauge", "mgmlmc_set_mass", "mgmlmc_set_hierarchy",
                     "mgmlmc_compute_deflation", "mgmlmc_estimate_level", "mgmlmc_estimate_trace",
                     "mgmlmc_destroy", "mgmlmc_last_error"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in sorted(declared_functions()):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_binding_covers_the_header():
    from paper_2211_15383_gb300 import _lib
    bound = {name for name, _, _ in _lib.SIGNATURES}
    assert bound == declared_functions()


def test_options_struct_matches(lib):
    from paper_2211_15383_gb300 import _lib
    _lib._lib = None
    o = _lib.Options()
    lib.mgmlmc_default_options(ctypes.byref(o))
    assert o.mg_precision == 64 and o.solve_tol == 1e-12 and o.max_block_rhs == 256


def test_invalid_arguments_rejected_without_gpu(lib):
    # calls that fail argument validation before touching the device
    lib.mgmlmc_create.restype = ctypes.c_int
    assert lib.mgmlmc_create(None, None, None, None, None, None) == -1
    lib.mgmlmc_set_mass.argtypes = [ctypes.c_void_p, ctypes.c_double]
    assert lib.mgmlmc_set_mass(None, 0.1) == -1
