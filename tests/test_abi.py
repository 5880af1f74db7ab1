"""The C-ABI library builds, loads and exports every entry point include/lbmp.h declares.

CPU-only: no compute call is made. Without a GPU the library must refuse to create a
context (no CPU fallback)."""
import ctypes
import os
import re

import pytest

from paper_1105_2904_gb300 import build as B
from paper_1105_2904_gb300 import lbmp

HEADER = os.path.join(B.ROOT, "include", "lbmp.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return lbmp.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", src)))


def test_header_declares_the_binding_names():
    assert declared_functions() == sorted(lbmp.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_no_cpu_fallback_without_a_device(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    h = ctypes.c_void_p()
    st = lib.lbm_create(ctypes.byref(h), 1, 8, 8, 8, 0.7, None)
    assert st == 3 and not h.value   # LBM_E_CUDA


def test_invalid_arguments_are_rejected_before_device_use(lib):
    h = ctypes.c_void_p()
    assert lib.lbm_create(ctypes.byref(h), 1, 8, 8, 8, 0.5, None) == 1    # tau <= 1/2
    assert lib.lbm_create(ctypes.byref(h), 0, 8, 8, 2, 0.7, None) == 1    # D2Q9 needs nz = 1
    assert lib.lbm_create(ctypes.byref(h), 7, 8, 8, 8, 0.7, None) == 1    # unknown lattice
    assert lib.lbm_create(ctypes.byref(h), 1, 0, 8, 8, 0.7, None) == 1    # empty axis
    assert lib.lbm_create(ctypes.byref(h), 1, 2048, 2048, 1024, 0.7, None) == 1  # > 2^31 sites


def test_binding_rejects_unknown_names_before_device_use():
    with pytest.raises(ValueError):
        lbmp.Simulation(1, 8, 8, 8, 0.7, streaming="aa")
    with pytest.raises(ValueError):
        lbmp.Simulation(1, 8, 8, 8, 0.7, precision="fp8")
    # null context pointers are refused by every entry point that takes one
    lib = lbmp.load()
    assert lib.lbm_set_streaming(None, 1) == 1
    assert lib.lbm_diagnostics(None, None) == 1


def test_bounds_checked_build_compiles_and_exports():
    # The LBM_DEBUG build (index checks reporting LBM_E_BOUNDS through the device status word)
    # builds from the same sources and exports the same entry points.
    so = B.build(debug=True)
    assert so == B.SO_DEBUG and os.path.exists(so)
    dbg = ctypes.CDLL(so)
    for name in declared_functions():
        assert hasattr(dbg, name), name
