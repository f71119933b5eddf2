"""CPU checks of the C ABI: the library builds, loads and exports every entry
point declared in include/tpss.h (no compute calls without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "tpss.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tpss_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1910_11239_gb300 import build_lib, tpss
    if not os.path.exists(tpss.LIB_PATH):
        build_lib.build()
    return tpss.LIB_PATH


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["tpss_create", "tpss_destroy", "tpss_setup_patches", "tpss_smooth_additive",
                 "tpss_smooth_multiplicative", "tpss_apply_operator", "tpss_vcycle", "tpss_pcg_solve"]:
        assert name in syms


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [s for s in declared_symbols() if not hasattr(L, s)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libpath):
    from paper_1910_11239_gb300 import tpss
    assert set(declared_symbols()) <= set(tpss.SIGNATURES)
    tpss.lib()


def test_last_error_is_empty_string_initially(libpath):
    from paper_1910_11239_gb300 import tpss
    assert tpss.lib().tpss_last_error() == b""


def test_null_arguments_rejected_without_gpu(libpath):
    # argument checks happen on the host before any CUDA call
    from paper_1910_11239_gb300 import tpss
    L = tpss.lib()
    assert L.tpss_create(None, None, None) == -1
    assert b"null" in L.tpss_last_error()
    assert L.tpss_smooth_additive(None, 0.7, 1, None, None, 1) == -1
    assert L.tpss_pcg_solve(None, None, None, 1e-8, 10, None, None, None) == -1
