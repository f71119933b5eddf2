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
    # the schedule option, its failure-path test hook and the batch constructor
    assert L.tpss_patches_set_additive_schedule(None, 4) == -1
    assert L.tpss_patches_test_wait_expiry(None) == -1
    assert b"null" in L.tpss_last_error()
    assert L.tpss_batch_create(None, 1, 1, None, 4, None, None) == -1


def test_mapped_mesh_arguments_are_checked_on_the_host(libpath):
    """tpss_create_mapped rejects bad arguments and invalid meshes before any
    device work (so this runs without a GPU): a non-convex cell, a degree
    outside the range of the dimension, non-finite vertices, a bad dim."""
    import numpy as np
    from paper_1910_11239_gb300 import tpss, workloads
    L = tpss.lib()
    EINVAL = -1   # TPSS_EINVAL in include/tpss.h

    def create(dim, degree, V):
        V = np.ascontiguousarray(V, dtype=np.float64)
        nc = (ctypes.c_int * 3)(*([s - 1 for s in reversed(V.shape[:-1])] + [1] * (3 - V.shape[-1])))
        h = ctypes.c_void_p()
        st = L.tpss_create_mapped(dim, degree, nc, ctypes.c_void_p(V.ctypes.data), 1, 4.0, 0, None,
                                  ctypes.byref(h))
        return st, L.tpss_last_error().decode()

    good2 = workloads.vertices_distorted(3, 1)
    bad2 = workloads.vertices_cartesian(np.full(2, 0.5), np.full(2, 0.5))
    bad2[1, 1] = [0.1, 0.1]                    # inside the triangle of cell (0, 0): not convex
    st, msg = create(2, 3, bad2)
    assert st == EINVAL and "convex" in msg
    flipped = good2[:, ::-1].copy()            # mirrored x: clockwise cells
    st, msg = create(2, 3, flipped)
    assert st == EINVAL and "convex" in msg
    st, msg = create(2, 16, good2)
    assert st == EINVAL and "degree" in msg
    st, msg = create(3, 8, workloads.vertices_distorted(2, 1, dim=3))
    assert st == EINVAL and "degree" in msg
    nan = good2.copy()
    nan[1, 1, 0] = np.nan
    st, msg = create(2, 3, nan)
    assert st == EINVAL and "finite" in msg
    st, msg = create(4, 3, good2)
    assert st == EINVAL and "dim" in msg
