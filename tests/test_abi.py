"""CPU-side checks of the C ABI: the library builds and loads, exports every
symbol declared in include/sparc.h, and rejects bad arguments before touching
the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2302_09708_gb300 import sparc, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sparc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(sparc_\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("sparc_create", "sparc_destroy", "sparc_hpsi", "sparc_cheb_filter",
                 "sparc_chefsi_step", "sparc_spectrum_bounds"):
        assert want in names


def test_library_exports_every_declared_symbol():
    L = sparc.load()
    for name in declared_functions():
        assert hasattr(L, name), name
    assert set(declared_functions()) <= set(sparc.EXPORTS) | {"sparc_last_error"}


def test_library_is_in_tree():
    path = sparc.library_path()
    assert os.path.commonpath([path, ROOT]) == ROOT
    assert os.path.exists(path)


def test_create_rejects_bad_grid_without_gpu():
    L = sparc.load()
    s = synth.free_system((13, 13, 13), 0.5, (0, 0, 0))
    out = ctypes.c_void_p()
    veff = np.ascontiguousarray(s.veff)
    for g in (sparc.sparc_grid(0, 13, 13, 0.5, (ctypes.c_int * 3)(0, 0, 0)),
              sparc.sparc_grid(13, 13, 13, -1.0, (ctypes.c_int * 3)(0, 0, 0)),
              sparc.sparc_grid(13, 13, 13, 0.5, (ctypes.c_int * 3)(0, 7, 0))):
        rc = L.sparc_create(ctypes.byref(g), veff.ctypes.data, None, None, ctypes.byref(out))
        assert rc == sparc.SPARC_ERR_INVALID_ARG
        assert out.value is None
        assert b"invalid argument" in L.sparc_last_error(None)
    rc = L.sparc_create(None, None, None, None, ctypes.byref(out))
    assert rc == sparc.SPARC_ERR_INVALID_ARG


def test_destroy_null_is_noop():
    assert sparc.load().sparc_destroy(None) == sparc.SPARC_OK



def test_every_declared_function_is_documented():
    """Each entry point in include/sparc.h is preceded by a comment block
    naming it (argument meaning, layout, ownership and errors live there)."""
    text = open(os.path.join(ROOT, "include", "sparc.h")).read()
    comments = " ".join(re.findall(r"/\*.*?\*/", text, flags=re.S))
    undocumented = [n for n in declared_functions() if n not in comments]
    # sparc_batch_* and sparc_destroy share comment blocks with their siblings
    assert not [n for n in undocumented
                if n not in ("sparc_batch_destroy", "sparc_batch_last_error",
                             "sparc_batch_get_info")], undocumented


def test_options_layout_and_validation_without_gpu():
    """sparc_options is six ints and an int64 (32 bytes, timeout_cycles at byte
    24); unknown flags, a nonzero reserved word, an out-of-range stencil shape
    and a negative wait bound are rejected before any device work."""
    assert ctypes.sizeof(sparc.sparc_options) == 32
    assert sparc.sparc_options.timeout_cycles.offset == 24
    assert ctypes.sizeof(sparc.sparc_tuning) == 7 * 4 + 8 * 4
    L = sparc.load()
    s = synth.free_system((13, 13, 13), 0.5, (0, 0, 0))
    g = sparc.sparc_grid(13, 13, 13, 0.5, (ctypes.c_int * 3)(0, 0, 0))
    veff = np.ascontiguousarray(s.veff)
    out = ctypes.c_void_p()
    for opt in (sparc.sparc_options(0, 4, 0, 16, 0, 0, 0),    # unknown flag bit
                sparc.sparc_options(0, 4, 0, 0, 0, 1, 0),     # reserved != 0
                sparc.sparc_options(0, 4, 0, 0, 99, 0, 0),    # no such stencil shape
                sparc.sparc_options(0, 4, 0, 0, -1, 0, 0),
                sparc.sparc_options(0, 4, 0, 0, 0, 0, -5)):   # negative wait bound
        rc = L.sparc_create(ctypes.byref(g), veff.ctypes.data, None, ctypes.byref(opt),
                            ctypes.byref(out))
        assert rc == sparc.SPARC_ERR_INVALID_ARG
        assert out.value is None
    t = sparc.sparc_tuning()
    assert L.sparc_get_tuning(None, ctypes.byref(t)) == sparc.SPARC_ERR_INVALID_ARG
