"""The C-ABI library loads and exports every function include/nuri.h declares (CPU only)."""
import ctypes
import os
import re

import paper_1807_08888_b300 as nuri
from paper_1807_08888_b300 import build as nuri_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "nuri.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nuri_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_binding_exports():
    assert declared_functions() == sorted(nuri.EXPORTS)


def test_library_exports_every_declared_symbol():
    nuri_build.build()
    lib = ctypes.CDLL(nuri.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_version_and_error_string_without_gpu():
    assert "sm_103a" in nuri.version()
    assert isinstance(nuri.lib().nuri_last_error(), bytes)


def test_invalid_arguments_are_rejected_without_touching_the_gpu():
    L = nuri.lib()
    h = ctypes.c_void_p()
    # negative n, NULL out and bad hop counts fail before any CUDA call
    assert L.nuri_load_graph(-1, 0, None, None, None, None, 0, 0, None, ctypes.byref(h)) == nuri.ERR_INVALID
    assert L.nuri_load_graph(3, 0, None, None, None, None, 9, 0, None, ctypes.byref(h)) == nuri.ERR_INVALID
    assert b"index_hops" in L.nuri_last_error()
    assert L.nuri_topk_cliques(None, 1, 0, 0, 0, None, None) == nuri.ERR_INVALID
