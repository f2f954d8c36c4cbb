"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, and exports every entry point include/fcs.h declares; the
Python binding names the same set."""
from __future__ import annotations

import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fcs.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fcs_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    import paper_2106_13062_gb300 as fcs
    return fcs.build()


def test_header_declares_the_hot_path():
    names = declared_functions()
    for required in ("fcs_make_hashes", "fcs_sketch_cp", "fcs_sketch_dense",
                     "fcs_contract", "fcs_recover", "fcs_sketch_outer",
                     "fcs_create", "fcs_destroy", "fcs_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"libfcs.so lacks {missing}"


def test_binding_names_match_header(libpath):
    import paper_2106_13062_gb300 as fcs
    assert sorted(fcs.exported_symbols()) == declared_functions()
    for n in declared_functions():
        if n.startswith("fcs_") and n not in ("fcs_create", "fcs_destroy",
                                              "fcs_set_stream", "fcs_last_error",
                                              "fcs_workspace_bytes",
                                              "fcs_version"):
            assert hasattr(fcs, n), f"binding lacks {n}"


def test_version_and_null_context(libpath):
    lib = ctypes.CDLL(libpath)
    lib.fcs_version.restype = ctypes.c_int
    assert lib.fcs_version() >= 10000
    lib.fcs_last_error.restype = ctypes.c_char_p
    lib.fcs_last_error.argtypes = [ctypes.c_void_p]
    assert lib.fcs_last_error(None) == b"null context"
    lib.fcs_destroy.argtypes = [ctypes.c_void_p]
    assert lib.fcs_destroy(None) == 0
    # every compute entry point rejects a NULL context before touching CUDA
    lib.fcs_make_hashes.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                    ctypes.c_void_p, ctypes.c_void_p]
    assert lib.fcs_make_hashes(None, 0, 3, None, None, 1, None, None) == 1


def test_binding_refuses_without_gpu(libpath):
    import torch
    import paper_2106_13062_gb300 as fcs
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        fcs.Context()
