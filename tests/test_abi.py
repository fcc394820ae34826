"""The C ABI: libedm.so builds, loads without a GPU and exports every function
include/edm.h declares (CPU only; no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "edm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(edm_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2105_12301_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("edm_create", "edm_destroy", "edm_status_string", "edm_embed",
                     "edm_knn", "edm_simplex_optimal_E", "edm_ccm_all", "edm_ccm_batched",
                     "edm_ctx_sync"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu(lib):
    lib.edm_status_string.restype = ctypes.c_char_p
    assert lib.edm_status_string(0) == b"ok"
    assert lib.edm_status_string(1) == b"invalid argument"
    assert lib.edm_status_string(4) == b"device-side wait timed out"


def test_null_arguments_are_rejected_without_gpu(lib):
    vp = ctypes.c_void_p
    lib.edm_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp]
    assert lib.edm_create(None, 0, None) == 1          # EDM_ERR_INVALID_ARG
    lib.edm_ctx_sync.argtypes = [vp]
    assert lib.edm_ctx_sync(None) == 1
    lib.edm_knn.argtypes = [vp, vp] + [ctypes.c_int] * 6 + [vp, vp]
    assert lib.edm_knn(None, None, 1, 10, 2, 1, 0, 3, None, None) == 1


def test_create_on_a_missing_device_fails_cleanly(lib):
    vp = ctypes.c_void_p
    lib.edm_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp]
    p = vp()
    assert lib.edm_create(ctypes.byref(p), 4096, None) == 2   # EDM_ERR_CUDA
    assert not p.value


def test_binding_fails_loudly_without_the_library(monkeypatch):
    from paper_2105_12301_gb300 import edm
    monkeypatch.setattr(edm, "_lib", None)
    monkeypatch.setattr(edm, "LIB_PATH", "/nonexistent/libedm.so")
    with pytest.raises(RuntimeError):
        edm.load()
