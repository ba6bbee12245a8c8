"""The C ABI library loads without a GPU and exports every symbol include/lw.h declares."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "lw.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lw_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1709_06816_gb300 import build
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        if not os.path.exists(build.LIB_PATH):
            pytest.skip("no nvcc and no prebuilt liblw.so")
        return build.LIB_PATH
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("lw_create", "lw_cluster", "lw_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(lib, name), name
    from paper_1709_06816_gb300 import native
    assert sorted(native.EXPORTS) == _declared()


def test_status_strings_without_gpu(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.lw_status_string.restype = ctypes.c_char_p
    lib.lw_status_string.argtypes = [ctypes.c_int]
    assert lib.lw_status_string(0) == b"ok"
    assert lib.lw_status_string(2).startswith(b"invalid input")
    lib.lw_destroy.argtypes = [ctypes.c_void_p]
    lib.lw_destroy(None)  # NULL is a no-op


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1709_06816_gb300 import native
    with pytest.raises(RuntimeError):
        native._lib_for_test = None
        saved = native._lib
        try:
            native._lib = None
            native.load(str(tmp_path / "missing.so"))
        finally:
            native._lib = saved
