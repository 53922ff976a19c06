"""Host-side checks of the C ABI (no GPU): the library builds, loads and exports
every function include/*.h declares; calls without a context are rejected."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", text, flags=re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "return", "sizeof", "defined"):
                names.add(name)
    return sorted(names)


def test_header_declares_entry_points():
    names = _declared_functions()
    for must in ("stencil_create", "stencil_jacobi", "stencil_gs_lex", "residual_norm", "stencil_solve_mixed"):
        assert must in names


def test_library_exports_every_declared_function():
    from paper_1004_1741_gb300 import build

    lib = ctypes.CDLL(build.build())
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_declared_functions():
    from paper_1004_1741_gb300 import capi

    assert set(_declared_functions()) <= set(capi.exported_names())


def test_null_context_and_create_errors():
    from paper_1004_1741_gb300 import build

    lib = ctypes.CDLL(build.build())
    lib.stencil_jacobi.restype = ctypes.c_int
    lib.stencil_jacobi.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_double, ctypes.c_int, ctypes.c_void_p]
    assert lib.stencil_jacobi(None, None, None, None, 1.0, 1, None) == -1
    lib.stencil_create.restype = ctypes.c_int
    lib.stencil_create.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t]
    assert lib.stencil_create(None, 0, 0) == -1
    lib.stencil_last_error.restype = ctypes.c_char_p
    lib.stencil_last_error.argtypes = [ctypes.c_void_p]
    assert b"NULL" in lib.stencil_last_error(None)
    lib.stencil_destroy.argtypes = [ctypes.c_void_p]
    lib.stencil_destroy(None)  # ignored


def test_create_without_gpu_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1004_1741_gb300 import capi

    with pytest.raises(capi.StencilError) as e:
        capi.Context(0)
    assert e.value.code in (capi.STENCIL_ERR_CUDA, capi.STENCIL_ERR_ARG)
