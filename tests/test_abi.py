"""Host-side checks of the C-ABI library (no GPU needed): it builds for
sm_103a, loads, exports every entry point declared in include/*.h, and
refuses to create a context when no device exists."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:PT_API\s+)?(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(pt_[a-z0-9_]+)\s*\(", text, re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1906_10598_b300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for required in ("pt_create", "pt_destroy", "pt_load_block", "pt_objective", "pt_de_solve", "pt_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_create_without_gpu_fails_cleanly(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    h = ctypes.c_void_p()
    lib.pt_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]
    rc = lib.pt_create(ctypes.byref(h), 0)
    assert rc < 0 and not h.value
    lib.pt_last_error.restype = ctypes.c_char_p
    lib.pt_last_error.argtypes = [ctypes.c_void_p]
    assert lib.pt_last_error(None) == b"null context"


def test_python_binding_requires_the_library(monkeypatch, tmp_path):
    import paper_1906_10598_b300 as pt
    monkeypatch.setattr(pt, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pt, "_lib", None)
    with pytest.raises(ImportError):
        pt.load_library()
