"""The C-ABI library builds, loads and exports every symbol include/*.h
declares.  CPU only: no compute call is made (gp_ctx_create without a GPU
must fail cleanly with a status code)."""

import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2207_06856_gb300", "libgpk.so")


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names += re.findall(r"GPK_API\s+[\w\s\*]+?\b(gp_\w+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_2207_06856_gb300 import build
        build.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("gp_kmvm", "gp_ctx_create", "gp_ctx_destroy", "gp_strerror"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_and_no_device_status(lib):
    lib.gp_strerror.restype = ctypes.c_char_p
    assert lib.gp_strerror(0) == b"success"
    assert lib.gp_strerror(-3) == b"context workspace too small"
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p = ctypes.c_void_p()
    lib.gp_ctx_create.argtypes = [ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)]
    assert lib.gp_ctx_create(0, 0, ctypes.byref(p)) != 0
    assert not p.value


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2207_06856_gb300 import gpk
    monkeypatch.setattr(gpk, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(gpk, "_lib", None)
    with pytest.raises(RuntimeError):
        gpk.lib()
