"""The C-ABI library builds, loads and exports every symbol include/*.h
declares.  CPU only: no compute call is made (gp_ctx_create without a GPU
must fail cleanly with a status code)."""

import ctypes
import glob
import os
import re

import numpy as np
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


def _size_queries():
    """The size queries validate their arguments on the host (no device work)."""
    from paper_2207_06856_gb300 import gpk
    g = gpk
    L = g.lib()
    h = g.Hyper(g.RBF, np.ones(8, np.float32), 1.0, 0.05).c()
    return g, L, h



def test_mvm_flag_validation_on_the_host():
    """Flag combinations gp_kmvm_workspace_size refuses (0) or accepts: the
    symmetric MVM is FP32 only, the FP32 value product FP16 only, unknown bits
    and XSPLIT together with NO_XSPLIT are invalid."""
    g, L, h = _size_queries()
    f = lambda flags, R=1: int(L.gp_kmvm_workspace_size(ctypes.byref(h), 4096, 4096, R, flags))
    assert f(g.FP32 | g.MVM_SYMMETRIC) > 0
    assert f(g.FP16 | g.MVM_SYMMETRIC) == 0
    assert f(g.FP16 | g.MVM_FP32_PV) > 0
    assert f(g.FP32 | g.MVM_FP32_PV) == 0
    assert f(g.BF16 | g.MVM_FP32_PV) == 0
    assert f(g.FP16 | g.MVM_FP32_PV, R=5) == 0        # one to four columns
    assert f(g.FP16 | g.MVM_FP32_PV | g.MVM_PSPLIT) == 0
    assert f(g.FP16 | g.MVM_XSPLIT | g.MVM_NO_XSPLIT) == 0
    assert f(g.FP16 | (1 << 30)) == 0


def test_cg_refine_options_on_the_host():
    """gp_cg_workspace_size: a refine MVM switched at a residual needs nothing
    else; switched at the first check (refine_resid = 0) it needs restarts;
    a negative switch residual is invalid; the refine operator adds its own
    workspace when it is neither the solve's nor the check's MVM."""
    g, L, h = _size_queries()

    def size(refine, rr, restarts=4, prec=g.FP16 | g.MVM_PSPLIT | g.MVM_XSPLIT):
        o = g._CgOpts(1e-2, 200, 0, prec, g.CG_STABLE, g.REORTH_PINV, 1, 0, restarts, g.FP32, 1, refine, rr)
        return int(L.gp_cg_workspace_size(ctypes.byref(h), 65536, 17, 100, ctypes.byref(o)))
    base = size(0, 0.0)
    assert base > 0
    assert size(g.FP16, 0.3) > base                    # a third operator
    assert size(g.FP16, 0.3, restarts=0) > 0
    assert size(g.FP16, 0.0, restarts=0) == 0          # switch at a check that never comes
    assert size(g.FP16, -1.0) == 0
    assert size(g.FP16 | (1 << 30), 0.3) == 0


def test_minres_options_on_the_host():
    g, L, h = _size_queries()

    def size(tol=1e-2, max_iter=200, restarts=4, norm=0, prec=g.FP16):
        o = g._MinresOpts(tol, max_iter, prec, restarts, g.FP32, norm)
        return int(L.gp_minres_workspace_size(ctypes.byref(h), 65536, 17, 100, ctypes.byref(o)))
    assert size() > 0
    assert size(norm=1) > 0
    assert size(norm=1, restarts=0) == 0               # the 2-norm target needs checks
    assert size(norm=2) == 0
    assert size(tol=-1.0) == 0
    assert size(max_iter=0) == 0 and size(max_iter=1001) == 0
    assert size(restarts=17) == 0
    assert size(prec=g.FP16 | g.MVM_SYMMETRIC) == 0     # the symmetric MVM is FP32 only
