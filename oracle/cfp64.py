"""Multi-threaded FP64 oracle routines (C + OpenMP) for full-size problems.

TEST INFRASTRUCTURE ONLY, like the rest of this package: the tests, the
smoke() self-check and the benchmark's CPU-baseline leg may use it, the
product path may not.  ``fp64_cg.c`` computes the same definitions as
``gp_oracle.kmvm`` / ``precond_apply`` / ``cg_standard`` (Eq. mvm,
Eq. woodbury, Alg. 1) on all host cores; it is pinned against the numpy
oracle and against closed forms in tests/test_oracle_c.py.

``build()`` compiles ``fp64_cg.c`` with gcc into ``liboracle64.so`` next to
this file (plain C, OpenMP; no x86-specific flags, so the same source builds
on the Arm GPU host).
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from .gp_oracle import Hyp, pivoted_cholesky, woodbury_core

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fp64_cg.c")
LIB = os.path.join(HERE, "liboracle64.so")
KERNEL_IDS = {"rbf": 0, "matern32": 1, "matern12": 2, "matern52": 3}

_lib = None


def build() -> str:
    """Compile liboracle64.so when it is missing or older than its source."""
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp"
    cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"gcc failed for {SRC}:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(LIB)
        P = ctypes.c_void_p
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.orc_kmvm.argtypes = [P, i64, i32, P, i32, f64, f64, P, i32, P, i64, i32, P]
        lib.orc_kmvm.restype = i32
        lib.orc_pcg.argtypes = [P, i64, i32, P, i32, f64, f64, P, i32, P, i32, P, f64, i32, f64, P, P, P, P]
        lib.orc_pcg.restype = i32
        lib.orc_quad_form_grad.argtypes = [P, i64, i32, P, i32, f64, P, P, i32, P, P]
        lib.orc_quad_form_grad.restype = i32
        lib.orc_threads.argtypes = []
        lib.orc_threads.restype = i32
        _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def threads() -> int:
    """Number of OpenMP threads the routines run on."""
    return int(_load().orc_threads())


def kmvm(X, V, hyp: Hyp, rows=None, add_noise: bool = True) -> np.ndarray:
    """Rows `rows` (all when None) of Ktilde V in FP64 (Eq. mvm); V: N x R."""
    X = _f64(X)
    V = _f64(V)
    vec = V.ndim == 1
    if vec:
        V = V[:, None]
    N, d = X.shape
    R = V.shape[1]
    ls = _f64(np.broadcast_to(hyp.lengthscale, (d,)))
    rws = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nr = N if rws is None else rws.shape[0]
    out = np.empty((nr, R))
    rc = _load().orc_kmvm(_ptr(X), N, d, _ptr(ls), KERNEL_IDS[hyp.kernel], float(hyp.outputscale),
                          float(hyp.noise), _ptr(V), R, None if rws is None else _ptr(rws), nr,
                          1 if add_noise else 0, _ptr(out))
    if rc != 0:
        raise RuntimeError(f"orc_kmvm failed ({rc})")
    return out[:, 0] if vec else out


def relative_residual(X, U, B, hyp: Hyp) -> np.ndarray:
    """Per-column ||Ktilde U - B|| / ||B|| over ALL rows, in FP64."""
    U = _f64(U)
    B = _f64(B)
    if U.ndim == 1:
        U, B = U[:, None], B[:, None]
    res = kmvm(X, U, hyp, add_noise=True) - B
    return np.linalg.norm(res, axis=0) / np.linalg.norm(B, axis=0)


def pcg(X, B, hyp: Hyp, L=None, tol: float = 1e-2, max_iter: int = 1000, time_limit_s: float = 0.0):
    """Preconditioned CG (Alg. 1) on every column of B (N x R), x_0 = 0, with
    P = L L^T + sigma^2 I (Eq. woodbury) or P = I when L is None.

    Returns (U, iterations, per-column relative residual, seconds per iteration).
    """
    X = _f64(X)
    B = _f64(B)
    if B.ndim == 1:
        B = B[:, None]
    N, d = X.shape
    R = B.shape[1]
    ls = _f64(np.broadcast_to(hyp.lengthscale, (d,)))
    if L is None or np.asarray(L).shape[1] == 0:
        Lc, Cc, k = np.zeros((N, 1)), np.ones((1, 1)), 0
    else:
        Lc = _f64(L)
        k = Lc.shape[1]
        Cc = _f64(woodbury_core(Lc, hyp.noise))
    U = np.empty((N, R))
    it = ctypes.c_int(0)
    rel = np.empty(R)
    spi = ctypes.c_double(0.0)
    rc = _load().orc_pcg(_ptr(X), N, d, _ptr(ls), KERNEL_IDS[hyp.kernel], float(hyp.outputscale), float(hyp.noise),
                         _ptr(B), R, _ptr(Lc), k, _ptr(Cc), float(tol), int(max_iter), float(time_limit_s),
                         _ptr(U), ctypes.byref(it), _ptr(rel), ctypes.byref(spi))
    if rc != 0:
        raise RuntimeError(f"orc_pcg failed ({rc})")
    return U, int(it.value), rel, float(spi.value)


def quad_form_grad(X, hyp: Hyp, U, V, wrt_X: bool = False):
    """Gradient of q = sum_c u_c^T Ktilde v_c (u, v fixed) w.r.t. (l_1..l_d, a^2,
    sigma^2) and optionally X: the same quantity as gp_oracle.quad_form_grad,
    matrix-free on all host cores.  U, V: N x R.  Returns (g [d+2], gX or None)."""
    X = _f64(X)
    N, d = X.shape
    U = _f64(np.asarray(U, dtype=np.float64).reshape(N, -1))
    V = _f64(np.asarray(V, dtype=np.float64).reshape(N, -1))
    ls = _f64(np.broadcast_to(hyp.lengthscale, (d,)))
    g = np.empty(d + 2)
    gX = np.empty((N, d)) if wrt_X else None
    rc = _load().orc_quad_form_grad(_ptr(X), N, d, _ptr(ls), KERNEL_IDS[hyp.kernel], float(hyp.outputscale),
                                    _ptr(U), _ptr(V), U.shape[1], _ptr(g), None if gX is None else _ptr(gX))
    if rc != 0:
        raise RuntimeError(f"orc_quad_form_grad failed ({rc})")
    return g, gX


def pseudo_loss_grad(X, hyp: Hyp, U, Z, W=None) -> np.ndarray:
    """Eq. approx as in gp_oracle.pseudo_loss_grad, with the bilinear-form
    gradients taken matrix-free (large N)."""
    U = np.asarray(U, dtype=np.float64)
    Z = np.asarray(Z, dtype=np.float64)
    M = Z.shape[1]
    Wp = Z if W is None else np.asarray(W, dtype=np.float64)
    g_probe, _ = quad_form_grad(X, hyp, U[:, 1:], Wp)
    g_y, _ = quad_form_grad(X, hyp, U[:, :1], U[:, :1])
    return g_probe / (2.0 * M) - 0.5 * g_y


def preconditioner(X, hyp: Hyp, rank: int):
    """The FP64 pivoted-Cholesky factor L (N x rank) of the oracle (Sec. 4.2)."""
    L, _ = pivoted_cholesky(X, hyp, rank)
    return L
