"""Thin Python binding over libgpk's C ABI (include/gpk.h).

Argument marshalling only: tensors are passed as raw device pointers with the
current torch CUDA stream; every step of the computation runs in the CUDA
library.  There is no CPU fallback: if libgpk.so is missing, or a tensor is
not a contiguous float32 CUDA tensor, the call raises.

Layouts follow the C ABI: inputs X are (N, d) row-major; blocks of vectors are
N x R column-major, i.e. torch tensors of shape (R, N) (row c = vector c).
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgpk.so")

# status codes
GP_OK = 0
GP_ERR_INVALID = -1
GP_ERR_CUDA = -2
GP_ERR_WORKSPACE = -3
GP_ERR_BREAKDOWN = -4
GP_ERR_NONFINITE = -5
GP_ERR_NOT_CONVERGED = -6
GP_ERR_TIMEOUT = -7
GP_ERR_OOM = -8
GP_ERR_UNSUPPORTED = -9

# kernels and precisions
RBF, MATERN32, MATERN12, MATERN52 = 0, 1, 2, 3
KERNELS = {"rbf": RBF, "matern32": MATERN32, "matern12": MATERN12, "matern52": MATERN52}
FP32, FP16, BF16 = 0, 1, 2
PRECISIONS = {"fp32": FP32, "fp16": FP16, "bf16": BF16}

MVM_ADD_NOISE = 0x100
MVM_XSPLIT = 0x200
MVM_NO_XSPLIT = 0x400
MVM_SCALE_SQRT_N = 0x800
MVM_VSPLIT = 0x1000
MVM_BF16_SINGLE = 0x2000
MVM_ONE_TILE = 0x4000
MVM_PSPLIT = 0x8000
MVM_HALF_EXP = 0x10000
MVM_SKIP_TILES = 0x20000
MVM_SYMMETRIC = 0x200000
MVM_FP32_PV = 0x400000


def MVM_SUM(scheme: int) -> int:
    """Summation-variant study flag: 1 FP32, 2 FP16, 3 FP16 block sums, 4 Kahan FP16."""
    return (int(scheme) & 0x7) << 18


def _check_flags(check_precision, prec: int) -> int:
    return PRECISIONS[check_precision] if isinstance(check_precision, str) else int(check_precision)


class GPKError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {strerror(status)} ({status})" if what else f"{strerror(status)} ({status})")


CG_STABLE, CG_STANDARD = 0, 1
REORTH_NONE, REORTH_PINV, REORTH_EUCLID = 0, 1, 2
REORTH = {"none": REORTH_NONE, "pinv": REORTH_PINV, "euclid": REORTH_EUCLID}


class _Precond(ctypes.Structure):
    _fields_ = [("L", ctypes.c_void_p), ("core", ctypes.c_void_p), ("rank", ctypes.c_int)]


class _CgOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("min_iter", ctypes.c_int),
                ("precision", ctypes.c_int), ("algorithm", ctypes.c_int), ("reorth", ctypes.c_int),
                ("reorth_passes", ctypes.c_int), ("x0_given", ctypes.c_int), ("restarts", ctypes.c_int),
                ("check_precision", ctypes.c_int), ("escalate", ctypes.c_int), ("refine_precision", ctypes.c_int),
                ("refine_resid", ctypes.c_double)]


class _CgStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("breakdowns", ctypes.c_int),
                ("restarts", ctypes.c_int), ("escalated", ctypes.c_int),
                ("col_iters", ctypes.POINTER(ctypes.c_int)), ("rel_resid", ctypes.POINTER(ctypes.c_double)),
                ("alpha", ctypes.POINTER(ctypes.c_double)), ("beta", ctypes.POINTER(ctypes.c_double)),
                ("gamma0", ctypes.POINTER(ctypes.c_double)), ("resid_hist", ctypes.POINTER(ctypes.c_double)),
                ("lanczos_len", ctypes.POINTER(ctypes.c_int))]


class _MinresOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("precision", ctypes.c_int),
                ("restarts", ctypes.c_int), ("check_precision", ctypes.c_int), ("norm", ctypes.c_int),
                ("refine_precision", ctypes.c_int), ("refine_resid", ctypes.c_double)]


class _MinresStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("breakdowns", ctypes.c_int),
                ("restarts", ctypes.c_int), ("col_iters", ctypes.POINTER(ctypes.c_int)),
                ("rel_resid", ctypes.POINTER(ctypes.c_double)), ("rel_resid_p", ctypes.POINTER(ctypes.c_double)),
                ("resid_hist", ctypes.POINTER(ctypes.c_double))]


class _Hyp(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("d", ctypes.c_int),
                ("lengthscale", ctypes.POINTER(ctypes.c_float)),
                ("outputscale", ctypes.c_double), ("noise", ctypes.c_double)]


class _ServerOpts(ctypes.Structure):
    _fields_ = [("arena_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int), ("rank", ctypes.c_int),
                ("precision", ctypes.c_int), ("mean_precision", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("restarts", ctypes.c_int), ("reorth", ctypes.c_int),
                ("refine_precision", ctypes.c_int), ("refine_resid", ctypes.c_double),
                ("large_n", ctypes.c_int64), ("large_reserve", ctypes.c_int)]


class _ReqStats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("restarts", ctypes.c_int),
                ("rel_resid", ctypes.c_double), ("t_submit_ms", ctypes.c_double), ("t_admit_ms", ctypes.c_double),
                ("t_done_ms", ctypes.c_double), ("bytes", ctypes.c_size_t)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("arena_bytes", ctypes.c_size_t),
                ("peak_bytes", ctypes.c_size_t), ("in_use_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_int),
                ("launches", ctypes.c_int64)]


_lib = None
_c_void_p = ctypes.c_void_p
_c_i64 = ctypes.c_int64
_c_int = ctypes.c_int
_c_size = ctypes.c_size_t


def _declare(lib):
    sig = {
        "gp_strerror": (ctypes.c_char_p, [_c_int]),
        "gp_ctx_create": (_c_int, [_c_int, _c_size, ctypes.POINTER(_c_void_p)]),
        "gp_ctx_destroy": (None, [_c_void_p]),
        "gp_ctx_reserve": (_c_int, [_c_void_p, _c_size]),
        "gp_ctx_workspace_bytes": (_c_size, [_c_void_p]),
        "gp_ctx_check": (_c_int, [_c_void_p, _c_void_p]),
        "gp_ctx_launch_count": (_c_i64, [_c_void_p]),
        "gp_wait_check": (_c_int, [_c_void_p, ctypes.c_double, _c_int, ctypes.POINTER(ctypes.c_longlong), _c_void_p]),
        "gp_kmvm_workspace_size": (_c_size, [ctypes.POINTER(_Hyp), _c_i64, _c_i64, _c_int, _c_int]),
        "gp_kmvm": (_c_int, [_c_void_p, ctypes.POINTER(_Hyp), _c_void_p, _c_i64, _c_void_p, _c_i64,
                             _c_void_p, _c_int, _c_void_p, _c_int, _c_void_p]),
        "gp_ctx_profile": (_c_int, [_c_void_p, _c_int]),
        "gp_ctx_profile_read": (_c_int, [_c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_c_i64)]),
        "gp_measure_peaks": (_c_int, [_c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double), _c_void_p]),
        "gp_measure_peaks2": (_c_int, [_c_void_p] + [ctypes.POINTER(ctypes.c_double)] * 5 + [_c_void_p]),
        "gp_kmvm_vjp_workspace_size": (_c_size, [ctypes.POINTER(_Hyp), _c_i64, _c_int]),
        "gp_kmvm_vjp": (_c_int, [_c_void_p, ctypes.POINTER(_Hyp), _c_void_p, _c_i64, _c_void_p, _c_void_p, _c_int,
                                 ctypes.POINTER(ctypes.c_double), _c_void_p, _c_void_p]),
        "gp_slq_quadrature": (_c_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _c_int,
                                       ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
        "gp_mll_workspace_size": (_c_size, [ctypes.POINTER(_Hyp), _c_i64, _c_int, _c_int, ctypes.POINTER(_CgOpts)]),
        "gp_mll_and_grad": (_c_int, [_c_void_p, ctypes.POINTER(_Hyp), _c_void_p, _c_void_p, _c_i64, _c_void_p, _c_int,
                                     _c_void_p, ctypes.POINTER(_Precond), ctypes.POINTER(_CgOpts), _c_int,
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _c_void_p,
                                     _c_void_p, ctypes.POINTER(_CgStats), _c_void_p]),
        "gp_pivchol_workspace_size": (_c_size, [ctypes.POINTER(_Hyp), _c_i64, _c_int]),
        "gp_pivchol_precond": (_c_int, [_c_void_p, ctypes.POINTER(_Hyp), _c_void_p, _c_i64, _c_int, _c_void_p,
                                        _c_void_p, _c_void_p, ctypes.POINTER(_c_int), _c_void_p]),
        "gp_cg_workspace_size": (_c_size, [ctypes.POINTER(_Hyp), _c_i64, _c_int, _c_int, ctypes.POINTER(_CgOpts)]),
        "gp_minres_workspace_size": (_c_size, [ctypes.POINTER(_Hyp), _c_i64, _c_int, _c_int,
                                               ctypes.POINTER(_MinresOpts)]),
        "gp_minres_solve": (_c_int, [_c_void_p, ctypes.POINTER(_Hyp), _c_void_p, _c_i64, _c_void_p, _c_int, _c_void_p,
                                     ctypes.POINTER(_Precond), ctypes.POINTER(_MinresOpts),
                                     ctypes.POINTER(_MinresStats), _c_void_p]),
        "gp_cg_solve": (_c_int, [_c_void_p, ctypes.POINTER(_Hyp), _c_void_p, _c_i64, _c_void_p, _c_int, _c_void_p,
                                 ctypes.POINTER(_Precond), ctypes.POINTER(_CgOpts), ctypes.POINTER(_CgStats),
                                 _c_void_p]),
        "gp_server_request_bytes": (_c_size, [ctypes.POINTER(_ServerOpts), ctypes.POINTER(_Hyp), _c_i64, _c_i64]),
        "gp_server_create": (_c_int, [_c_int, ctypes.POINTER(_ServerOpts), ctypes.POINTER(_c_void_p)]),
        "gp_server_submit": (_c_int, [_c_void_p, ctypes.POINTER(_Hyp), _c_void_p, _c_i64, _c_void_p, _c_void_p,
                                      _c_i64, _c_void_p, ctypes.POINTER(ctypes.c_uint64)]),
        "gp_server_wait": (_c_int, [_c_void_p, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(_ReqStats)]),
        "gp_server_stats": (_c_int, [_c_void_p, ctypes.POINTER(_ServerStats)]),
        "gp_server_destroy": (None, [_c_void_p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def lib():
    """Load libgpk.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2207_06856_gb300.build.build()")
        _lib = _declare(ctypes.CDLL(LIB_PATH))
    return _lib


def strerror(status: int) -> str:
    return lib().gp_strerror(int(status)).decode()


def _check(status: int, what: str):
    if status != GP_OK:
        raise GPKError(status, what)


@dataclass
class Hyper:
    """theta = (lengthscale[d], outputscale a^2, noise sigma^2) and the kernel."""
    kernel: int
    lengthscale: np.ndarray
    outputscale: float = 1.0
    noise: float = 0.0

    def __post_init__(self):
        if isinstance(self.kernel, str):
            self.kernel = KERNELS[self.kernel]
        self.lengthscale = np.ascontiguousarray(np.atleast_1d(self.lengthscale), dtype=np.float32)

    @property
    def d(self) -> int:
        return int(self.lengthscale.shape[0])

    def c(self) -> _Hyp:
        h = _Hyp(int(self.kernel), self.d,
                 self.lengthscale.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                 float(self.outputscale), float(self.noise))
        h._keep = self.lengthscale  # keep the array alive with the struct
        return h


def _stream_ptr(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dev_ptr(t, what: str, shape=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if t.dtype != torch.float32:
        raise TypeError(f"{what} must be float32")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{what} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return int(t.data_ptr())


class Context:
    """A libgpk context on one CUDA device (owns the device workspace)."""

    def __init__(self, device: int = 0, workspace_bytes: int = 0):
        self._p = _c_void_p()
        _check(lib().gp_ctx_create(int(device), int(workspace_bytes), ctypes.byref(self._p)), "gp_ctx_create")
        self.device = device

    def close(self):
        if self._p:
            lib().gp_ctx_destroy(self._p)
            self._p = _c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def ptr(self):
        return self._p

    def reserve(self, nbytes: int):
        _check(lib().gp_ctx_reserve(self._p, int(nbytes)), "gp_ctx_reserve")

    @property
    def workspace_bytes(self) -> int:
        return int(lib().gp_ctx_workspace_bytes(self._p))

    @property
    def launches(self) -> int:
        return int(lib().gp_ctx_launch_count(self._p))

    def check(self, stream=None):
        _check(lib().gp_ctx_check(self._p, _c_void_p(_stream_ptr(stream))), "device error")

    def wait_check(self, limit_ms: float, sleep: bool = False, stream=None) -> int:
        """gp_wait_check: run a bounded device wait that nothing completes; the
        timeout shows at the next check().  Returns the SM cycles it waited."""
        cyc = ctypes.c_longlong(0)
        _check(lib().gp_wait_check(self._p, float(limit_ms), 1 if sleep else 0, ctypes.byref(cyc),
                                   _c_void_p(_stream_ptr(stream))), "gp_wait_check")
        return int(cyc.value)

    def profile(self, enable: bool = True):
        """Record CUDA events around every tensor-core MVM launch."""
        _check(lib().gp_ctx_profile(self._p, 1 if enable else 0), "gp_ctx_profile")

    def profile_read(self):
        """(summed milliseconds, launch count) of the profiled MVM launches; resets."""
        ms = ctypes.c_double(0.0)
        n = _c_i64(0)
        _check(lib().gp_ctx_profile_read(self._p, ctypes.byref(ms), ctypes.byref(n)), "gp_ctx_profile_read")
        return float(ms.value), int(n.value)

    def measure_peaks(self, stream=None) -> dict:
        """Measured throughput (ops/s) of ex2, sqrt (special function units) and FP32 FMA."""
        e, q, f, k, m = (ctypes.c_double() for _ in range(5))
        _check(lib().gp_measure_peaks2(self._p, ctypes.byref(e), ctypes.byref(q), ctypes.byref(f), ctypes.byref(k),
                                       ctypes.byref(m), _stream_ptr(stream)), "gp_measure_peaks2")
        return {"ex2_per_s": e.value, "sqrt_per_s": q.value, "ffma_per_s": f.value,
                "pack_f16x2_per_s": k.value, "fp16_epilogue_values_per_s": m.value}


def kmvm_workspace_size(hyp: Hyper, Nr: int, Nc: int, R: int, flags: int) -> int:
    h = hyp.c()
    return int(lib().gp_kmvm_workspace_size(ctypes.byref(h), int(Nr), int(Nc), int(R), int(flags)))


def kmvm(ctx: Context, hyp: Hyper, Xr, V, Xc=None, precision="fp16", add_noise=False, flags=0,
         out=None, stream=None):
    """out = a^2 K(Xr, Xc) V (+ sigma^2 V): gp_kmvm.  Xr (Nr, d), Xc (Nc, d),
    V (R, Nc) -> out (R, Nr), all float32 CUDA tensors."""
    import torch
    Xc = Xr if Xc is None else Xc
    Nr, d = Xr.shape
    Nc = Xc.shape[0]
    R = V.shape[0]
    if d != hyp.d or Xc.shape[1] != d:
        raise ValueError("input dimension does not match the lengthscales")
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    fl = prec | int(flags) | (MVM_ADD_NOISE if add_noise else 0)
    if out is None:
        out = torch.empty((R, Nr), dtype=torch.float32, device=V.device)
    need = kmvm_workspace_size(hyp, Nr, Nc, R, fl & ~MVM_ADD_NOISE)
    if need > ctx.workspace_bytes:
        ctx.reserve(need)
    h = hyp.c()
    st = lib().gp_kmvm(ctx.ptr, ctypes.byref(h), _dev_ptr(Xr, "Xr", (Nr, d)), Nr, _dev_ptr(Xc, "Xc", (Nc, d)), Nc,
                       _dev_ptr(V, "V", (R, Nc)), R, _dev_ptr(out, "out", (R, Nr)), fl, _stream_ptr(stream))
    _check(st, "gp_kmvm")
    return out


@dataclass
class Precond:
    """Pivoted-Cholesky preconditioner P = L L^T + sigma^2 I (Eq. woodbury).
    L: (rank, N) float32 CUDA tensor (N x rank column-major); core: the lower
    Cholesky factor of I + sigma^-2 L^T L as a (rank, rank) float64 CUDA
    tensor holding it column-major (core.T is the factor); piv: int32 pivots."""
    L: object
    core: object
    piv: object
    rank: int

    def c(self) -> _Precond:
        return _Precond(int(self.L.data_ptr()), int(self.core.data_ptr()), int(self.rank))


def pivchol_precond(ctx: Context, hyp: Hyper, X, rank: int, stream=None) -> Precond:
    """gp_pivchol_precond: rank-k pivoted Cholesky of K(X, X) and its FP64 Woodbury core."""
    import torch
    N, d = X.shape
    h = hyp.c()
    need = int(lib().gp_pivchol_workspace_size(ctypes.byref(h), N, int(rank)))
    if need == 0:
        raise GPKError(GP_ERR_INVALID, "gp_pivchol_workspace_size")
    if need > ctx.workspace_bytes:
        ctx.reserve(need)
    L = torch.empty((rank, N), dtype=torch.float32, device=X.device)
    piv = torch.empty((rank,), dtype=torch.int32, device=X.device)
    core = torch.zeros((rank * rank,), dtype=torch.float64, device=X.device)
    rk = _c_int(0)
    st = lib().gp_pivchol_precond(ctx.ptr, ctypes.byref(h), _dev_ptr(X, "X", (N, d)), N, int(rank), int(L.data_ptr()),
                                  int(piv.data_ptr()), int(core.data_ptr()), ctypes.byref(rk), _stream_ptr(stream))
    _check(st, "gp_pivchol_precond")
    k = int(rk.value)
    return Precond(L[:k], core[:k * k].view(k, k), piv[:k], k)


def cg_solve(ctx: Context, hyp: Hyper, X, B, precond: Precond | None = None, tol: float = 1e-2,
             max_iter: int = 50, min_iter: int = 0, precision="fp16", algorithm: str = "stable",
             reorth: str = "pinv", reorth_passes: int = 1, U=None, flags: int = 0, restarts: int = 4,
             check_precision="fp32", escalate: bool = True, refine_precision=None, refine_resid: float = 0.0,
             stream=None):
    """gp_cg_solve: (K + sigma^2 I) U = B.  B (R, N) -> (U (R, N), status, info).
    info holds the per-column iterations, relative residuals, alpha/beta
    histories (numpy arrays) and gamma_0.  status is GP_OK,
    GP_ERR_NOT_CONVERGED or GP_ERR_BREAKDOWN (other errors raise).
    refine_precision: MVM flags (or a precision name) the solve switches to,
    once every active column's recursive relative residual is <= refine_resid
    (> 0), or at the first true-residual check (refine_resid = 0); None keeps
    the solve's MVM throughout."""
    import torch
    N, d = X.shape
    R = B.shape[0]
    prec = (PRECISIONS[precision] if isinstance(precision, str) else int(precision)) | int(flags)
    opts = _CgOpts(float(tol), int(max_iter), int(min_iter), prec,
                   CG_STABLE if algorithm == "stable" else CG_STANDARD,
                   REORTH[reorth] if isinstance(reorth, str) else int(reorth), int(reorth_passes),
                   1 if U is not None else 0, int(restarts), _check_flags(check_precision, prec),
                   1 if escalate else 0, 0 if refine_precision is None else _check_flags(refine_precision, prec),
                   float(refine_resid))
    h = hyp.c()
    rank = precond.rank if precond is not None else 0
    need = int(lib().gp_cg_workspace_size(ctypes.byref(h), N, R, rank, ctypes.byref(opts)))
    if need == 0:
        raise GPKError(GP_ERR_INVALID, "gp_cg_workspace_size")
    if need > ctx.workspace_bytes:
        ctx.reserve(need)
    if U is None:
        U = torch.empty((R, N), dtype=torch.float32, device=B.device)
    col_iters = np.zeros(R, np.int32)
    rel = np.zeros(R, np.float64)
    al = np.zeros(max_iter * R, np.float64)
    be = np.zeros(max_iter * R, np.float64)
    g0 = np.zeros(R, np.float64)
    rh = np.zeros((max_iter + 1) * R, np.float64)
    P = ctypes.POINTER
    lz = np.zeros(R, np.int32)
    stats = _CgStats(0, 0, 0, 0, 0, col_iters.ctypes.data_as(P(ctypes.c_int)), rel.ctypes.data_as(P(ctypes.c_double)),
                     al.ctypes.data_as(P(ctypes.c_double)), be.ctypes.data_as(P(ctypes.c_double)),
                     g0.ctypes.data_as(P(ctypes.c_double)), rh.ctypes.data_as(P(ctypes.c_double)),
                     lz.ctypes.data_as(P(ctypes.c_int)))
    pc = precond.c() if precond is not None else _Precond(None, None, 0)
    st = lib().gp_cg_solve(ctx.ptr, ctypes.byref(h), _dev_ptr(X, "X", (N, d)), N, _dev_ptr(B, "B", (R, N)), R,
                           _dev_ptr(U, "U", (R, N)), ctypes.byref(pc), ctypes.byref(opts), ctypes.byref(stats),
                           _stream_ptr(stream))
    if st not in (GP_OK, GP_ERR_NOT_CONVERGED, GP_ERR_BREAKDOWN):
        _check(st, "gp_cg_solve")
    it = int(stats.iters)
    info = {"iters": it, "converged": int(stats.converged), "breakdowns": int(stats.breakdowns),
            "restarts": int(stats.restarts), "escalated": int(stats.escalated),
            "col_iters": col_iters, "rel_resid": rel, "gamma0": g0,
            "alpha": al.reshape(max_iter, R)[:it], "beta": be.reshape(max_iter, R)[:it],
            "resid_hist": rh.reshape(max_iter + 1, R)[:it + 1], "lanczos_len": lz}
    return U, st, info


def minres_solve(ctx: Context, hyp: Hyper, X, B, precond: Precond | None = None, tol: float = 1e-2,
                 max_iter: int = 200, precision="fp16", flags: int = 0, restarts: int = 4, check_precision="fp32",
                 norm: str = "p", refine_precision=None, refine_resid: float = 0.0, stream=None):
    """gp_minres_solve: (K + sigma^2 I) U = B by preconditioned MINRES.
    B (R, N) -> (U (R, N), status, info).  tol applies to the residual in the
    P^-1 norm (norm="p") or, at the true-residual checks, in the 2-norm
    (norm="2"); refine_precision / refine_resid: the relaxed MVM schedule of
    cg_solve; info holds per-column iterations, the final 2-norm and P^-1-norm
    relative residuals (recomputed with the check MVM) and the recurrence's
    P^-1-norm residual history.  status is GP_OK, GP_ERR_NOT_CONVERGED or
    GP_ERR_BREAKDOWN (other errors raise)."""
    import torch
    N, d = X.shape
    R = B.shape[0]
    prec = (PRECISIONS[precision] if isinstance(precision, str) else int(precision)) | int(flags)
    opts = _MinresOpts(float(tol), int(max_iter), prec, int(restarts), _check_flags(check_precision, prec),
                       {"p": 0, "2": 1}[norm],
                       0 if refine_precision is None else _check_flags(refine_precision, prec), float(refine_resid))
    h = hyp.c()
    rank = precond.rank if precond is not None else 0
    need = int(lib().gp_minres_workspace_size(ctypes.byref(h), N, R, rank, ctypes.byref(opts)))
    if need == 0:
        raise GPKError(GP_ERR_INVALID, "gp_minres_workspace_size")
    if need > ctx.workspace_bytes:
        ctx.reserve(need)
    U = torch.empty((R, N), dtype=torch.float32, device=B.device)
    col_iters = np.zeros(R, np.int32)
    rel = np.zeros(R, np.float64)
    relp = np.zeros(R, np.float64)
    rh = np.zeros((max_iter + 1) * R, np.float64)
    P = ctypes.POINTER
    stats = _MinresStats(0, 0, 0, 0, col_iters.ctypes.data_as(P(ctypes.c_int)), rel.ctypes.data_as(P(ctypes.c_double)),
                         relp.ctypes.data_as(P(ctypes.c_double)), rh.ctypes.data_as(P(ctypes.c_double)))
    pc = precond.c() if precond is not None else _Precond(None, None, 0)
    st = lib().gp_minres_solve(ctx.ptr, ctypes.byref(h), _dev_ptr(X, "X", (N, d)), N, _dev_ptr(B, "B", (R, N)), R,
                               _dev_ptr(U, "U", (R, N)), ctypes.byref(pc), ctypes.byref(opts), ctypes.byref(stats),
                               _stream_ptr(stream))
    if st not in (GP_OK, GP_ERR_NOT_CONVERGED, GP_ERR_BREAKDOWN):
        _check(st, "gp_minres_solve")
    it = int(stats.iters)
    info = {"iters": it, "converged": int(stats.converged), "breakdowns": int(stats.breakdowns),
            "restarts": int(stats.restarts), "col_iters": col_iters, "rel_resid": rel, "rel_resid_p": relp,
            "resid_hist": rh.reshape(max_iter + 1, R)[:it + 1]}
    return U, st, info


def kmvm_tile_count(ctx: Context, hyp: Hyper, Xr, Xc=None, precision="fp16", flags=0, stream=None):
    """gp_kmvm_tile_count: (evaluated, total) (row-tile pair, column tile) entries
    of the MVM gp_kmvm runs with these flags (GP_MVM_SKIP_TILES skips the
    entries whose kernel values all round to zero)."""
    Xc = Xr if Xc is None else Xc
    Nr, d = Xr.shape
    Nc = Xc.shape[0]
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    fl = prec | int(flags)
    need = kmvm_workspace_size(hyp, Nr, Nc, 1, fl)
    if need > ctx.workspace_bytes:
        ctx.reserve(need)
    fn = lib().gp_kmvm_tile_count
    fn.restype = _c_int
    fn.argtypes = [_c_void_p, ctypes.POINTER(_Hyp), _c_void_p, _c_i64, _c_void_p, _c_i64, _c_int,
                   ctypes.POINTER(_c_i64), ctypes.POINTER(_c_i64), _c_void_p]
    ev, tot = _c_i64(0), _c_i64(0)
    h = hyp.c()
    st = fn(ctx.ptr, ctypes.byref(h), _dev_ptr(Xr, "Xr", (Nr, d)), Nr, _dev_ptr(Xc, "Xc", (Nc, d)), Nc, fl,
            ctypes.byref(ev), ctypes.byref(tot), _stream_ptr(stream))
    _check(st, "gp_kmvm_tile_count")
    return int(ev.value), int(tot.value)


def kmvm_noalloc(hyp: Hyper, Xr, V, Xc=None, precision="fp16", add_noise=False, flags=0, out=None, stream=None):
    """gp_kmvm_noalloc: the same product as kmvm, with no context and no device
    allocation inside the library (fixed scratch of GPK_NOALLOC_SCRATCH_BYTES)."""
    import torch
    fn = lib().gp_kmvm_noalloc
    fn.restype = _c_int
    fn.argtypes = [ctypes.POINTER(_Hyp), _c_void_p, _c_i64, _c_void_p, _c_i64, _c_void_p, _c_int, _c_void_p,
                   _c_int, _c_void_p]
    Xc = Xr if Xc is None else Xc
    Nr, d = Xr.shape
    Nc = Xc.shape[0]
    R = V.shape[0]
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    fl = prec | int(flags) | (MVM_ADD_NOISE if add_noise else 0)
    if out is None:
        out = torch.empty((R, Nr), dtype=torch.float32, device=V.device)
    h = hyp.c()
    st = fn(ctypes.byref(h), _dev_ptr(Xr, "Xr", (Nr, d)), Nr, _dev_ptr(Xc, "Xc", (Nc, d)), Nc,
            _dev_ptr(V, "V", (R, Nc)), R, _dev_ptr(out, "out", (R, Nr)), fl, _stream_ptr(stream))
    _check(st, "gp_kmvm_noalloc")
    return out


def kmvm_noalloc_status(stream=None) -> int:
    """gp_kmvm_noalloc_check: device-side status of the no-alloc calls on the
    current device since the last check (synchronises the stream, clears it)."""
    fn = lib().gp_kmvm_noalloc_check
    fn.restype = _c_int
    fn.argtypes = [_c_void_p]
    return int(fn(_stream_ptr(stream)))


MLL_PRECOND_PROBES = 0x1
MLL_WANT_LOGDET = 0x2


def kmvm_vjp(ctx: Context, hyp: Hyper, X, U, W, want_X: bool = False, precision="fp32", stream=None):
    """gp_kmvm_vjp / gp_kmvm_vjp_prec: gradient of sum_c u_c^T Ktilde w_c w.r.t.
    (l_1..l_d, a^2, sigma^2) (numpy, d + 2) and optionally X (CUDA tensor N x d).
    U, W: (R, N).  precision "fp32": the CUDA-core backward; "fp16": the
    tensor-core backward (RBF / Matern-3/2 / Matern-5/2)."""
    import torch
    N, d = X.shape
    R = U.shape[0]
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    h = hyp.c()
    fw = lib().gp_kmvm_vjp_prec_workspace_size
    fw.restype = ctypes.c_size_t
    fw.argtypes = [ctypes.POINTER(_Hyp), _c_i64, _c_int, _c_int]
    need = int(fw(ctypes.byref(h), N, R, prec))
    if need == 0:
        raise GPKError(GP_ERR_UNSUPPORTED if prec != FP32 else GP_ERR_INVALID, "gp_kmvm_vjp_prec_workspace_size")
    if need > ctx.workspace_bytes:
        ctx.reserve(need)
    g = np.zeros(d + 2, np.float64)
    gX = torch.empty((N, d), dtype=torch.float32, device=X.device) if want_X else None
    fn = lib().gp_kmvm_vjp_prec
    fn.restype = _c_int
    fn.argtypes = [_c_void_p, ctypes.POINTER(_Hyp), _c_void_p, _c_i64, _c_void_p, _c_void_p, _c_int, _c_int,
                   _c_void_p, _c_void_p, _c_void_p]
    st = fn(ctx.ptr, ctypes.byref(h), _dev_ptr(X, "X", (N, d)), N, _dev_ptr(U, "U", (R, N)),
            _dev_ptr(W, "W", (R, N)), R, prec, g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            int(gX.data_ptr()) if gX is not None else None, _stream_ptr(stream))
    _check(st, "gp_kmvm_vjp_prec")
    return g, gX


def slq_quadrature(alpha, beta, gamma0: float) -> float:
    """gp_slq_quadrature (host only): gamma0 * e1^T log(T) e1 for the Lanczos
    tridiagonal of CG step sizes alpha[0..J), beta[0..J-1)."""
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta if len(beta) else [0.0], dtype=np.float64)
    out = ctypes.c_double(0.0)
    P = ctypes.POINTER(ctypes.c_double)
    _check(lib().gp_slq_quadrature(a.ctypes.data_as(P), b.ctypes.data_as(P), int(a.shape[0]), float(gamma0),
                                   ctypes.byref(out)), "gp_slq_quadrature")
    return float(out.value)


def mll_and_grad(ctx: Context, hyp: Hyper, X, y, Z, precond: Precond | None = None, E=None,
                 precond_probes: bool = False, want_logdet: bool = True, tol: float = 1e-2, max_iter: int = 100,
                 precision="fp16", want_X: bool = False, return_U: bool = False, restarts: int = 4,
                 check_precision="fp32", escalate: bool = True, min_iter: int = 0, loss_depth: int = 0,
                 stream=None):
    """gp_mll_and_grad.  X (N, d), y (N,), Z (M, N) probes [, E (M, rank) normals]
    -> (mll, grad (numpy, d + 2), grad_X or None, U or None, info).  min_iter: CG
    iterations run before the tolerance is tested (a loose tolerance such as the
    training loop's 1.0 is otherwise met by x_0 = 0).  loss_depth: with
    want_logdet, the Lanczos depth (iterations of every column) the loss value
    is taken from, whatever the tolerance (GP_MLL_SLQ_MIN_ITER)."""
    import torch
    N, d = X.shape
    M = Z.shape[0]
    R = M + 1
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    opts = _CgOpts(float(tol), int(max_iter), int(min_iter), prec, CG_STABLE, REORTH_PINV, 1, 0, int(restarts),
                   _check_flags(check_precision, prec), 1 if escalate else 0)
    h = hyp.c()
    rank = precond.rank if precond is not None else 0
    need = int(lib().gp_mll_workspace_size(ctypes.byref(h), N, M, rank, ctypes.byref(opts)))
    if need == 0:
        raise GPKError(GP_ERR_INVALID, "gp_mll_workspace_size")
    if need > ctx.workspace_bytes:
        ctx.reserve(need)
    flags = (MLL_PRECOND_PROBES if precond_probes else 0) | (MLL_WANT_LOGDET if want_logdet else 0) | \
        ((int(loss_depth) & 0xff) << 8)
    mll = ctypes.c_double(0.0)
    g = np.zeros(d + 2, np.float64)
    gX = torch.empty((N, d), dtype=torch.float32, device=X.device) if want_X else None
    U = torch.empty((R, N), dtype=torch.float32, device=X.device) if return_U else None
    col_iters = np.zeros(R, np.int32)
    rel = np.zeros(R, np.float64)
    g0 = np.zeros(R, np.float64)
    lz = np.zeros(R, np.int32)
    Pd, Pi = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    stats = _CgStats(0, 0, 0, 0, 0, col_iters.ctypes.data_as(Pi), rel.ctypes.data_as(Pd), None, None,
                     g0.ctypes.data_as(Pd), None, lz.ctypes.data_as(Pi))
    pc = precond.c() if precond is not None else _Precond(None, None, 0)
    st = lib().gp_mll_and_grad(ctx.ptr, ctypes.byref(h), _dev_ptr(X, "X", (N, d)), _dev_ptr(y, "y", (N,)), N,
                               _dev_ptr(Z, "Z", (M, N)), M,
                               _dev_ptr(E, "E", (M, rank)) if E is not None else None,
                               ctypes.byref(pc), ctypes.byref(opts), flags, ctypes.byref(mll),
                               g.ctypes.data_as(Pd), int(gX.data_ptr()) if gX is not None else None,
                               int(U.data_ptr()) if U is not None else None, ctypes.byref(stats), _stream_ptr(stream))
    _check(st, "gp_mll_and_grad")
    info = {"iters": int(stats.iters), "converged": int(stats.converged), "restarts": int(stats.restarts),
            "col_iters": col_iters, "rel_resid": rel, "gamma0": g0, "lanczos_len": lz}
    return float(mll.value), g, gX, U, info


# ---- serving ----------------------------------------------------------------------


def _server_opts(arena_bytes, max_slots, rank, precision, mean_precision, tol, max_iter, restarts, reorth,
                 refine_precision=None, refine_resid=0.0, large_n=0, large_reserve=0):
    return _ServerOpts(int(arena_bytes), int(max_slots), int(rank), PRECISIONS.get(precision, precision),
                       PRECISIONS.get(mean_precision, mean_precision), float(tol), int(max_iter), int(restarts),
                       REORTH.get(reorth, reorth),
                       0 if refine_precision is None else PRECISIONS.get(refine_precision, refine_precision),
                       float(refine_resid), int(large_n), int(large_reserve))


class ServeFuture:
    """Handle of one submitted request; result() blocks until it completes."""

    def __init__(self, server, rid, keep, mean):
        self._server, self.id, self._keep, self._mean = server, rid, keep, mean
        self._done = None

    def result(self, timeout: float | None = None):
        """(mean (n_test,) float32 numpy array, stats dict); raises GPKError for a
        failed request (GP_ERR_NOT_CONVERGED is reported in stats, not raised)."""
        if self._done is None:
            st = _ReqStats()
            rc = lib().gp_server_wait(self._server._h, ctypes.c_uint64(self.id),
                                      -1.0 if timeout is None else float(timeout), ctypes.byref(st))
            if rc == GP_ERR_TIMEOUT and st.t_done_ms == 0.0 and timeout is not None:
                raise TimeoutError(f"request {self.id} still running after {timeout} s")
            stats = {"status": st.status, "iters": st.iters, "restarts": st.restarts, "rel_resid": st.rel_resid,
                     "t_submit_ms": st.t_submit_ms, "t_admit_ms": st.t_admit_ms, "t_done_ms": st.t_done_ms,
                     "latency_ms": st.t_done_ms - st.t_submit_ms, "bytes": int(st.bytes)}
            self._done = (self._mean.numpy().copy(), stats)
            self._keep = None
            if st.status not in (GP_OK, GP_ERR_NOT_CONVERGED):
                raise GPKError(st.status, f"request {self.id}")
        return self._done


class Server:
    """Continuous-batching GP posterior-mean server (gp_server_*).

    Each request solves (K + sigma^2 I) v = y with the stable preconditioned CG
    and returns mu* = K(X*, X) v.  Inputs are copied into page-locked host
    tensors at submit so the library's uploads are asynchronous.  The default
    CG MVM forms S on the tensor cores from FP16 inputs carried as hi + lo and
    keeps the kernel values and the one-column value product in FP32
    (MVM_FP32_PV): over the serving workload's range of noise levels a single
    FP16 rounding of the kernel tile can leave the operator too inexact for CG
    to converge, and for one right-hand side the FP32 product is also twice as
    fast as the hi + lo FP16 tile on the tensor cores.  Requests with
    N >= large_n leave large_reserve SMs to the kernels of smaller requests."""

    def __init__(self, device: int = 0, arena_bytes: int = 8 << 30, max_slots: int = 8, rank: int = 20,
                 precision=FP16 | MVM_XSPLIT | MVM_FP32_PV, mean_precision="fp32", tol: float = 1e-2,
                 max_iter: int = 1000, restarts: int = 4, reorth="pinv", refine_precision=None,
                 refine_resid: float = 0.0, large_n: int = 32768, large_reserve: int = 16):
        self.opts = _server_opts(arena_bytes, max_slots, rank, precision, mean_precision, tol, max_iter, restarts,
                                 reorth, refine_precision, refine_resid, large_n, large_reserve)
        h = _c_void_p()
        _check(lib().gp_server_create(int(device), ctypes.byref(self.opts), ctypes.byref(h)), "gp_server_create")
        self._h = h

    def request_bytes(self, hyp: Hyper, N: int, n_test: int) -> int:
        hc = hyp.c()
        return int(lib().gp_server_request_bytes(ctypes.byref(self.opts), ctypes.byref(hc), int(N), int(n_test)))

    @staticmethod
    def pinned(a):
        """A page-locked contiguous float32 host tensor holding `a` (returned
        as is when it already is one)."""
        import torch
        if isinstance(a, torch.Tensor) and not a.is_cuda and a.dtype == torch.float32 and a.is_contiguous() \
                and a.is_pinned():
            return a
        return torch.as_tensor(np.ascontiguousarray(np.asarray(a), dtype=np.float32)).pin_memory()

    def submit(self, hyp: Hyper, X, y, X_test) -> ServeFuture:
        """Queue one request (X (N, d), y (N,), X_test (n_test, d)); returns a
        ServeFuture.  Page-locked float32 tensors are used in place."""
        import torch
        X, y, Xs = self.pinned(X), self.pinned(y), self.pinned(X_test)
        N, d = X.shape
        n_test = Xs.shape[0]
        if y.shape != (N,) or Xs.shape[1] != d or hyp.d != d:
            raise ValueError("shape mismatch between X, y, X_test and the lengthscales")
        mean = torch.empty(n_test, dtype=torch.float32).pin_memory()
        hc = hyp.c()
        rid = ctypes.c_uint64()
        _check(lib().gp_server_submit(self._h, ctypes.byref(hc), X.data_ptr(), int(N), y.data_ptr(), Xs.data_ptr(),
                                      int(n_test), mean.data_ptr(), ctypes.byref(rid)), "gp_server_submit")
        return ServeFuture(self, rid.value, (X, y, Xs, hc), mean)

    def stats(self) -> dict:
        st = _ServerStats()
        _check(lib().gp_server_stats(self._h, ctypes.byref(st)), "gp_server_stats")
        return {k: getattr(st, k) for k, _ in _ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib().gp_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass



# the C entry points' names (without the gp_ prefix) for every call of the boundary
pivchol = pivchol_precond
