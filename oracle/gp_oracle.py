"""FP64 reference computations for the low-precision GP solve (oracle).

TEST INFRASTRUCTURE ONLY -- see the package docstring.  Plain numpy in
float64; every function names the passage of the paper it follows.

Notation (paper, Sec. 2.2 and Eq. mvm):
  X        N x d inputs, one point per row
  theta    (l_1..l_d, a^2, sigma^2): ARD lengthscales, outputscale, noise
  K        K_ij = a^2 k(x_i, x_j)          (no noise)
  Ktilde   K + sigma^2 I                    (Sec. 2.2)
  r^2      sum_k (x_ik - x_jk)^2 / l_k^2    (ARD-scaled squared distance)

Kernels (k is the unit-outputscale kernel as a function of r):
  'rbf'       exp(-r^2/2)                               (App. C.1)
  'matern12'  exp(-r)                                   (Sec. 3.1, App. C.1)
  'matern32'  (1 + sqrt3 r) exp(-sqrt3 r)   textbook form; the paper uses the
                                            kernel (tables, Fig. 5e) without
                                            writing it out
  'matern52'  (1 + sqrt5 r + 5r^2/3) exp(-sqrt5 r)  textbook form, as above

Readings of the paper that this file takes (each is also listed with the
design notes of the repository):
  * Alg. 2's loop condition is printed inverted ("while ||r|| < eps"); it is
    read as "while the relative residual ||r_k|| / ||b|| exceeds eps" with an
    optional iteration floor and cap.
  * Alg. 1/2 print d_0 = -r_0 and d_{k+1} = -r_{k+1} + beta d_k although
    z = P(r) is formed; the preconditioned update d = -z (+ beta d) is used.
  * P(.) in Alg. 2 is the application of P^{-1} (Eq. woodbury).
  * Re-orthogonalisation: 'euclid' is the literal form of Alg. 2 (u_j the
    Euclidean-normalised past residuals); 'pinv' projects in the
    P^{-1} inner product, in which preconditioned residuals are orthogonal.
  * The Hutchinson constant is 1/(2M) (Eq. approx_loss / approx).
  * The RQ support bound uses eps^(-1/alpha) (App. C.1 prints eps^(1/alpha)).
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Hyp", "KERNELS", "unit_kernel", "unit_kernel_dr2", "sqdist",
    "kernel_matrix", "ktilde_dense", "kmvm", "kmvm_rows",
    "cholesky_solve", "logdet_exact", "mll_exact", "dktilde_dtheta",
    "mll_grad_exact", "quad_form_grad", "pseudo_loss_grad",
    "lse_dot", "LSEBreakdown",
    "pivoted_cholesky", "woodbury_core", "precond_apply", "precond_logdet",
    "cg_standard", "cg_stable", "cg_mbcg", "CGResult", "minres", "MinresResult",
    "lanczos_tridiagonal", "slq_quadrature",
    "max_distance", "relative_residual",
]

KERNELS = ("rbf", "matern32", "matern12", "matern52")


@dataclass
class Hyp:
    """GP hyperparameters theta = (l_1..l_d, a^2, sigma^2) (Sec. 2.2, Eq. mvm)."""
    kernel: str
    lengthscale: np.ndarray
    outputscale: float = 1.0   # a^2
    noise: float = 0.01        # sigma^2

    def __post_init__(self):
        if self.kernel not in KERNELS:
            raise ValueError(f"unknown kernel {self.kernel!r}")
        self.lengthscale = np.atleast_1d(np.asarray(self.lengthscale, dtype=np.float64))


# ---------------------------------------------------------------------------
# Kernel functions (Sec. 2.2, App. C.1)
# ---------------------------------------------------------------------------

def unit_kernel(r2: np.ndarray, kernel: str) -> np.ndarray:
    """k as a function of the squared scaled distance r^2 (outputscale 1)."""
    r2 = np.maximum(np.asarray(r2, dtype=np.float64), 0.0)
    if kernel == "rbf":
        return np.exp(-0.5 * r2)
    r = np.sqrt(r2)
    if kernel == "matern12":
        return np.exp(-r)
    if kernel == "matern32":
        s = math.sqrt(3.0) * r
        return (1.0 + s) * np.exp(-s)
    if kernel == "matern52":
        s = math.sqrt(5.0) * r
        return (1.0 + s + s * s / 3.0) * np.exp(-s)
    raise ValueError(kernel)


def unit_kernel_dr2(r2: np.ndarray, kernel: str) -> np.ndarray:
    """dk/d(r^2), the derivative used by every hyperparameter gradient.

    rbf: -k/2;  matern32: -(3/2) exp(-sqrt3 r);  matern52:
    -(5/6)(1 + sqrt5 r) exp(-sqrt5 r);  matern12: -exp(-r)/(2r), taken as 0
    at r = 0 where every (x_i - x_j) factor it multiplies is also 0.
    """
    r2 = np.maximum(np.asarray(r2, dtype=np.float64), 0.0)
    if kernel == "rbf":
        return -0.5 * np.exp(-0.5 * r2)
    r = np.sqrt(r2)
    if kernel == "matern32":
        return -1.5 * np.exp(-math.sqrt(3.0) * r)
    if kernel == "matern52":
        s = math.sqrt(5.0) * r
        return -(5.0 / 6.0) * (1.0 + s) * np.exp(-s)
    if kernel == "matern12":
        out = np.zeros_like(r)
        nz = r > 0
        out[nz] = -np.exp(-r[nz]) / (2.0 * r[nz])
        return out
    raise ValueError(kernel)


def sqdist(X1: np.ndarray, X2: np.ndarray, lengthscale: np.ndarray) -> np.ndarray:
    """r^2_ij = sum_k (x1_ik - x2_jk)^2 / l_k^2, formed from differences
    (not from the expanded |x|^2 + |x'|^2 - 2 x.x', which cancels)."""
    X1 = np.asarray(X1, dtype=np.float64)
    X2 = np.asarray(X2, dtype=np.float64)
    ls = np.asarray(lengthscale, dtype=np.float64)
    r2 = np.zeros((X1.shape[0], X2.shape[0]))
    for k in range(X1.shape[1]):
        diff = (X1[:, k:k + 1] - X2[None, :, k]) / ls[k]
        r2 += diff * diff
    return r2


def kernel_matrix(X1, X2, hyp: Hyp) -> np.ndarray:
    """K(X1, X2)_ij = a^2 k(x_i, x_j)  (Eq. mvm, without the noise term)."""
    return hyp.outputscale * unit_kernel(sqdist(X1, X2, hyp.lengthscale), hyp.kernel)


def ktilde_dense(X, hyp: Hyp) -> np.ndarray:
    """Ktilde = K + sigma^2 I  (Sec. 2.2)."""
    K = kernel_matrix(X, X, hyp)
    K[np.diag_indices_from(K)] += hyp.noise
    return K


def kmvm(Xr, Xc, V, hyp: Hyp, add_noise: bool = False, block_rows: int = 256) -> np.ndarray:
    """Matrix-free kernel MVM (Eq. mvm):

        (Ktilde v)_i = a^2 sum_j k(x_i, x_j) v_j + sigma^2 v_i.

    Xr: rows (Nr x d), Xc: columns (Nc x d), V: Nc x R.  The noise term needs
    Xr to be Xc (a square operator).  Rows are processed block by block only
    so that the Nr x Nc matrix never has to exist at once.
    """
    Xr = np.asarray(Xr, dtype=np.float64)
    Xc = np.asarray(Xc, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    vec = V.ndim == 1
    if vec:
        V = V[:, None]
    out = np.empty((Xr.shape[0], V.shape[1]))
    for i0 in range(0, Xr.shape[0], block_rows):
        i1 = min(i0 + block_rows, Xr.shape[0])
        out[i0:i1] = kernel_matrix(Xr[i0:i1], Xc, hyp) @ V
    if add_noise:
        if Xr.shape[0] != Xc.shape[0]:
            raise ValueError("the noise term needs a square operator")
        out += hyp.noise * V
    return out[:, 0] if vec else out


def kmvm_rows(X, rows, V, hyp: Hyp, add_noise: bool = True) -> np.ndarray:
    """Rows `rows` of Ktilde V exactly (Eq. mvm), for spot checks at large N."""
    X = np.asarray(X, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    rows = np.asarray(rows)
    out = kmvm(X[rows], X, V, hyp, add_noise=False)
    if add_noise:
        out = out + hyp.noise * V[rows]
    return out


def relative_residual(X, U, B, hyp: Hyp, rows=None) -> np.ndarray:
    """Per-column ||Ktilde U - B|| / ||B|| in FP64, over all rows or a sample."""
    U = np.asarray(U, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    if U.ndim == 1:
        U, B = U[:, None], B[:, None]
    if rows is None:
        res = kmvm(X, X, U, hyp, add_noise=True) - B
        return np.linalg.norm(res, axis=0) / np.linalg.norm(B, axis=0)
    res = kmvm_rows(X, rows, U, hyp, add_noise=True) - B[rows]
    return np.linalg.norm(res, axis=0) / np.linalg.norm(B[rows], axis=0)


# ---------------------------------------------------------------------------
# Exact solves, log-determinant, marginal likelihood (Sec. 2.2)
# ---------------------------------------------------------------------------

def _cholesky(A):
    return np.linalg.cholesky(A)


def _cho_solve(Lc, B):
    Y = np.linalg.solve(Lc, B)        # forward substitution (triangular)
    return np.linalg.solve(Lc.T, Y)   # back substitution


def cholesky_solve(X, hyp: Hyp, B) -> np.ndarray:
    """Ktilde^{-1} B through the Cholesky factor of the dense Ktilde (Sec. 2.2)."""
    Lc = _cholesky(ktilde_dense(X, hyp))
    return _cho_solve(Lc, np.asarray(B, dtype=np.float64))


def logdet_exact(X, hyp: Hyp) -> float:
    """log |Ktilde| = 2 sum log diag(chol(Ktilde))."""
    Lc = _cholesky(ktilde_dense(X, hyp))
    return 2.0 * float(np.sum(np.log(np.diag(Lc))))


def mll_exact(X, y, hyp: Hyp) -> float:
    """Negative log marginal likelihood (Eq. loss):
        1/2 log|Ktilde| + 1/2 y^T Ktilde^{-1} y + N/2 log(2 pi)."""
    y = np.asarray(y, dtype=np.float64)
    Lc = _cholesky(ktilde_dense(X, hyp))
    alpha = _cho_solve(Lc, y)
    N = y.shape[0]
    return float(np.sum(np.log(np.diag(Lc))) + 0.5 * y @ alpha + 0.5 * N * math.log(2.0 * math.pi))


def dktilde_dtheta(X, hyp: Hyp) -> list:
    """Dense derivatives of Ktilde w.r.t. theta = (l_1..l_d, a^2, sigma^2).

    d/dl_m  : a^2 k'(r^2) * (-2 (x_im - x_jm)^2 / l_m^3)
    d/da^2  : k
    d/dsig^2: I
    """
    X = np.asarray(X, dtype=np.float64)
    ls = hyp.lengthscale
    r2 = sqdist(X, X, ls)
    dk = unit_kernel_dr2(r2, hyp.kernel)
    mats = []
    for m in range(X.shape[1]):
        diff = X[:, m:m + 1] - X[None, :, m]
        mats.append(hyp.outputscale * dk * (-2.0 * diff * diff / ls[m] ** 3))
    mats.append(unit_kernel(r2, hyp.kernel))
    mats.append(np.eye(X.shape[0]))
    return mats


def mll_grad_exact(X, y, hyp: Hyp) -> np.ndarray:
    """Exact gradient of the loss (Eq. gradient, first line):
        1/2 tr(Ktilde^{-1} dKtilde) - 1/2 alpha^T dKtilde alpha,  alpha = Ktilde^{-1} y."""
    y = np.asarray(y, dtype=np.float64)
    Kt = ktilde_dense(X, hyp)
    Kinv = np.linalg.inv(Kt)
    alpha = Kinv @ y
    return np.array([0.5 * np.sum(Kinv * dK.T) - 0.5 * alpha @ dK @ alpha
                     for dK in dktilde_dtheta(X, hyp)])


def quad_form_grad(X, hyp: Hyp, U, V, wrt_X: bool = False):
    """Gradient of q(theta, X) = sum_c u_c^T Ktilde v_c (u, v held fixed).

    This is the quantity a backward pass through the MVM of Eq. mvm returns.
    Returns (g_theta [d+2], g_X [N x d] or None).
    """
    X = np.asarray(X, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64).reshape(X.shape[0], -1)
    V = np.asarray(V, dtype=np.float64).reshape(X.shape[0], -1)
    g = np.array([np.sum(U * (dK @ V)) for dK in dktilde_dtheta(X, hyp)])
    if not wrt_X:
        return g, None
    ls = hyp.lengthscale
    r2 = sqdist(X, X, ls)
    W = hyp.outputscale * unit_kernel_dr2(r2, hyp.kernel)
    G = U @ V.T + V @ U.T                     # G_ij = sum_c u_ic v_jc + u_jc v_ic
    WG = W * G
    gX = np.zeros_like(X)
    for m in range(X.shape[1]):
        diff = X[:, m:m + 1] - X[None, :, m]   # x_im - x_jm
        gX[:, m] = np.sum(WG * 2.0 * diff, axis=1) / ls[m] ** 2
    return g, gX


def pseudo_loss_grad(X, hyp: Hyp, U, Z, W=None) -> np.ndarray:
    """Gradient of the pseudo-loss (Eq. approx_loss -> Eq. approx):

        1/(2M) sum_{j>=1} u_j^T (dKtilde w_j) - 1/2 u_0^T (dKtilde u_0)

    U = [u_0 .. u_M] (N x (M+1)) are the detached solves of Eq. cg, Z the
    probes.  w_j = z_j for probes with E[z z^T] = I (the paper's form); for
    probes drawn with E[z z^T] = P pass W = P^{-1} Z so the trace estimate
    stays unbiased.
    """
    U = np.asarray(U, dtype=np.float64)
    Z = np.asarray(Z, dtype=np.float64)
    M = Z.shape[1]
    Wp = Z if W is None else np.asarray(W, dtype=np.float64)
    g_probe, _ = quad_form_grad(X, hyp, U[:, 1:], Wp)
    g_y, _ = quad_form_grad(X, hyp, U[:, :1], U[:, :1])
    return g_probe / (2.0 * M) - 0.5 * g_y


# ---------------------------------------------------------------------------
# LSE scalar trick (Sec. 4.2, "Rescaling Conjugate Gradients")
# ---------------------------------------------------------------------------

class LSEBreakdown(ArithmeticError):
    """The signed sum inside LSE is not positive: log(w^T z) does not exist."""


def lse_dot(w, z) -> float:
    """log(w^T z) by the paper's transformation:

        y_i = log|w_i| + log|z_i|,  s_i = sign(w_i z_i),
        LSE = y_max + log( sum_i s_i exp(y_i - y_max) ).

    Entries with w_i z_i = 0 contribute nothing (log 0 = -inf) and are
    skipped.  A non-positive signed sum raises LSEBreakdown.
    """
    w = np.asarray(w, dtype=np.float64).ravel()
    z = np.asarray(z, dtype=np.float64).ravel()
    keep = (w != 0.0) & (z != 0.0)
    if not np.any(keep):
        raise LSEBreakdown("w^T z has no nonzero terms")
    y = np.log(np.abs(w[keep])) + np.log(np.abs(z[keep]))
    s = np.sign(w[keep]) * np.sign(z[keep])   # sign of the product, without forming it
    y_max = np.max(y)
    total = np.sum(s * np.exp(y - y_max))
    if not total > 0.0:
        raise LSEBreakdown(f"signed sum {total!r} is not positive")
    return float(y_max + math.log(total))


# ---------------------------------------------------------------------------
# Pivoted-Cholesky preconditioner and Woodbury apply (Sec. 4.2, Eq. woodbury)
# ---------------------------------------------------------------------------

def pivoted_cholesky(X, hyp: Hyp, rank: int, rel_tol: float = 1e-10):
    """Rank-k partial pivoted Cholesky of K (no noise), from rows K e_p and the
    diagonal, which is the constant a^2 for a stationary kernel (Sec. 4.2).

    Step m: p = argmax of the remaining diagonal (numpy's argmax: lowest index
    on ties); stop if that value is <= rel_tol * a^2; otherwise
        l_m = (K e_p - L_{:, <m} L_{p, <m}^T) / sqrt(diag_p),
        diag <- diag - l_m^2.
    Returns (L [N x m], pivots [m]).
    """
    X = np.asarray(X, dtype=np.float64)
    N = X.shape[0]
    diag = np.full(N, float(hyp.outputscale))
    L = np.zeros((N, rank))
    piv = []
    for m in range(rank):
        p = int(np.argmax(diag))
        if diag[p] <= rel_tol * hyp.outputscale:
            break
        row = kernel_matrix(X[p:p + 1], X, hyp)[0]
        col = (row - L[:, :m] @ L[p, :m]) / math.sqrt(diag[p])
        L[:, m] = col
        diag = diag - col * col
        piv.append(p)
    return L[:, :len(piv)], np.array(piv, dtype=np.int64)


def woodbury_core(L, noise: float) -> np.ndarray:
    """Cholesky factor of the k x k core I + sigma^{-2} L^T L (Eq. woodbury)."""
    L = np.asarray(L, dtype=np.float64)
    C = np.eye(L.shape[1]) + (L.T @ L) / noise
    return _cholesky(C)


def precond_apply(L, noise: float, W) -> np.ndarray:
    """P^{-1} w = sigma^{-2} w - sigma^{-4} L (I + sigma^{-2} L^T L)^{-1} L^T w
    (Eq. woodbury), P = L L^T + sigma^2 I."""
    L = np.asarray(L, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    if L.shape[1] == 0:
        return W / noise
    Cc = woodbury_core(L, noise)
    c = _cho_solve(Cc, L.T @ W)
    return W / noise - (L @ c) / (noise * noise)


def precond_logdet(L, noise: float) -> float:
    """log|L L^T + sigma^2 I| = N log sigma^2 + log|I + sigma^{-2} L^T L|
    (matrix determinant lemma)."""
    L = np.asarray(L, dtype=np.float64)
    N = L.shape[0]
    if L.shape[1] == 0:
        return N * math.log(noise)
    Cc = woodbury_core(L, noise)
    return N * math.log(noise) + 2.0 * float(np.sum(np.log(np.diag(Cc))))


# ---------------------------------------------------------------------------
# Conjugate gradients: Alg. 1 (standard) and Alg. 2 (enhanced stability)
# ---------------------------------------------------------------------------

@dataclass
class CGResult:
    x: np.ndarray
    iters: int
    resid: list = field(default_factory=list)     # ||r_k|| / ||b|| per iterate
    alphas: list = field(default_factory=list)
    betas: list = field(default_factory=list)     # beta_{k+1}, k = 0, 1, ...
    gamma0: float = 0.0                           # r_0^T z_0
    breakdown: bool = False


def _identity(r):
    return r


def cg_standard(matvec, b, x0=None, precond=None, tol=1e-6, max_iter=None,
                min_iter=0) -> CGResult:
    """Preconditioned CG, Alg. 1 (App. A), one right-hand side.

    r_0 = K(x_0) - b, z_0 = P(r_0), d_0 = -z_0, gamma_0 = r_0^T z_0;
    alpha_k = gamma_k / d_k^T K(d_k); x += alpha d; r += alpha K(d);
    z = P(r); gamma' = r^T z; beta = gamma'/gamma; d = -z + beta d.
    """
    b = np.asarray(b, dtype=np.float64)
    P = precond or _identity
    N = b.shape[0]
    max_iter = N if max_iter is None else max_iter
    x = np.zeros(N) if x0 is None else np.array(x0, dtype=np.float64)
    r = matvec(x) - b
    z = P(r)
    d = -z
    gamma = float(r @ z)
    bnorm = float(np.linalg.norm(b))
    res = CGResult(x=x, iters=0, gamma0=gamma)
    res.resid.append(float(np.linalg.norm(r)) / bnorm)
    k = 0
    while (res.resid[-1] > tol or k < min_iter) and k < max_iter:
        Kd = matvec(d)
        alpha = gamma / float(d @ Kd)
        x = x + alpha * d
        r = r + alpha * Kd
        z = P(r)
        gamma_new = float(r @ z)
        beta = gamma_new / gamma
        d = -z + beta * d
        gamma = gamma_new
        k += 1
        res.alphas.append(alpha)
        res.betas.append(beta)
        res.resid.append(float(np.linalg.norm(r)) / bnorm)
    res.x, res.iters = x, k
    return res


def cg_stable(matvec, b, x0=None, precond=None, tol=1e-6, max_iter=None,
              min_iter=0, reorth: str = "pinv") -> CGResult:
    """Enhanced-stability CG, Alg. 2 (Sec. 4.2), one right-hand side.

    Differences from Alg. 1: alpha and beta are carried in log scale through
    LSE (log alpha_k = log gamma_k - LSE(d_k^T K d_k); log gamma = LSE(r^T z);
    beta = exp(log gamma_{k+1} - log gamma_k)), and after the residual update
    r_{k+1} is re-orthogonalised against all previous residuals r_0..r_k:
      'euclid': r <- r - (u_j^T r) u_j, u_j = r_j / ||r_j||, j = 0..k in turn
      'pinv'  : r <- r - (zeta_j^T r) rho_j, rho_j = r_j / sqrt(r_j^T z_j),
                zeta_j = z_j / sqrt(r_j^T z_j)  (P^{-1}-orthogonal form)
      'none'  : no re-orthogonalisation.
    The multi-RHS solve of Eq. cg runs this per column with per-column scalars
    (App. A, mBCG), so batching does not change any column's arithmetic.
    """
    b = np.asarray(b, dtype=np.float64)
    P = precond or _identity
    N = b.shape[0]
    max_iter = N if max_iter is None else max_iter
    x = np.zeros(N) if x0 is None else np.array(x0, dtype=np.float64)
    r = matvec(x) - b
    z = P(r)
    d = -z
    bnorm = float(np.linalg.norm(b))
    res = CGResult(x=x, iters=0)
    res.resid.append(float(np.linalg.norm(r)) / bnorm)
    if res.resid[-1] == 0.0:
        return res
    log_gamma = lse_dot(r, z)
    res.gamma0 = math.exp(log_gamma)
    basis_r, basis_z = [], []

    def remember(rv, zv, lg):
        if reorth == "euclid":
            basis_r.append(rv / np.linalg.norm(rv))
        elif reorth == "pinv":
            s = math.exp(-0.5 * lg)
            basis_r.append(rv * s)
            basis_z.append(zv * s)

    remember(r, z, log_gamma)
    k = 0
    while (res.resid[-1] > tol or k < min_iter) and k < max_iter:
        Kd = matvec(d)
        try:
            log_alpha = log_gamma - lse_dot(d, Kd)
        except LSEBreakdown:
            res.breakdown = True
            break
        alpha = math.exp(log_alpha)
        x = x + alpha * d
        r = r + alpha * Kd
        if reorth == "euclid":
            for u in basis_r:
                r = r - (u @ r) * u
        elif reorth == "pinv":
            for rho, zeta in zip(basis_r, basis_z):
                r = r - (zeta @ r) * rho
        z = P(r)
        try:
            log_gamma_new = lse_dot(r, z)
        except LSEBreakdown:
            res.breakdown = True
            k += 1
            res.alphas.append(alpha)
            res.resid.append(float(np.linalg.norm(r)) / bnorm)
            break
        beta = math.exp(log_gamma_new - log_gamma)
        d = -z + beta * d
        log_gamma = log_gamma_new
        remember(r, z, log_gamma)
        k += 1
        res.alphas.append(alpha)
        res.betas.append(beta)
        res.resid.append(float(np.linalg.norm(r)) / bnorm)
    res.x, res.iters = x, k
    return res


def cg_mbcg(matmat, B, precond=None, tol=1e-6, max_iter=None) -> list:
    """mBCG (App. A): Alg. 1 on every column of B (N x R) at once.  Each column
    keeps its own alpha_k, beta_k, gamma_k and stops on its own tolerance; the
    only thing shared is that one matrix product K [d_1 .. d_R] serves all
    columns per step.  Returns one CGResult per column (alphas, betas and
    gamma0 feed lanczos_tridiagonal / slq_quadrature)."""
    B = np.asarray(B, dtype=np.float64)
    P = precond or _identity
    N, R = B.shape
    max_iter = N if max_iter is None else max_iter
    X = np.zeros((N, R))
    Rm = -B.copy()                       # r_0 = K x_0 - b with x_0 = 0
    Z = P(Rm)
    D = -Z
    gamma = np.sum(Rm * Z, axis=0)
    bnorm = np.linalg.norm(B, axis=0)
    res = [CGResult(x=X[:, c], iters=0, gamma0=float(gamma[c])) for c in range(R)]
    rel = np.linalg.norm(Rm, axis=0) / bnorm
    for c in range(R):
        res[c].resid.append(float(rel[c]))
    active = rel > tol
    k = 0
    while np.any(active) and k < max_iter:
        KD = matmat(D)
        alpha = np.where(active, gamma / np.where(active, np.sum(D * KD, axis=0), 1.0), 0.0)
        X = X + alpha * D
        Rm = Rm + alpha * KD
        Z = P(Rm)
        gamma_new = np.sum(Rm * Z, axis=0)
        beta = np.where(active, gamma_new / np.where(active, gamma, 1.0), 0.0)
        D = np.where(active, -Z + beta * D, D)
        gamma = np.where(active, gamma_new, gamma)
        rel = np.linalg.norm(Rm, axis=0) / bnorm
        k += 1
        for c in np.nonzero(active)[0]:
            res[c].alphas.append(float(alpha[c]))
            res[c].betas.append(float(beta[c]))
            res[c].resid.append(float(rel[c]))
            res[c].iters = k
        active = active & (rel > tol)
    for c in range(R):
        res[c].x = X[:, c]
    return res


# ---------------------------------------------------------------------------
# MINRES (Conclusion: a further iterative method for the low-precision approach)
# ---------------------------------------------------------------------------

@dataclass
class MinresResult:
    x: np.ndarray
    iters: int
    resid_p: list = field(default_factory=list)   # ||r_k||_{P^-1} / ||b||_{P^-1} from the recurrence
    alphas: list = field(default_factory=list)    # Lanczos diagonal
    betas: list = field(default_factory=list)     # Lanczos off-diagonal beta_{k+1}
    breakdown: bool = False


def minres(matvec, b, precond=None, tol=1e-6, max_iter=None) -> MinresResult:
    """Preconditioned MINRES (Paige and Saunders' method), one right-hand
    side, x_0 = 0.  The paper only names MINRES as a target of its approach
    (Conclusion); this is the textbook method, written out.

    With P SPD and M = P^-1 (`precond` applies P^-1), the Lanczos process of
    M A in the P inner product gives unnormalised vectors r_k (r_1 = b) with
    y_k = M r_k, beta_k = sqrt(r_k^T y_k), v_k = y_k / beta_k (P-orthonormal),
        r_{k+1} = A v_k - alpha_k r_k / beta_k - (beta_k / beta_{k-1}) r_{k-1},
        alpha_k = v_k^T A v_k,
    i.e. the tridiagonal T_k (alpha on the diagonal, beta off it).  x_k
    minimises ||b - A x||_M over the Krylov space: with the QR factorisation
    of the (k+1) x k tridiagonal by Givens rotations, the new rotation
    (c_k, s_k) annihilates beta_{k+1}; the directions w_k = (v_k - eps_k w_{k-2}
    - delta_k w_{k-1}) / gamma_k and x_k = x_{k-1} + tau_k w_k with tau_k = c_k
    phibar_{k-1}, and ||r_k||_M = |phibar_k| = |s_k phibar_{k-1}|.
    """
    b = np.asarray(b, dtype=np.float64)
    P = precond or _identity
    N = b.shape[0]
    max_iter = N if max_iter is None else max_iter
    x = np.zeros(N)
    r_prev = np.zeros(N)           # r_{k-1}
    r_cur = b.copy()               # r_k
    y = P(r_cur)
    beta1 = math.sqrt(float(r_cur @ y))
    res = MinresResult(x=x, iters=0)
    res.resid_p.append(1.0 if beta1 > 0 else 0.0)
    if beta1 == 0.0:
        return res
    beta_prev, beta = 0.0, beta1
    # rotation state: the previous rotation (c, s), the entries it leaves in
    # the next column (dbar: the rotated sub-diagonal, eps: the fill-in two rows up)
    c, s = -1.0, 0.0
    dbar, eps = 0.0, 0.0
    phibar = beta1
    w_prev2 = np.zeros(N)          # w_{k-2}
    w_prev = np.zeros(N)           # w_{k-1}
    k = 0
    while res.resid_p[-1] > tol and k < max_iter:
        v = y / beta
        Av = matvec(v)
        u = Av - (beta / beta_prev) * r_prev if beta_prev > 0.0 else Av
        alpha = float(v @ u)
        u = u - (alpha / beta) * r_cur
        r_prev, r_cur = r_cur, u
        y = P(r_cur)
        ry = float(r_cur @ y)
        if not (ry >= 0.0) or not math.isfinite(ry):
            res.breakdown = True
            break
        beta_prev, beta = beta, math.sqrt(ry)
        # apply the previous rotation to the new column (alpha, beta) of T
        eps_k = eps                          # fill-in from two rotations ago
        delta = c * dbar + s * alpha         # entry above the diagonal
        gbar = s * dbar - c * alpha          # diagonal before the new rotation
        eps = s * beta                       # fill-in for the next column
        dbar = -c * beta                     # sub-diagonal carried to the next column
        gamma = math.hypot(gbar, beta)
        gamma = max(gamma, 1e-300)
        c, s = gbar / gamma, beta / gamma    # the rotation annihilating beta_{k+1}
        tau = c * phibar
        phibar = s * phibar
        w = (v - eps_k * w_prev2 - delta * w_prev) / gamma
        x = x + tau * w
        w_prev2, w_prev = w_prev, w
        k += 1
        res.alphas.append(alpha)
        res.betas.append(beta)
        res.resid_p.append(abs(phibar) / beta1)
        if beta == 0.0:
            break
    res.x, res.iters = x, k
    return res


# ---------------------------------------------------------------------------
# Lanczos tridiagonal from CG coefficients and SLQ (Sec. 4.3 context)
# ---------------------------------------------------------------------------

def lanczos_tridiagonal(alphas, betas) -> np.ndarray:
    """Tridiagonal T_J of the Lanczos process that (preconditioned) CG runs
    implicitly, from its step sizes (standard CG/Lanczos relation; the paper
    avoids the Lanczos log-determinant and gives no formula):

        T_00 = 1/alpha_0,  T_kk = 1/alpha_k + beta_k / alpha_{k-1}  (k >= 1),
        T_{k,k+1} = T_{k+1,k} = sqrt(beta_{k+1}) / alpha_k,

    where beta_{k+1} is the coefficient that forms d_{k+1} (Alg. 2 indexing;
    betas[k] holds beta_{k+1}).
    """
    J = len(alphas)
    T = np.zeros((J, J))
    for k in range(J):
        T[k, k] = 1.0 / alphas[k]
        if k >= 1:
            T[k, k] += betas[k - 1] / alphas[k - 1]
        if k + 1 < J:
            T[k, k + 1] = T[k + 1, k] = math.sqrt(betas[k]) / alphas[k]
    return T


def slq_quadrature(T, norm2: float) -> float:
    """Gauss quadrature of w^T log(A) w from a Lanczos tridiagonal T with start
    vector w / ||w||: ||w||^2 * sum_i (e_1^T q_i)^2 log(theta_i)."""
    evals, evecs = np.linalg.eigh(T)
    return float(norm2 * np.sum(evecs[0, :] ** 2 * np.log(evals)))


# ---------------------------------------------------------------------------
# Finite support of finite-precision kernels (Sec. 3.1, App. C.1)
# ---------------------------------------------------------------------------

def max_distance(kernel: str, lengthscale: float, eps: float, alpha: float = 5.0,
                 period: float = 1.0, lam: float = 1.0) -> float:
    """Largest distance d at which the unit kernel is still >= eps (App. C.1).

    matern12: exp(-d/l) < eps  <=>  d > -l log eps
    rbf     : exp(-d^2/(2 l^2)) < eps  <=>  d > l sqrt(-2 log eps)
    rq      : (1 + d^2/(2 alpha l^2))^-alpha < eps  <=>  d > l sqrt(2 alpha (eps^(-1/alpha) - 1))
    periodic: exp(-(2/lam) sin^2(pi d / p)) < eps  <=>  d > (p/pi) arcsin(sqrt(-lam log(eps) / 2)),
              defined when -lam log(eps) / 2 <= 1 (returns inf otherwise)
    matern32 / matern52: no closed form (App. C.1); found by bisection on the
              monotone unit kernel.
    """
    le = math.log(eps)
    if kernel == "matern12":
        return -lengthscale * le
    if kernel == "rbf":
        return lengthscale * math.sqrt(-2.0 * le)
    if kernel == "rq":
        return lengthscale * math.sqrt(2.0 * alpha * (eps ** (-1.0 / alpha) - 1.0))
    if kernel == "periodic":
        arg = -lam * le / 2.0
        if arg > 1.0:
            return math.inf
        return period / math.pi * math.asin(math.sqrt(arg))
    if kernel in ("matern32", "matern52"):
        lo, hi = 0.0, 1.0
        while unit_kernel(np.array(hi * hi), kernel) >= eps:
            hi *= 2.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if unit_kernel(np.array(mid * mid), kernel) >= eps:
                lo = mid
            else:
                hi = mid
        return lengthscale * 0.5 * (lo + hi)
    raise ValueError(kernel)
