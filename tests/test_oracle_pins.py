"""Pins of the FP64 oracle against facts fixed outside the oracle itself:
closed forms, limits, library routines, brute force on tiny inputs, and the
numbers the paper prints.  CPU only."""

import json
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _hyp(kernel, d, ls=1.0, a2=1.0, s2=0.05):
    return O.Hyp(kernel, np.full(d, ls), a2, s2)


def _points(N, d, seed=0, scale=1.0):
    return scale * np.random.default_rng(seed).standard_normal((N, d))


# --- kernel functions -------------------------------------------------------

@pytest.mark.parametrize("kernel,nu", [("matern12", 0.5), ("matern32", 1.5), ("matern52", 2.5)])
def test_matern_against_bessel_form(kernel, nu):
    """General Matern: 2^(1-nu)/Gamma(nu) (sqrt(2 nu) r)^nu K_nu(sqrt(2 nu) r)."""
    sp = pytest.importorskip("scipy.special")
    r = np.linspace(0.01, 6.0, 97)
    s = math.sqrt(2 * nu) * r
    ref = 2 ** (1 - nu) / sp.gamma(nu) * s ** nu * sp.kv(nu, s)
    np.testing.assert_allclose(O.unit_kernel(r * r, kernel), ref, rtol=1e-10)
    assert O.unit_kernel(np.array(0.0), kernel) == 1.0


def test_rbf_against_gaussian_density():
    st = pytest.importorskip("scipy.stats")
    r = np.linspace(0.0, 9.0, 91)
    np.testing.assert_allclose(O.unit_kernel(r * r, "rbf"),
                               st.norm.pdf(r) * math.sqrt(2 * math.pi), rtol=1e-12)


@pytest.mark.parametrize("kernel", O.KERNELS)
def test_kernel_derivative_by_finite_difference(kernel):
    r2 = np.linspace(0.05, 9.0, 50)
    h = 1e-6
    fd = (O.unit_kernel(r2 + h, kernel) - O.unit_kernel(r2 - h, kernel)) / (2 * h)
    np.testing.assert_allclose(O.unit_kernel_dr2(r2, kernel), fd, rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("kernel,nu", [("rbf", None), ("matern32", 1.5), ("matern12", 0.5),
                                       ("matern52", 2.5)])
def test_kernel_matrix_against_sklearn_ard(kernel, nu):
    """An independent ARD implementation (scikit-learn) on tiny inputs."""
    kern = pytest.importorskip("sklearn.gaussian_process.kernels")
    rng = np.random.default_rng(3)
    X1, X2 = rng.standard_normal((7, 3)), rng.standard_normal((5, 3))
    ls = np.array([0.7, 1.3, 2.1])
    k = kern.RBF(length_scale=ls) if nu is None else kern.Matern(length_scale=ls, nu=nu)
    hyp = O.Hyp(kernel, ls, 1.7, 0.0)
    np.testing.assert_allclose(O.kernel_matrix(X1, X2, hyp), 1.7 * k(X1, X2), rtol=1e-12)


# --- MVM (Eq. mvm) ----------------------------------------------------------

@pytest.mark.parametrize("kernel", O.KERNELS)
def test_kmvm_rank_one_limit(kernel):
    """l -> infinity: every distance rounds to 0 and Ktilde v = a^2 (1^T v) 1 + sigma^2 v."""
    X = _points(50, 4)
    V = np.random.default_rng(1).standard_normal((50, 3))
    hyp = O.Hyp(kernel, np.full(4, 1e20), 1.3, 0.07)
    ref = 1.3 * np.ones((50, 1)) * V.sum(axis=0)[None, :] + 0.07 * V
    np.testing.assert_allclose(O.kmvm(X, X, V, hyp, add_noise=True), ref, rtol=1e-12)


@pytest.mark.parametrize("kernel", O.KERNELS)
def test_kmvm_far_apart_limit(kernel):
    """Points much farther apart than l: Ktilde v = (a^2 + sigma^2) v."""
    X = np.arange(20, dtype=float)[:, None] * 1000.0 * np.ones((1, 2))
    V = np.random.default_rng(2).standard_normal((20, 2))
    hyp = O.Hyp(kernel, np.full(2, 0.01), 0.8, 0.2)
    np.testing.assert_allclose(O.kmvm(X, X, V, hyp, add_noise=True), 1.0 * V, rtol=1e-14)


def test_kmvm_symmetry_and_blocks():
    X = _points(300, 5)
    rng = np.random.default_rng(4)
    u, v = rng.standard_normal(300), rng.standard_normal(300)
    hyp = _hyp("matern32", 5, ls=0.9)
    Kv = O.kmvm(X, X, v, hyp, add_noise=True, block_rows=37)
    Ku = O.kmvm(X, X, u, hyp, add_noise=True, block_rows=64)
    assert abs(u @ Kv - v @ Ku) < 1e-10 * abs(u @ Kv)
    np.testing.assert_allclose(Kv, O.ktilde_dense(X, hyp) @ v, rtol=1e-12, atol=1e-12)
    rows = np.array([0, 17, 299])
    np.testing.assert_allclose(O.kmvm_rows(X, rows, v, hyp), Kv[rows], rtol=1e-12)


# --- exact solves, log-determinant, MLL (Sec. 2.2) ----------------------------

def test_cholesky_solve_residual():
    X = _points(200, 3)
    hyp = _hyp("rbf", 3, ls=0.6, s2=0.01)
    B = np.random.default_rng(5).standard_normal((200, 4))
    U = O.cholesky_solve(X, hyp, B)
    res = np.linalg.norm(O.ktilde_dense(X, hyp) @ U - B) / np.linalg.norm(B)
    assert res < 1e-12


def test_sherman_morrison_rank_one_limit():
    """Ktilde = sigma^2 I + a^2 1 1^T: Ktilde^{-1} = sigma^-2 (I - a^2/(sigma^2 + N a^2) 1 1^T)."""
    N, a2, s2 = 40, 1.5, 0.3
    X = _points(N, 2)
    hyp = O.Hyp("rbf", np.full(2, 1e9), a2, s2)
    B = np.random.default_rng(6).standard_normal((N, 2))
    inv = (np.eye(N) - a2 / (s2 + N * a2) * np.ones((N, N))) / s2
    np.testing.assert_allclose(O.cholesky_solve(X, hyp, B), inv @ B, rtol=1e-10)


def test_logdet_limits_and_library():
    N, a2, s2 = 30, 1.2, 0.1
    X = _points(N, 2)
    one = O.Hyp("matern32", np.full(2, 1e9), a2, s2)
    assert abs(O.logdet_exact(X, one) - ((N - 1) * math.log(s2) + math.log(s2 + N * a2))) < 1e-9
    Xfar = np.arange(N, dtype=float)[:, None] * 1e3 * np.ones((1, 2))
    diag = O.Hyp("rbf", np.full(2, 0.01), a2, s2)
    assert abs(O.logdet_exact(Xfar, diag) - N * math.log(a2 + s2)) < 1e-10
    hyp = _hyp("rbf", 2, ls=0.5)
    sign, ld = np.linalg.slogdet(O.ktilde_dense(X, hyp))
    assert sign > 0 and abs(O.logdet_exact(X, hyp) - ld) < 1e-9


def test_mll_against_multivariate_normal():
    st = pytest.importorskip("scipy.stats")
    X = _points(60, 3)
    y = np.sin(X.sum(axis=1))
    hyp = _hyp("matern32", 3, ls=0.8, a2=1.4, s2=0.02)
    ref = -st.multivariate_normal(mean=np.zeros(60), cov=O.ktilde_dense(X, hyp)).logpdf(y)
    assert abs(O.mll_exact(X, y, hyp) - ref) < 1e-9 * abs(ref)


@pytest.mark.parametrize("kernel", O.KERNELS)
def test_mll_gradient_by_finite_differences(kernel):
    X = _points(40, 3)
    y = np.cos(X[:, 0]) + 0.1 * np.random.default_rng(7).standard_normal(40)
    ls, a2, s2 = np.array([0.7, 1.1, 1.6]), 1.3, 0.05
    g = O.mll_grad_exact(X, y, O.Hyp(kernel, ls, a2, s2))
    theta = np.concatenate([ls, [a2, s2]])

    def f(t):
        return O.mll_exact(X, y, O.Hyp(kernel, t[:3], t[3], t[4]))

    for m in range(5):
        h = 1e-5 * theta[m]
        tp, tm = theta.copy(), theta.copy()
        tp[m] += h
        tm[m] -= h
        fd = (f(tp) - f(tm)) / (2 * h)
        assert abs(g[m] - fd) < 1e-6 * max(1.0, abs(fd)), (m, g[m], fd)


def test_noise_gradient_closed_form():
    """d/dsigma^2 = 1/2 tr(Ktilde^{-1}) - 1/2 ||alpha||^2."""
    X = _points(35, 2)
    y = np.sin(3 * X[:, 1])
    hyp = _hyp("rbf", 2, ls=0.7, s2=0.03)
    Kinv = np.linalg.inv(O.ktilde_dense(X, hyp))
    alpha = Kinv @ y
    assert abs(O.mll_grad_exact(X, y, hyp)[-1] - (0.5 * np.trace(Kinv) - 0.5 * alpha @ alpha)) < 1e-9


def test_pseudo_loss_gradient_is_exact_with_unit_probes():
    """Eq. approx with probes sqrt(N) e_i (M = N) and exact solves equals Eq. gradient."""
    N = 30
    X = _points(N, 2)
    y = np.sin(2 * X[:, 0])
    hyp = _hyp("matern32", 2, ls=0.9, s2=0.04)
    Z = math.sqrt(N) * np.eye(N)
    U = O.cholesky_solve(X, hyp, np.column_stack([y, Z]))
    np.testing.assert_allclose(O.pseudo_loss_grad(X, hyp, U, Z), O.mll_grad_exact(X, y, hyp),
                               rtol=1e-9, atol=1e-10)


def test_pseudo_loss_gradient_with_preconditioner_probes():
    """Probes with E[zz^T] = P paired with P^{-1} z: with z_j = sqrt(N) P^{1/2} e_j the
    estimator is again exact."""
    N = 28
    X = _points(N, 2, seed=9)
    y = np.cos(X[:, 1])
    hyp = _hyp("rbf", 2, ls=0.8, s2=0.05)
    L, _ = O.pivoted_cholesky(X, hyp, 5)
    P = L @ L.T + hyp.noise * np.eye(N)
    w, Q = np.linalg.eigh(P)
    Z = math.sqrt(N) * (Q * np.sqrt(w)) @ Q.T
    U = O.cholesky_solve(X, hyp, np.column_stack([y, Z]))
    W = O.precond_apply(L, hyp.noise, Z)
    np.testing.assert_allclose(O.pseudo_loss_grad(X, hyp, U, Z, W=W),
                               O.mll_grad_exact(X, y, hyp), rtol=1e-8, atol=1e-9)


@pytest.mark.parametrize("kernel", O.KERNELS)
def test_quad_form_gradient_wrt_inputs(kernel):
    rng = np.random.default_rng(8)
    X = rng.standard_normal((15, 3))
    U, V = rng.standard_normal((15, 2)), rng.standard_normal((15, 2))
    hyp = O.Hyp(kernel, np.array([0.8, 1.2, 1.0]), 1.1, 0.02)
    _, gX = O.quad_form_grad(X, hyp, U, V, wrt_X=True)

    def q(Xp):
        return np.sum(U * O.kmvm(Xp, Xp, V, hyp, add_noise=True))

    for i, m in [(0, 0), (3, 2), (14, 1), (7, 0)]:
        h = 1e-6
        Xp, Xm = X.copy(), X.copy()
        Xp[i, m] += h
        Xm[i, m] -= h
        fd = (q(Xp) - q(Xm)) / (2 * h)
        assert abs(gX[i, m] - fd) < 1e-6 * max(1.0, abs(fd))


# --- LSE (Sec. 4.2) ---------------------------------------------------------

def test_lse_identity():
    rng = np.random.default_rng(10)
    for _ in range(20):
        w = rng.standard_normal(500) * np.exp(rng.uniform(-30, 30))
        z = w + 0.3 * rng.standard_normal(500) * np.abs(w)
        dot = float(w @ z)
        assert abs(math.exp(O.lse_dot(w, z)) - dot) < 1e-12 * abs(dot)


def test_lse_extreme_scales_and_zeros():
    w = np.array([1e-200, 0.0, 3e-200, -1e-200])
    z = np.array([1e-200, 5.0, 1e-200, 1e-200])
    # w^T z = 3e-400 underflows as a plain FP64 dot product; LSE keeps it.
    assert abs(O.lse_dot(w, z) - (math.log(3e-200) + math.log(1e-200))) < 1e-12
    with pytest.raises(O.LSEBreakdown):
        O.lse_dot(np.array([1.0, -2.0]), np.array([1.0, 1.0]))
    with pytest.raises(O.LSEBreakdown):
        O.lse_dot(np.zeros(3), np.ones(3))


# --- pivoted Cholesky and Woodbury (Sec. 4.2, Eq. woodbury) -------------------

def test_pivoted_cholesky_invariants():
    X = _points(120, 3, seed=11)
    hyp = _hyp("matern32", 3, ls=0.9, a2=1.4)
    K = O.kernel_matrix(X, X, hyp)
    prev = None
    for rank in (1, 5, 20):
        L, piv = O.pivoted_cholesky(X, hyp, rank)
        assert piv[0] == 0                     # constant diagonal: tie -> lowest index
        assert len(set(piv.tolist())) == len(piv)
        np.testing.assert_allclose((L @ L.T)[piv], K[piv], atol=1e-10)
        rem = np.diag(K - L @ L.T)
        assert rem.min() > -1e-10
        if prev is not None:
            assert np.all(rem <= prev + 1e-10)
        prev = rem


def test_pivoted_cholesky_full_rank_is_cholesky():
    X = _points(25, 2, seed=12)
    hyp = _hyp("matern12", 2, ls=0.5)
    K = O.kernel_matrix(X, X, hyp)
    L, piv = O.pivoted_cholesky(X, hyp, 25, rel_tol=0.0)
    assert len(piv) == 25
    np.testing.assert_allclose(L @ L.T, K, atol=1e-10)
    Lp = L[piv]
    assert np.allclose(np.triu(Lp, 1), 0.0, atol=1e-12)   # lower triangular in pivot order
    np.testing.assert_allclose(Lp, np.linalg.cholesky(K[np.ix_(piv, piv)]), atol=1e-9)


def test_woodbury_is_dense_inverse():
    X = _points(80, 3, seed=13)
    hyp = _hyp("rbf", 3, ls=0.8, s2=0.02)
    L, _ = O.pivoted_cholesky(X, hyp, 10)
    P = L @ L.T + hyp.noise * np.eye(80)
    W = np.random.default_rng(14).standard_normal((80, 3))
    np.testing.assert_allclose(O.precond_apply(L, hyp.noise, W), np.linalg.solve(P, W), rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(O.precond_apply(L, hyp.noise, P @ W), W, rtol=1e-9, atol=1e-9)
    assert abs(O.precond_logdet(L, hyp.noise) - np.linalg.slogdet(P)[1]) < 1e-9


# --- CG (Alg. 1, Alg. 2) -----------------------------------------------------

# the literal Euclidean re-orthogonalization is the P = I case, so it runs
# without a preconditioner only
@pytest.mark.parametrize("reorth,rank", [("none", 0), ("none", 6), ("euclid", 0), ("pinv", 0), ("pinv", 6)])
def test_stable_cg_finite_termination(reorth, rank):
    """In exact arithmetic CG reaches the solution within N steps (Sec. 2.3)."""
    N = 48
    X = _points(N, 2, seed=15)
    hyp = _hyp("matern32", 2, ls=0.7, s2=0.1)
    Kt = O.ktilde_dense(X, hyp)
    b = np.random.default_rng(16).standard_normal(N)
    pre = None
    if rank:
        L, _ = O.pivoted_cholesky(X, hyp, rank)
        pre = lambda r: O.precond_apply(L, hyp.noise, r)  # noqa: E731
    res = O.cg_stable(lambda v: Kt @ v, b, precond=pre, tol=1e-11, max_iter=N, reorth=reorth)
    assert res.iters <= N
    np.testing.assert_allclose(res.x, np.linalg.solve(Kt, b), rtol=1e-7, atol=1e-8)


def test_standard_and_stable_cg_agree_without_reorth():
    N = 40
    X = _points(N, 3, seed=17)
    hyp = _hyp("rbf", 3, ls=1.0, s2=0.5)
    Kt = O.ktilde_dense(X, hyp)
    L, _ = O.pivoted_cholesky(X, hyp, 4)
    pre = lambda r: O.precond_apply(L, hyp.noise, r)  # noqa: E731
    b = np.random.default_rng(18).standard_normal(N)
    a = O.cg_standard(lambda v: Kt @ v, b, precond=pre, tol=1e-6)
    s = O.cg_stable(lambda v: Kt @ v, b, precond=pre, tol=1e-6, reorth="none")
    # LSE reaches the same scalars through log/exp, so they differ only by
    # rounding, which CG amplifies slowly over the iterations.
    assert a.iters == s.iters
    np.testing.assert_allclose(a.alphas, s.alphas, rtol=1e-7)
    np.testing.assert_allclose(a.betas, s.betas, rtol=1e-7)
    np.testing.assert_allclose(a.x, s.x, rtol=1e-8, atol=1e-10)


def test_reorth_forms_coincide_without_preconditioner():
    N = 36
    X = _points(N, 2, seed=19)
    hyp = _hyp("rbf", 2, ls=0.6, s2=0.05)
    Kt = O.ktilde_dense(X, hyp)
    b = np.random.default_rng(20).standard_normal(N)
    e = O.cg_stable(lambda v: Kt @ v, b, tol=1e-9, reorth="euclid")
    p = O.cg_stable(lambda v: Kt @ v, b, tol=1e-9, reorth="pinv")
    assert e.iters == p.iters
    np.testing.assert_allclose(e.x, p.x, rtol=1e-9, atol=1e-11)


# --- Lanczos / SLQ -----------------------------------------------------------

@pytest.mark.parametrize("rank", [0, 4])
def test_slq_full_lanczos_unit_probes_is_exact(rank):
    """Probes w_j = sqrt(N) e_j through P^{1/2} and N Lanczos steps: the SLQ estimate of
    log|P^{-1} Ktilde| is exact, so logdet P + SLQ = log|Ktilde|."""
    N = 24
    X = _points(N, 2, seed=21)
    hyp = _hyp("matern32", 2, ls=0.8, s2=0.2)
    Kt = O.ktilde_dense(X, hyp)
    if rank:
        L, _ = O.pivoted_cholesky(X, hyp, rank)
        pre = lambda r: O.precond_apply(L, hyp.noise, r)  # noqa: E731
        P = L @ L.T + hyp.noise * np.eye(N)
        ldP = O.precond_logdet(L, hyp.noise)
    else:
        pre, P, ldP = None, np.eye(N), 0.0
    w, Q = np.linalg.eigh(P)
    Phalf = (Q * np.sqrt(w)) @ Q.T
    est = 0.0
    for j in range(N):
        z = math.sqrt(N) * Phalf[:, j]
        res = O.cg_stable(lambda v: Kt @ v, z, precond=pre, tol=0.0, max_iter=N, reorth="pinv")
        T = O.lanczos_tridiagonal(res.alphas, res.betas)
        est += O.slq_quadrature(T, res.gamma0) / N
    assert abs(ldP + est - O.logdet_exact(X, hyp)) < 1e-7 * abs(O.logdet_exact(X, hyp))


def test_lanczos_tridiagonal_spectrum():
    """With N steps the Ritz values are the eigenvalues of the (preconditioned) matrix."""
    N = 20
    X = _points(N, 2, seed=22)
    hyp = _hyp("rbf", 2, ls=0.9, s2=0.3)
    Kt = O.ktilde_dense(X, hyp)
    b = np.random.default_rng(23).standard_normal(N)
    res = O.cg_stable(lambda v: Kt @ v, b, tol=0.0, max_iter=N, reorth="pinv")
    T = O.lanczos_tridiagonal(res.alphas, res.betas)
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(T)), np.sort(np.linalg.eigvalsh(Kt)), rtol=1e-8)


# --- finite support (Sec. 3.1, App. C.1) ----------------------------------------

@pytest.mark.parametrize("kernel", ["rbf", "matern12", "matern32", "matern52"])
def test_max_distance_is_where_kernel_reaches_eps(kernel):
    for eps in (2.0 ** -10, 2.0 ** -14, 2.0 ** -24, 1e-38):
        for ls in (0.3, 1.0, 4.0):
            dmax = O.max_distance(kernel, ls, eps)
            assert abs(O.unit_kernel(np.array((dmax / ls) ** 2), kernel) - eps) < 1e-9 * eps


def test_max_distance_rq_and_periodic():
    eps, ls, alpha = 2.0 ** -14, 0.7, 5.0
    d = O.max_distance("rq", ls, eps, alpha=alpha)
    assert abs((1 + d * d / (2 * alpha * ls * ls)) ** (-alpha) - eps) < 1e-12
    p, lam = 2.0, 0.1
    d = O.max_distance("periodic", 1.0, eps, period=p, lam=lam)
    assert abs(math.exp(-(2 / lam) * math.sin(math.pi * d / p) ** 2) - eps) < 1e-12
    assert O.max_distance("periodic", 1.0, eps, lam=5.0) == math.inf


def test_max_distance_ordering():
    """App. C.1: Matern-3/2 and -5/2 supports lie between Matern-1/2 and RBF."""
    for eps in (2.0 ** -10, 2.0 ** -24):
        r = O.max_distance("rbf", 1.0, eps)
        m12 = O.max_distance("matern12", 1.0, eps)
        assert r < O.max_distance("matern52", 1.0, eps) < O.max_distance("matern32", 1.0, eps) < m12


def test_paper_support_example():
    """Sec. 3.1: d = 0.75 and the half-precision eps give the printed 9.24."""
    with open(os.path.join(GOLDEN, "support_example.json")) as f:
        g = json.load(f)
    # Matern-1/2 at lengthscale l has support -l log eps; it equals d at l = d / (-log eps),
    # whose inverse is the printed value.
    l_crit = g["d"] / -math.log(g["eps"])
    assert abs(O.max_distance("matern12", l_crit, g["eps"]) - g["d"]) < 1e-12
    assert round(1.0 / l_crit, g["printed_digits"]) == g["printed_value"]


def test_paper_float_format_numbers():
    with open(os.path.join(GOLDEN, "float_formats.json")) as f:
        g = json.load(f)
    assert abs(float(np.finfo(np.float32).max) - g["single_max"]) < 1e31
    assert abs(float(np.finfo(np.float32).tiny) - g["single_min_normal"]) < 1e-41
    assert abs(float(np.finfo(np.float16).tiny) - g["half_min_normal"]) < 1e-9
    assert abs(2.0 ** -24 - g["single_roundoff"]) < 1e-8


def test_mbcg_equals_alg1_column_by_column():
    """mBCG (App. A) runs Alg. 1 per column with per-column scalars: each
    column's step sizes equal cg_standard's while rounding (the summation order
    of the dot products differs) has not grown yet, the iteration counts agree
    to one step, and both reach the Cholesky solution."""
    rng = np.random.default_rng(31)
    X = rng.standard_normal((120, 3))
    h = O.Hyp("matern32", np.array([0.9, 1.2, 0.7]), 1.1, 0.5)
    Kt = O.ktilde_dense(X, h)
    L, _ = O.pivoted_cholesky(X, h, 10)
    pre = lambda r: O.precond_apply(L, h.noise, r)   # noqa: E731
    B = rng.standard_normal((120, 4))
    B[:, 3] *= 1e-3                                    # scaled column: the same relative trajectory
    res = O.cg_mbcg(lambda V: Kt @ V, B, precond=pre, tol=1e-8, max_iter=200)
    exact = O.cholesky_solve(X, h, B)
    for c in range(4):
        ref = O.cg_standard(lambda v: Kt @ v, B[:, c], precond=pre, tol=1e-8, max_iter=200)
        assert abs(res[c].iters - ref.iters) <= 1
        np.testing.assert_allclose(res[c].alphas[:12], ref.alphas[:12], rtol=1e-9)
        np.testing.assert_allclose(res[c].betas[:12], ref.betas[:12], rtol=1e-9)
        assert abs(res[c].gamma0 - ref.gamma0) <= 1e-12 * abs(ref.gamma0)
        assert np.linalg.norm(res[c].x - exact[:, c]) <= 1e-6 * np.linalg.norm(exact[:, c])


# ---- MINRES (Conclusion: a further iterative method for the approach) -------------------

def _spd_problem(N=60, seed=0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((N, N))
    A = A @ A.T / N + 0.05 * np.eye(N)
    return A, rng.standard_normal(N)


@pytest.mark.parametrize("precond", [False, True])
def test_minres_iterates_match_the_library_routine(precond):
    """k steps of the oracle's MINRES equal k steps of scipy's MINRES (the
    library routine of the same method), with and without an SPD
    preconditioner (here P = diag(A): P^-1 applied as r / d)."""
    sla = pytest.importorskip("scipy.sparse.linalg")
    import inspect
    A, b = _spd_problem()
    d = np.diag(A).copy()
    kw = "rtol" if "rtol" in inspect.signature(sla.minres).parameters else "tol"
    M = sla.LinearOperator(A.shape, matvec=lambda r: r / d) if precond else None
    for k in (1, 4, 12, 30):
        res = O.minres(lambda v: A @ v, b, precond=(lambda r: r / d) if precond else None, tol=0.0, max_iter=k)
        xs, _ = sla.minres(A, b, M=M, maxiter=k, **{kw: 0.0})
        assert res.iters == k
        # rounding-order differences grow with k on this condition number (~100); a
        # wrong coefficient or sign shows at the 1e-2 level from the first steps
        assert np.linalg.norm(res.x - xs) <= (1e-12 if k < 10 else 1e-7) * np.linalg.norm(xs), k


@pytest.mark.parametrize("precond", [False, True])
def test_minres_minimises_the_preconditioned_residual_over_the_krylov_space(precond):
    """The defining property: x_k = argmin ||b - A x||_M over the Krylov space
    span{M b, (M A) M b, ..., (M A)^{k-1} M b}, M = P^-1 -- brute force by least
    squares on an orthonormal basis of that space, in the M inner product (M =
    G G^T, ||r||_M = ||G^T r||).  Also: the recurrence's phibar / beta_1 is that
    minimum relative to ||b||_M at every k."""
    A, b = _spd_problem(N=40, seed=3)
    Mm = np.diag(1.0 / np.diag(A)) if precond else np.eye(40)
    G = np.linalg.cholesky(Mm)
    for k in (1, 3, 6, 10):
        res = O.minres(lambda v: A @ v, b, precond=lambda r: Mm @ r, tol=0.0, max_iter=k)
        Kb = [Mm @ b]
        for _ in range(k - 1):
            Kb.append(Mm @ (A @ Kb[-1]))
        Q, _ = np.linalg.qr(np.array(Kb).T)
        c, *_ = np.linalg.lstsq(G.T @ A @ Q, G.T @ b, rcond=None)
        x_star = Q @ c
        assert np.linalg.norm(res.x - x_star) <= 1e-8 * np.linalg.norm(x_star), k
        r = b - A @ res.x
        rel = math.sqrt(r @ (Mm @ r)) / math.sqrt(b @ (Mm @ b))
        assert abs(res.resid_p[-1] - rel) <= 1e-10, (k, res.resid_p[-1], rel)


def test_minres_finite_termination_and_monotone_residual():
    """In exact arithmetic MINRES solves an N x N SPD system in at most N
    steps; its P^-1-norm residual never increases (it minimises over growing
    spaces).  Small N, FP64: the exact solution to 1e-10."""
    A, b = _spd_problem(N=25, seed=5)
    res = O.minres(lambda v: A @ v, b, tol=1e-13, max_iter=200)
    x = np.linalg.solve(A, b)
    assert np.linalg.norm(res.x - x) <= 1e-9 * np.linalg.norm(x)
    assert all(r1 <= r0 * (1 + 1e-12) for r0, r1 in zip(res.resid_p, res.resid_p[1:]))


def test_minres_on_the_gp_operator_with_the_woodbury_preconditioner():
    """The configuration the GPU path runs: Ktilde of a GP kernel, P the rank-k
    pivoted-Cholesky preconditioner applied by Eq. woodbury; the solution
    converges to the Cholesky solve and the recurrence's norm matches the
    recomputed P^-1-norm residual."""
    rng = np.random.default_rng(7)
    X = rng.standard_normal((300, 3))
    hyp = O.Hyp("rbf", np.array([0.9, 1.1, 1.0]), 1.2, 0.05)
    Kt = O.ktilde_dense(X, hyp)
    L, _ = O.pivoted_cholesky(X, hyp, 20)
    b = rng.standard_normal(300)
    P = lambda r: O.precond_apply(L, hyp.noise, r)
    res = O.minres(lambda v: Kt @ v, b, precond=P, tol=1e-10, max_iter=300)
    x = O.cholesky_solve(X, hyp, b[:, None])[:, 0]
    assert np.linalg.norm(res.x - x) <= 1e-7 * np.linalg.norm(x)
    r = b - Kt @ res.x
    assert abs(math.sqrt(r @ P(r)) / math.sqrt(b @ P(b)) - res.resid_p[-1]) <= 1e-9
