"""Pins of the multi-threaded FP64 oracle routines (oracle/fp64_cg.c).

They are checked against the numpy oracle (itself pinned in
test_oracle_pins.py) and against facts that hold independently of either:
the rank-one and far-apart limits of the kernel matrix (Eq. mvm), exact
solves by Cholesky (Sec. 2.2), the one-step convergence of CG when the
pivoted-Cholesky preconditioner reaches full rank (Eq. woodbury: P = Ktilde),
and finite termination of CG (Alg. 1)."""

import numpy as np
import pytest

import oracle as O
from oracle import cfp64 as C


@pytest.fixture(scope="module", autouse=True)
def _built():
    C.build()


@pytest.mark.parametrize("kern", list(O.KERNELS))
def test_kmvm_equals_numpy_oracle(kern):
    rng = np.random.default_rng(1)
    X = rng.standard_normal((257, 6))
    V = rng.standard_normal((257, 5))
    h = O.Hyp(kern, rng.uniform(0.5, 2.0, 6), 1.3, 0.07)
    ref = O.kmvm(X, X, V, h, add_noise=True)
    got = C.kmvm(X, V, h)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    rows = np.array([0, 5, 100, 256])
    assert np.max(np.abs(C.kmvm(X, V, h, rows=rows) - ref[rows])) <= 1e-12 * np.max(np.abs(ref))
    no_noise = C.kmvm(X, V, h, add_noise=False)
    assert np.max(np.abs(no_noise + h.noise * V - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_kmvm_rank_one_limit():
    """l -> infinity: Ktilde v = a^2 (1^T v) 1 + sigma^2 v exactly in FP64."""
    rng = np.random.default_rng(2)
    X = rng.standard_normal((300, 3))
    V = rng.standard_normal((300, 2))
    h = O.Hyp("rbf", np.full(3, 1e9), 0.8, 0.3)
    ref = 0.8 * np.ones((300, 1)) * V.sum(axis=0, keepdims=True) + 0.3 * V
    assert np.allclose(C.kmvm(X, V, h), ref, rtol=1e-12, atol=1e-12)


def test_kmvm_far_apart_limit():
    """Points 50 lengthscales apart: Ktilde = (a^2 + sigma^2) I to exp(-1250)."""
    g = np.arange(5.0)
    X = np.stack(np.meshgrid(g, g, indexing="ij"), -1).reshape(-1, 2) * 50.0
    V = np.random.default_rng(3).standard_normal((25, 3))
    h = O.Hyp("matern12", np.ones(2), 1.5, 0.2)
    assert np.allclose(C.kmvm(X, V, h), 1.7 * V, rtol=1e-12, atol=1e-300)


def test_pcg_reaches_cholesky_solution():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((400, 4))
    h = O.Hyp("rbf", np.ones(4), 1.0, 0.05)
    B = rng.standard_normal((400, 3))
    ref = O.cholesky_solve(X, h, B)
    for L in (None, C.preconditioner(X, h, 20)):
        U, it, rel, _ = C.pcg(X, B, h, L=L, tol=1e-11, max_iter=400)
        assert np.all(rel <= 1e-11) and it < 400
        assert np.max(np.abs(U - ref)) <= 1e-8 * np.max(np.abs(ref))
        assert np.all(C.relative_residual(X, U, B, h) <= 1e-10)


def test_pcg_full_rank_preconditioner_is_exact():
    """At rank N the pivoted Cholesky factor reproduces K, so P = Ktilde and
    one CG step solves the system (Eq. woodbury)."""
    rng = np.random.default_rng(5)
    X = rng.standard_normal((60, 2))
    h = O.Hyp("matern32", np.array([0.7, 1.3]), 1.1, 0.1)
    L = C.preconditioner(X, h, 60)
    B = rng.standard_normal((60, 2))
    U, it, rel, _ = C.pcg(X, B, h, L=L, tol=1e-9, max_iter=5)
    assert it == 1
    assert np.max(np.abs(U - O.cholesky_solve(X, h, B))) <= 1e-7


def test_pcg_finite_termination():
    """Exact-arithmetic CG ends within N steps; in FP64 on a well-conditioned
    N = 40 system it reaches 1e-10 within N iterations (Alg. 1)."""
    rng = np.random.default_rng(6)
    X = rng.standard_normal((40, 3))
    h = O.Hyp("rbf", np.full(3, 1.5), 1.0, 0.5)
    B = rng.standard_normal((40, 1))
    U, it, rel, _ = C.pcg(X, B, h, tol=1e-10, max_iter=40)
    assert it <= 40 and rel[0] <= 1e-10


def test_pcg_iteration_budget_and_time_limit():
    rng = np.random.default_rng(7)
    X = rng.standard_normal((200, 3))
    h = O.Hyp("rbf", np.ones(3), 1.0, 0.01)
    B = rng.standard_normal((200, 2))
    U, it, rel, spi = C.pcg(X, B, h, tol=0.0, max_iter=3)
    assert it == 3 and spi > 0.0 and np.all(rel > 0.0)
    U, it, rel, spi = C.pcg(X, B, h, tol=0.0, max_iter=1000, time_limit_s=1e-9)
    assert it == 1   # the limit is checked after the first iteration


def test_invalid_arguments_are_refused():
    X = np.zeros((4, 2))
    V = np.zeros((4, 1))
    with pytest.raises(RuntimeError):
        C.kmvm(X, np.zeros((4, 0)), O.Hyp("rbf", np.ones(2)))
    assert C.threads() >= 1
    _ = C.kmvm(X, V, O.Hyp("rbf", np.ones(2)))


@pytest.mark.parametrize("kern", list(O.KERNELS))
def test_quad_form_grad_equals_numpy_oracle(kern):
    rng = np.random.default_rng(8)
    X = rng.standard_normal((150, 4))
    U = rng.standard_normal((150, 3))
    V = rng.standard_normal((150, 3))
    h = O.Hyp(kern, rng.uniform(0.6, 1.8, 4), 1.2, 0.09)
    ref, refX = O.quad_form_grad(X, h, U, V, wrt_X=True)
    g, gX = C.quad_form_grad(X, h, U, V, wrt_X=True)
    assert np.max(np.abs(g - ref)) <= 1e-10 * np.max(np.abs(ref))
    assert np.max(np.abs(gX - refX)) <= 1e-10 * np.max(np.abs(refX))
    Z = rng.standard_normal((150, 2))
    Uf = rng.standard_normal((150, 3))
    a = C.pseudo_loss_grad(X, h, Uf, Z)
    b = O.pseudo_loss_grad(X, h, Uf, Z)
    assert np.max(np.abs(a - b)) <= 1e-10 * np.max(np.abs(b))


def test_quad_form_grad_finite_differences():
    """d/da^2 and d/dl_m of u^T Ktilde v by central differences of the C MVM."""
    rng = np.random.default_rng(9)
    X = rng.standard_normal((120, 3))
    u = rng.standard_normal((120, 1))
    v = rng.standard_normal((120, 1))
    ls = np.array([0.8, 1.1, 1.5])
    h = O.Hyp("matern52", ls, 1.3, 0.1)
    g, _ = C.quad_form_grad(X, h, u, v)
    q = lambda hh: float(u[:, 0] @ C.kmvm(X, v, hh)[:, 0])   # noqa: E731
    eps = 1e-6
    for m in range(3):
        lp, lm = ls.copy(), ls.copy()
        lp[m] += eps
        lm[m] -= eps
        fd = (q(O.Hyp("matern52", lp, 1.3, 0.1)) - q(O.Hyp("matern52", lm, 1.3, 0.1))) / (2 * eps)
        assert abs(fd - g[m]) <= 1e-6 * max(1.0, abs(fd))
    fd = (q(O.Hyp("matern52", ls, 1.3 + eps, 0.1)) - q(O.Hyp("matern52", ls, 1.3 - eps, 0.1))) / (2 * eps)
    assert abs(fd - g[3]) <= 1e-6 * max(1.0, abs(fd))
    fd = (q(O.Hyp("matern52", ls, 1.3, 0.1 + eps)) - q(O.Hyp("matern52", ls, 1.3, 0.1 - eps))) / (2 * eps)
    assert abs(fd - g[4]) <= 1e-6 * max(1.0, abs(fd))
