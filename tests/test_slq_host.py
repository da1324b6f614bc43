"""gp_slq_quadrature (host-side Lanczos quadrature of the library) against the
FP64 oracle.  CPU only: the function needs no GPU."""

import math

import numpy as np
import pytest

import oracle as O


@pytest.fixture(scope="module")
def gpk():
    from paper_2207_06856_gb300 import build, gpk as g
    import os
    if not os.path.exists(g.LIB_PATH):
        build.build()
    return g


def _cg_coeffs(N, seed, J=None, noise=0.1):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((N, 3))
    hyp = O.Hyp("matern32", np.ones(3), 1.2, noise)
    Kt = O.ktilde_dense(X, hyp)
    z = rng.standard_normal(N)
    res = O.cg_stable(lambda v: Kt @ v, z, tol=0.0, max_iter=J or N, reorth="pinv")
    return Kt, z, res


@pytest.mark.parametrize("seed,J", [(0, 5), (1, 12), (2, 30), (3, 40)])
def test_slq_matches_oracle_quadrature(gpk, seed, J):
    _, _, res = _cg_coeffs(40, seed, J=J)
    T = O.lanczos_tridiagonal(res.alphas, res.betas)
    ref = O.slq_quadrature(T, res.gamma0)
    got = gpk.slq_quadrature(res.alphas, res.betas[:len(res.alphas) - 1], res.gamma0)
    assert abs(got - ref) <= 1e-10 * max(1.0, abs(ref))


def test_slq_full_lanczos_is_exact_quadratic_form(gpk):
    """With N steps the Gauss quadrature is exact: z^T log(K) z."""
    Kt, z, res = _cg_coeffs(30, 7)
    w, Q = np.linalg.eigh(Kt)
    exact = float(z @ (Q * np.log(w)) @ Q.T @ z)
    got = gpk.slq_quadrature(res.alphas, res.betas[:len(res.alphas) - 1], res.gamma0)
    assert abs(got - exact) <= 1e-8 * abs(exact)


def test_slq_single_step_and_errors(gpk):
    # J = 1: T = [1/alpha_0], quadrature = gamma0 log(1/alpha_0)
    assert abs(gpk.slq_quadrature([0.25], [], 3.0) - 3.0 * math.log(4.0)) < 1e-14
    with pytest.raises(gpk.GPKError):
        gpk.slq_quadrature([0.5, -0.1], [0.2], 1.0)
