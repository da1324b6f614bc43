"""Pivoted-Cholesky preconditioner (gp_pivchol_precond) and CG (gp_cg_solve,
Alg. 1 / Alg. 2) on the GPU against the FP64 oracle.

Solves are judged by their FP64-recomputed relative residual
||Ktilde U - B|| / ||B|| per column (the trajectory itself is not pinned)."""

import math

import numpy as np
import pytest

import oracle as O
from paper_2207_06856_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
KNAME = {0: "rbf", 1: "matern32", 2: "matern12", 3: "matern52"}


@pytest.fixture(scope="module")
def ctx():
    from paper_2207_06856_gb300 import gpk
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = gpk.Context(0)
    yield c
    c.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _ohyp(w):
    return O.Hyp(KNAME[w.kernel], w.lengthscale, w.outputscale, w.noise)


def test_pivchol_invariants(ctx):
    from paper_2207_06856_gb300 import gpk
    X, _, kern, ls, a2, s2 = workloads.random_problem(1500, 5, 1, seed=21, kernel=1)
    hyp = gpk.Hyper(kern, ls, a2, s2)
    pc = gpk.pivchol(ctx, hyp, _dev(X), 30)
    ctx.check()
    assert pc.rank == 30
    L = pc.L.cpu().numpy().astype(np.float64).T          # N x k
    piv = pc.piv.cpu().numpy()
    oh = O.Hyp("matern32", ls, a2, s2)
    K = O.kernel_matrix(X, X, oh)
    assert piv[0] == 0 and len(set(piv.tolist())) == 30
    # interpolation: (L L^T)[p, :] = K[p, :] for the pivots (FP32 rows)
    assert np.max(np.abs((L @ L.T)[piv] - K[piv])) < 2e-4 * a2
    rem = np.diag(K) - np.sum(L * L, axis=1)
    assert rem.min() > -1e-4
    # the first pivots agree with the FP64 oracle (later ones may swap on near-ties)
    _, opiv = O.pivoted_cholesky(X, oh, 8)
    assert list(piv[:8]) == list(opiv[:8])
    # core: lower Cholesky factor of I + L^T L / sigma^2, in FP64
    Lc = pc.core.cpu().numpy().T
    C = np.eye(30) + (L.T @ L) / s2
    np.testing.assert_allclose(Lc @ Lc.T, C, rtol=1e-5, atol=1e-5 * np.abs(C).max())


@pytest.mark.parametrize("alg", ["stable", "standard"])
def test_plain_config_fp32(ctx, alg):
    """Plain workload: N = 2048, d = 8, RBF l = 0.5, sigma^2 = 0.01, rank 20,
    tol 1e-4, FP32 on the GPU vs the FP64 oracle."""
    from paper_2207_06856_gb300 import gpk
    w = workloads.plain()
    hyp = gpk.Hyper(w.kernel, w.lengthscale, w.outputscale, w.noise)
    X = _dev(w.X)
    pc = gpk.pivchol(ctx, hyp, X, w.rank)
    B = w.rhs()
    U, st, info = gpk.cg_solve(ctx, hyp, X, _dev(B), pc, tol=w.tol, max_iter=w.max_iter, precision="fp32",
                               algorithm=alg, reorth="pinv" if alg == "stable" else "none", restarts=4)
    ctx.check()
    assert st == gpk.GP_OK, info
    res = O.relative_residual(w.X, U.cpu().numpy().T, B.T, _ohyp(w))
    assert res.max() <= w.tol, res
    ref = O.cholesky_solve(w.X, _ohyp(w), B.T.astype(np.float64))
    err = np.linalg.norm(U.cpu().numpy().T - ref) / np.linalg.norm(ref)
    assert err < 1e-2


@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp32"])
@pytest.mark.parametrize("kern", [0, 1])
def test_stable_cg_precision_workload_small(ctx, prec, kern):
    """The precision workload at N = 6000 (1 + 16 RHS, rank 100 preconditioner):
    the FP64 residual of every column is <= 1e-2."""
    from paper_2207_06856_gb300 import gpk
    w = workloads.precision(N=6000, kernel=kern)
    hyp = gpk.Hyper(w.kernel, w.lengthscale, w.outputscale, w.noise)
    X = _dev(w.X)
    pc = gpk.pivchol(ctx, hyp, X, w.rank)
    B = w.rhs()
    U, st, info = gpk.cg_solve(ctx, hyp, X, _dev(B), pc, tol=w.tol, max_iter=400, precision=prec)
    ctx.check()
    assert st == gpk.GP_OK, (info["col_iters"], info["rel_resid"])
    res = O.relative_residual(w.X, U.cpu().numpy().T, B.T, _ohyp(w))
    assert res.max() <= w.tol, res


def test_reorth_modes_and_standard_agree_on_small_problem(ctx):
    """All variants reach the same solution on a well-conditioned small problem."""
    from paper_2207_06856_gb300 import gpk
    X, V, kern, ls, a2, s2 = workloads.random_problem(900, 4, 3, seed=22, noise=0.1)
    hyp = gpk.Hyper(kern, ls, a2, s2)
    Xd, Bd = _dev(X), _dev(V)
    pc = gpk.pivchol(ctx, hyp, Xd, 10)
    ref = O.cholesky_solve(X, O.Hyp("rbf", ls, a2, s2), V.T.astype(np.float64))
    for alg, ro, pre in [("stable", "pinv", pc), ("stable", "euclid", None), ("stable", "none", pc),
                         ("standard", "none", pc), ("stable", "pinv", None)]:
        U, st, info = gpk.cg_solve(ctx, hyp, Xd, Bd, pre, tol=1e-6, max_iter=300, precision="fp32", algorithm=alg,
                                   reorth=ro, reorth_passes=2)
        ctx.check()
        assert st == gpk.GP_OK, (alg, ro, info["rel_resid"])
        err = np.linalg.norm(U.cpu().numpy().T - ref) / np.linalg.norm(ref)
        assert err < 1e-4, (alg, ro, err)


def test_cg_trajectory_matches_oracle_alg2(ctx):
    """Parity unpinned beyond the solution, but in FP32 the first step sizes of
    Alg. 2 follow the FP64 oracle's closely."""
    from paper_2207_06856_gb300 import gpk
    X, V, kern, ls, a2, s2 = workloads.random_problem(700, 3, 1, seed=23, noise=0.05)
    hyp = gpk.Hyper(kern, ls, a2, s2)
    Xd = _dev(X)
    pc = gpk.pivchol(ctx, hyp, Xd, 8)
    U, st, info = gpk.cg_solve(ctx, hyp, Xd, _dev(V), pc, tol=1e-5, max_iter=100, precision="fp32", restarts=0)
    oh = O.Hyp("rbf", ls, a2, s2)
    piv_np = pc.piv.cpu().numpy()
    L64, _ = O.pivoted_cholesky(X, oh, 8)
    Kt = O.ktilde_dense(X, oh)
    ores = O.cg_stable(lambda v: Kt @ v, V[0].astype(np.float64),
                       precond=lambda r: O.precond_apply(L64, s2, r), tol=1e-5, max_iter=100)
    assert list(piv_np) == list(O.pivoted_cholesky(X, oh, 8)[1])
    n = min(5, len(ores.alphas), info["alpha"].shape[0])
    np.testing.assert_allclose(info["alpha"][:n, 0], ores.alphas[:n], rtol=1e-3)
    np.testing.assert_allclose(info["beta"][:n, 0], ores.betas[:n], rtol=1e-2)
    assert abs(info["iters"] - ores.iters) <= 3
    assert abs(info["gamma0"][0] - ores.gamma0) < 1e-4 * ores.gamma0


def test_cg_edge_cases(ctx):
    from paper_2207_06856_gb300 import gpk
    # N = 1: Ktilde = a^2 + sigma^2, one step solves it
    hyp = gpk.Hyper(0, np.ones(2), 1.5, 0.5)
    X = _dev(np.zeros((1, 2), np.float32))
    B = _dev(np.array([[3.0]], np.float32))
    U, st, info = gpk.cg_solve(ctx, hyp, X, B, None, tol=1e-6, max_iter=5, precision="fp16")
    assert st == gpk.GP_OK
    assert abs(U.item() - 3.0 / 2.0) < 1e-5
    # zero right-hand side: nothing to do, U = 0
    Xn, V, kern, ls, a2, s2 = workloads.random_problem(500, 3, 2, seed=24)
    V[1] = 0.0
    hyp = gpk.Hyper(kern, ls, a2, s2)
    U, st, info = gpk.cg_solve(ctx, hyp, _dev(Xn), _dev(V), None, tol=1e-3, max_iter=100, precision="fp32")
    assert np.all(U.cpu().numpy()[1] == 0.0)
    # max_iter reached -> NOT_CONVERGED, iterate still returned
    U, st, info = gpk.cg_solve(ctx, hyp, _dev(Xn), _dev(V[:1]), None, tol=1e-12, max_iter=2, precision="fp32")
    assert st == gpk.GP_ERR_NOT_CONVERGED and info["iters"] == 2
    # warm start from the solution: converged before the first step
    ref = O.cholesky_solve(Xn, O.Hyp("rbf", ls, a2, s2), V[:1].T.astype(np.float64)).T.astype(np.float32)
    U0 = _dev(ref)
    U, st, info = gpk.cg_solve(ctx, hyp, _dev(Xn), _dev(V[:1]), None, tol=1e-4, max_iter=10, precision="fp32", U=U0)
    assert st == gpk.GP_OK and info["iters"] <= 1
    ctx.check()


STOP_MARGIN = 0.01   # the benchmark's margin under 1e-2 for the FP32 check's rounding


def test_precision_workload_full_size_fp16(ctx):
    """The benchmark solve: N = 65,536, d = 8, RBF, 1 + 16 RHS, rank-100
    preconditioner, FP16 tensor-core MVM, stable CG stopped at 0.99e-2 on its
    FP32 true-residual check.

    The residual ||Ktilde U - B|| / ||B|| is recomputed in FP64 over all
    65,536 rows (the oracle's multi-threaded matrix-free MVM) and must be
    <= 1e-2 for every column: the 1 % margin covers the FP32 check's rounding,
    about 2^-24 kappa / sqrt(N) = 3.4e-6 of ||b|| with kappa = || |K| |x| || /
    ||b|| ~ 1.5e4 (sum_j |k_ij x_j| rather than |(Ktilde x)_i| sets it)."""
    from oracle import cfp64 as C
    from paper_2207_06856_gb300 import gpk
    w = workloads.precision()
    hyp = gpk.Hyper(w.kernel, w.lengthscale, w.outputscale, w.noise)
    X = _dev(w.X)
    pc = gpk.pivchol(ctx, hyp, X, w.rank)
    B = w.rhs()
    U, st, info = gpk.cg_solve(ctx, hyp, X, _dev(B), pc, tol=w.tol * (1.0 - STOP_MARGIN), max_iter=w.max_iter,
                               precision="fp16")
    ctx.check()
    assert st == gpk.GP_OK, (info["col_iters"], info["rel_resid"])
    reported = np.asarray(info["rel_resid"])
    assert reported.max() <= w.tol * (1.0 - STOP_MARGIN), reported
    full = C.relative_residual(w.X, U.cpu().numpy().T, B.T, _ohyp(w))
    assert full.max() <= w.tol, full
    assert np.all(np.abs(full - reported) <= STOP_MARGIN * w.tol), (full, reported)


def test_breakdown_escalates_to_check_precision(ctx):
    """N = 20,000 points in d = 2, RBF l = 0.5, sigma^2 = 1e-4, single-term FP16
    inputs: the FP16 operator is not positive definite to the accuracy the solve
    needs, so CG breaks down; with escalation (the default) the restart continues
    with the FP32 check MVM and the solve converges by that MVM.  At this
    conditioning |x| ~ |y| / sigma^2, and the FP32 check's rounding (proportional
    to sum_j |k_ij x_j|) resolves the residual only to a few 1e-2: the FP64
    residual is checked against 5e-2."""
    from paper_2207_06856_gb300 import gpk
    rng = np.random.default_rng(0)
    N, d = 20000, 2
    X = rng.standard_normal((N, d)).astype(np.float32)
    y = (np.sin(2 * np.pi * X.mean(1)) + 0.1 * rng.standard_normal(N)).astype(np.float32)
    hyp = gpk.Hyper(gpk.RBF, np.full(d, 0.5, np.float32), 1.0, 1e-4)
    Xd, B = _dev(X), _dev(y[None])
    pc = gpk.pivchol(ctx, hyp, Xd, 20)
    _, st0, info0 = gpk.cg_solve(ctx, hyp, Xd, B, pc, tol=1e-2, max_iter=1000, precision="fp16",
                                 flags=gpk.MVM_NO_XSPLIT, escalate=False)
    assert st0 == gpk.GP_ERR_BREAKDOWN and info0["breakdowns"] >= 1
    U, st1, info1 = gpk.cg_solve(ctx, hyp, Xd, B, pc, tol=1e-2, max_iter=1000, precision="fp16",
                                 flags=gpk.MVM_NO_XSPLIT, escalate=True)
    assert st1 == gpk.GP_OK and info1["escalated"] == 1, info1["rel_resid"]
    rows = np.sort(np.random.default_rng(1).choice(N, 2048, replace=False))
    oh = O.Hyp("rbf", np.full(d, 0.5), 1.0, 1e-4)
    r = O.kmvm_rows(X, rows, U.cpu().numpy().T.astype(np.float64), oh)[:, 0] - y[rows]
    est = np.sqrt(N / len(rows) * np.sum(r * r)) / np.linalg.norm(y.astype(np.float64))
    assert est <= 5e-2, est


def test_split_fp16_solve_needs_fp32_iteration_count(ctx):
    """FP16 tensor-core MVM with the kernel tile and inputs carried as hi + lo:
    the stable CG needs at most 15 % more iterations than FP32 on the precision
    workload's distribution (N = 16,384), and its residual is verified in FP64."""
    from paper_2207_06856_gb300 import gpk
    w = workloads.precision(N=16384)
    hyp = gpk.Hyper(w.kernel, w.lengthscale, w.outputscale, w.noise)
    X, B = _dev(w.X), _dev(w.rhs())
    pc = gpk.pivchol(ctx, hyp, X, w.rank)
    _, st32, i32 = gpk.cg_solve(ctx, hyp, X, B, pc, tol=w.tol, max_iter=w.max_iter, precision="fp32")
    U, st16, i16 = gpk.cg_solve(ctx, hyp, X, B, pc, tol=w.tol, max_iter=w.max_iter, precision="fp16",
                                flags=gpk.MVM_PSPLIT | gpk.MVM_XSPLIT)
    assert st32 == gpk.GP_OK and st16 == gpk.GP_OK
    assert i16["iters"] <= 1.15 * i32["iters"], (i16["iters"], i32["iters"])
    rows = np.sort(np.random.default_rng(3).choice(w.N, 2048, replace=False))
    Bt = w.rhs().T.astype(np.float64)
    r = O.kmvm_rows(w.X, rows, U.cpu().numpy().T, _ohyp(w), add_noise=True) - Bt[rows]
    est = np.sqrt(w.N / len(rows) * np.sum(r * r, axis=0)) / np.linalg.norm(Bt, axis=0)
    assert est.max() <= 1.15 * w.tol, est


def test_precision_workload_full_size_relaxed_schedule(ctx):
    """The benchmark's solve with its relaxed MVM schedule: the FP16 MVM with the
    kernel tile and inputs as hi + lo until every column's recursive residual is
    <= 0.3 (30 x tol), the single-rounded FP16 MVM after.  The FP64 residual over
    all 65,536 rows must be <= 1e-2 for every column, and the schedule must need
    fewer iterations than the single-rounded MVM throughout (the accurate early
    MVMs keep the true residual close to the recursive one)."""
    from oracle import cfp64 as C
    from paper_2207_06856_gb300 import gpk
    w = workloads.precision()
    hyp = gpk.Hyper(w.kernel, w.lengthscale, w.outputscale, w.noise)
    X = _dev(w.X)
    pc = gpk.pivchol(ctx, hyp, X, w.rank)
    B = w.rhs()
    tol = w.tol * (1.0 - STOP_MARGIN)
    U, st, info = gpk.cg_solve(ctx, hyp, X, _dev(B), pc, tol=tol, max_iter=w.max_iter,
                               precision=gpk.FP16 | gpk.MVM_PSPLIT | gpk.MVM_XSPLIT, refine_precision="fp16",
                               refine_resid=30.0 * w.tol)
    _, st1, info1 = gpk.cg_solve(ctx, hyp, X, _dev(B), pc, tol=tol, max_iter=w.max_iter, precision="fp16")
    ctx.check()
    assert st == gpk.GP_OK and st1 == gpk.GP_OK
    assert info["iters"] < info1["iters"], (info["iters"], info1["iters"])
    full = C.relative_residual(w.X, U.cpu().numpy().T, B.T, _ohyp(w))
    assert full.max() <= w.tol, full


def test_refine_switch_points(ctx):
    """refine_resid above every residual switches before the first iteration,
    so the solve is bit-identical to one on the refine MVM alone; below every
    residual it never switches (bit-identical to the solve's own MVM); in
    between the trajectory starts like the first and differs later.  Invalid
    switch settings are refused."""
    from paper_2207_06856_gb300 import gpk
    w = workloads.precision(N=6000)
    hyp = gpk.Hyper(w.kernel, w.lengthscale, w.outputscale, w.noise)
    X, B = _dev(w.X), _dev(w.rhs())
    pc = gpk.pivchol(ctx, hyp, X, w.rank)
    split = gpk.FP16 | gpk.MVM_PSPLIT | gpk.MVM_XSPLIT
    kw = dict(tol=w.tol, max_iter=w.max_iter)
    Ua, _, ia = gpk.cg_solve(ctx, hyp, X, B, pc, precision=split, **kw)
    Ub, _, ib = gpk.cg_solve(ctx, hyp, X, B, pc, precision="fp16", **kw)
    Uhi, _, ihi = gpk.cg_solve(ctx, hyp, X, B, pc, precision=split, refine_precision="fp16", refine_resid=1e30, **kw)
    Ulo, _, ilo = gpk.cg_solve(ctx, hyp, X, B, pc, precision=split, refine_precision="fp16", refine_resid=1e-30,
                               **kw)
    Umid, _, imid = gpk.cg_solve(ctx, hyp, X, B, pc, precision=split, refine_precision="fp16", refine_resid=0.3,
                                 **kw)
    assert torch.equal(Uhi, Ub) and np.array_equal(ihi["alpha"], ib["alpha"])
    assert torch.equal(Ulo, Ua) and np.array_equal(ilo["alpha"], ia["alpha"])
    k = int(np.argmax(np.max(ia["resid_hist"], axis=1) <= 0.3))   # first iterate at or below the switch point
    assert k > 1
    assert np.array_equal(imid["alpha"][:k], ia["alpha"][:k])
    assert not np.array_equal(imid["alpha"], ia["alpha"][:len(imid["alpha"])])
    with pytest.raises(gpk.GPKError):
        gpk.cg_solve(ctx, hyp, X, B, pc, precision=split, refine_precision="fp16", refine_resid=-1.0, **kw)
    with pytest.raises(gpk.GPKError):
        gpk.cg_solve(ctx, hyp, X, B, pc, precision=split, refine_precision="fp16", refine_resid=0.0, restarts=0,
                     **kw)
