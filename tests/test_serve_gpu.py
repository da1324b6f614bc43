"""Serving with continuous batching (gp_server_*): predictive means against the
FP64 oracle, the same result alone and in a mix, the arena budget, and
admission of requests that arrive while others are in flight."""

import numpy as np
import pytest

import oracle as O
from paper_2207_06856_gb300 import workloads

torch = pytest.importorskip("torch")
KNAME = {0: "rbf", 1: "matern32", 2: "matern12", 3: "matern52"}


def _requests(n, seed, n_min=300, n_max=3000, n_test=256):
    """Small serving requests with the serving workload's distributions."""
    reqs = workloads.serving(n_requests=n, rate_per_s=100.0, seed=seed, n_min=n_min, n_max=n_max, n_test=n_test)
    return reqs


def _hyp(gpk, r):
    return gpk.Hyper(r.kernel, r.lengthscale, r.outputscale, r.noise)


def _ohyp(r):
    return O.Hyp(KNAME[r.kernel], r.lengthscale.astype(np.float64), r.outputscale, r.noise)


@pytest.fixture(scope="module")
def gpk():
    from paper_2207_06856_gb300 import gpk as g
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return g


@pytest.mark.gpu
def test_serve_fp32_matches_exact_posterior_mean(gpk):
    """FP32 MVMs, CG to 1e-6: mu* = K(X*, X) Ktilde^{-1} y against the oracle's
    Cholesky solve, within the first-order perturbation bound of FP32
    arithmetic alone: mu - mu_exact = K* Ktilde^{-1} r_true + dK* v with
    ||r_true|| <= rel_resid ||y|| + ||dKtilde v||, and each FP32 MVM errs by at
    most EPS32 = 1e-5 of its result (the FP32 MVM tolerance the MVM parity tests
    establish against the FP64 oracle).  Every norm is taken in FP64 from the
    oracle; nothing in the bound comes from the device.  Factor 2: the solver
    meets those errors at its iterates, not at v."""
    EPS32 = 1e-5
    srv = gpk.Server(0, arena_bytes=1 << 30, max_slots=4, rank=20, precision="fp32", mean_precision="fp32",
                     tol=1e-6, max_iter=600)
    try:
        reqs = _requests(6, seed=3)
        futs = [srv.submit(_hyp(gpk, r), r.X, r.y, r.Xstar) for r in reqs]
        for r, f in zip(reqs, futs):
            mean, st = f.result(timeout=120)
            assert st["status"] == gpk.GP_OK, st
            oh = _ohyp(r)
            Kt = O.ktilde_dense(r.X, oh)
            Ks = O.kernel_matrix(r.Xstar, r.X, oh)
            y = r.y.astype(np.float64)
            v = np.linalg.solve(Kt, y)
            ref = Ks @ v
            A = np.linalg.solve(Kt, Ks.T).T          # K* Ktilde^{-1} (Ktilde symmetric)
            bound = np.linalg.norm(A, 2) * (st["rel_resid"] * np.linalg.norm(y) + EPS32 * np.linalg.norm(Kt @ v)) \
                + EPS32 * np.linalg.norm(ref)
            err = np.linalg.norm(mean - ref)
            assert err <= 2.0 * bound, (r.rid, r.X.shape, err, bound)
    finally:
        srv.close()


@pytest.mark.gpu
@pytest.mark.parametrize("relaxed", [False, True])
def test_serve_fp16_within_cg_bound(gpk, relaxed):
    """The served configurations (S from hi + lo FP16 inputs on the tensor
    cores with the FP32 value product -- the default -- or that MVM until every
    residual is <= 0.3 and the single-rounded FP16 one after; CG to 1e-2,
    rank 20):
    the reported residual is <= 1e-2 and the mean is within the bound that
    residual implies: mu - mu_exact = K* Ktilde^{-1} r, so
    ||mu - mu_exact|| <= ||K* Ktilde^{-1}||_2 ||r||, ||r|| = rel_resid ||y||
    (the residual comes from the FP32 check MVM, so the FP16 MVM's error is
    inside it; the operator norm is taken in FP64)."""
    srv = gpk.Server(0, arena_bytes=1 << 30, max_slots=4, rank=20,
                     refine_precision="fp16" if relaxed else None, refine_resid=0.3 if relaxed else 0.0)
    try:
        reqs = _requests(6, seed=5)
        futs = [srv.submit(_hyp(gpk, r), r.X, r.y, r.Xstar) for r in reqs]
        for r, f in zip(reqs, futs):
            mean, st = f.result(timeout=120)
            assert st["status"] == gpk.GP_OK and st["rel_resid"] <= 1e-2, st
            oh = _ohyp(r)
            Kt = O.ktilde_dense(r.X, oh)
            Ks = O.kernel_matrix(r.Xstar, r.X, oh)
            y = r.y.astype(np.float64)
            ref = Ks @ np.linalg.solve(Kt, y)
            A = np.linalg.solve(Kt, Ks.T).T          # K* Ktilde^{-1} (Ktilde symmetric)
            bound = np.linalg.norm(A, 2) * st["rel_resid"] * np.linalg.norm(y)
            # 1.05: the residual is itself measured with an FP32 MVM
            assert np.linalg.norm(mean - ref) <= 1.05 * bound + 1e-5 * np.linalg.norm(ref), (r.rid, bound)
    finally:
        srv.close()


@pytest.mark.gpu
@pytest.mark.parametrize("large_n", [32768, 1500])
def test_same_result_alone_and_in_mix(gpk, large_n):
    """Each request served alone (one at a time) and in a mix of twelve with
    up to six in flight gives bit-identical means; the mix really overlapped.
    With large_n = 1500 the larger half of the requests plan their kernels for
    all but 16 SMs: still the same result alone and in the mix."""
    reqs = _requests(12, seed=7)
    srv = gpk.Server(0, arena_bytes=2 << 30, max_slots=6, rank=20, large_n=large_n, large_reserve=16)
    try:
        alone = []
        for r in reqs:
            alone.append(srv.submit(_hyp(gpk, r), r.X, r.y, r.Xstar).result(timeout=120)[0])
        futs = [srv.submit(_hyp(gpk, r), r.X, r.y, r.Xstar) for r in reqs]
        mix = [f.result(timeout=120) for f in futs]
        for a, (m, st) in zip(alone, mix):
            assert st["status"] == gpk.GP_OK
            np.testing.assert_array_equal(a, m)
        s = srv.stats()
        assert s["max_inflight"] > 1, s
        assert s["completed"] == 24
    finally:
        srv.close()


@pytest.mark.gpu
def test_arena_budget_never_exceeded(gpk):
    """An arena sized for two of the requests: every request completes, the
    peak use stays within the arena, at most two are in flight at once, and a
    request larger than the whole arena is refused at submit."""
    reqs = _requests(8, seed=11, n_min=2000, n_max=2500)
    probe = gpk.Server(0, arena_bytes=1 << 20, max_slots=1, rank=20)
    need = max(probe.request_bytes(_hyp(gpk, r), r.X.shape[0], r.Xstar.shape[0]) for r in reqs)
    probe.close()
    arena = 2 * need + (need // 2)
    srv = gpk.Server(0, arena_bytes=arena, max_slots=8, rank=20)
    try:
        futs = [srv.submit(_hyp(gpk, r), r.X, r.y, r.Xstar) for r in reqs]
        for f in futs:
            _, st = f.result(timeout=120)
            assert st["status"] == gpk.GP_OK
            assert st["bytes"] <= need
        s = srv.stats()
        assert s["peak_bytes"] <= arena and s["max_inflight"] <= 2 and s["in_use_bytes"] == 0, s
        big = _requests(1, seed=12, n_min=60000, n_max=60001)[0]
        with pytest.raises(gpk.GPKError) as e:
            srv.submit(_hyp(gpk, big), big.X, big.y, big.Xstar)
        assert e.value.status == gpk.GP_ERR_WORKSPACE
    finally:
        srv.close()


@pytest.mark.gpu
def test_late_small_requests_overlap_a_large_one(gpk):
    """A large request is submitted first; small requests submitted while it
    runs are admitted and finish before it does (continuous batching, not a
    queue)."""
    # the large request is well conditioned (RBF, l = 1, sigma^2 = 0.05) so it
    # converges in a few tens of iterations: the test is about overlap
    big = workloads.Request(rid=0, arrival_s=0.0, X=(r := np.random.default_rng(13)).standard_normal(
        (150000, 8)).astype(np.float32), y=np.zeros(150000, np.float32), Xstar=r.standard_normal((256, 8)).astype(
        np.float32), kernel=0, lengthscale=np.ones(8, np.float32), outputscale=1.0, noise=0.05)
    big.y[:] = np.sin(big.X.sum(axis=1)) + 0.1 * r.standard_normal(150000)
    small = _requests(4, seed=14, n_min=500, n_max=800)
    srv = gpk.Server(0, arena_bytes=4 << 30, max_slots=8, rank=20)
    try:
        fb = srv.submit(_hyp(gpk, big), big.X, big.y, big.Xstar)
        fs = [srv.submit(_hyp(gpk, r), r.X, r.y, r.Xstar) for r in small]
        sts = [f.result(timeout=120)[1] for f in fs]
        _, stb = fb.result(timeout=300)
        assert stb["status"] == gpk.GP_OK, stb
        for st in sts:
            assert st["status"] == gpk.GP_OK
            assert st["t_admit_ms"] < stb["t_done_ms"] and st["t_done_ms"] < stb["t_done_ms"], (st, stb)
    finally:
        srv.close()


def test_request_bytes_is_exact_layout_and_monotone():
    """CPU: the footprint query needs no device; it grows with N and n_test and
    refuses invalid requests."""
    from paper_2207_06856_gb300 import build, gpk as g
    import os
    if not os.path.exists(g.LIB_PATH):
        build.build()
    opts = g._server_opts(1 << 30, 4, 20, "fp16", "fp32", 1e-2, 200, 4, "pinv")
    import ctypes
    h = g.Hyper(g.RBF, np.ones(8, np.float32), 1.0, 0.05).c()
    f = lambda N, nt: g.lib().gp_server_request_bytes(ctypes.byref(opts), ctypes.byref(h), N, nt)  # noqa: E731
    a, b, c = f(1000, 1024), f(2000, 1024), f(1000, 4096)
    assert 0 < a < b and a < c
    # at least the persistent part: X, y, v, X*, mu*, L (rank 20)
    assert a >= 4 * (1000 * 8 + 2 * 1000 + 1024 * 8 + 1024 + 1000 * 20)
    assert f(0, 1024) == 0 and f(1000, 0) == 0
    bad = g.Hyper(g.RBF, np.ones(8, np.float32), 1.0, 0.0).c()   # noise must be > 0
    assert g.lib().gp_server_request_bytes(ctypes.byref(opts), ctypes.byref(bad), 1000, 1024) == 0


@pytest.mark.gpu
def test_wait_timeout_and_invalid_requests(gpk):
    """A host wait that runs out raises TimeoutError and leaves the request
    pending (a second wait returns its result); invalid submissions are refused
    at submit without reaching the device; a one-slot server serialises."""
    reqs = _requests(3, seed=21, n_min=20000, n_max=30000)
    srv = gpk.Server(0, arena_bytes=2 << 30, max_slots=1, rank=20)
    try:
        futs = [srv.submit(_hyp(gpk, r), r.X, r.y, r.Xstar) for r in reqs]
        with pytest.raises(TimeoutError):
            futs[-1].result(timeout=1e-4)
        outs = [f.result(timeout=120)[1] for f in futs]
        assert all(st["status"] == gpk.GP_OK for st in outs)
        assert srv.stats()["max_inflight"] == 1
        for a, b in zip(outs, outs[1:]):
            assert b["t_admit_ms"] >= a["t_done_ms"] - 1.0   # one slot: admitted after the previous finished
        r = reqs[0]
        with pytest.raises(gpk.GPKError) as e:                # noise must be > 0
            srv.submit(gpk.Hyper(r.kernel, r.lengthscale, r.outputscale, 0.0), r.X, r.y, r.Xstar)
        assert e.value.status == gpk.GP_ERR_INVALID
        with pytest.raises(ValueError):                       # X_test with the wrong d
            srv.submit(_hyp(gpk, r), r.X, r.y, r.Xstar[:, :-1])
    finally:
        srv.close()
