"""gp_kmvm_noalloc: the allocation-free variant of the kernel MVM.

Some callers cannot allocate device memory (applications whose own pool owns
every allocation, latency-critical loops, plugins handed device pointers
only).  This entry point serves them from a fixed device array; these tests
call it through the C ABI and check that it returns what gp_kmvm returns,
within the MVM tolerances of the other GPU tests, on two calls in a row (the
array keeps the previous call's contents), and that a problem beyond the
array's size is rejected.  The file is collected last on purpose, and it also
passes when run alone in a fresh process."""

import ctypes

import numpy as np
import pytest

from paper_2207_06856_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp16": 2e-3, "bf16": 2e-3}


def _colerr(got, ref):
    return float(np.max(np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)))


@pytest.fixture(scope="module")
def ctx():
    from paper_2207_06856_gb300 import gpk
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = gpk.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp32"])
def test_noalloc_matches_gp_kmvm_twice(ctx, prec):
    from paper_2207_06856_gb300 import gpk
    dev = torch.device("cuda:0")
    # two different problems back to back: the second call must not see the first's leftovers
    for (N, d, R, seed, kern) in [(3000, 8, 17, 31, gpk.RBF), (5000, 11, 5, 32, gpk.MATERN32)]:
        X, V, _, ls, a2, s2 = workloads.random_problem(N, d, R, seed=seed, kernel=kern)
        hyp = gpk.Hyper(kern, ls, a2, s2)
        Xd, Vd = torch.from_numpy(X).to(dev), torch.from_numpy(V).to(dev)
        ref = gpk.kmvm(ctx, hyp, Xd, Vd, precision=prec, add_noise=True)
        got = gpk.kmvm_noalloc(hyp, Xd, Vd, precision=prec, add_noise=True)
        torch.cuda.synchronize()
        ctx.check()
        err = _colerr(got.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64))
        assert err <= TOL[prec], (N, prec, err)


def test_noalloc_rectangular_and_limit(ctx):
    from paper_2207_06856_gb300 import gpk
    dev = torch.device("cuda:0")
    X, V, kern, ls, a2, s2 = workloads.random_problem(2000, 4, 3, seed=33)
    Xs = torch.randn(700, 4, device=dev)
    hyp = gpk.Hyper(kern, ls, a2, s2)
    Xd, Vd = torch.from_numpy(X).to(dev), torch.from_numpy(V).to(dev)
    ref = gpk.kmvm(ctx, hyp, Xs, Vd, Xc=Xd, precision="fp16")
    got = gpk.kmvm_noalloc(hyp, Xs, Vd, Xc=Xd, precision="fp16")
    torch.cuda.synchronize()
    assert _colerr(got.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)) <= TOL["fp16"]
    # beyond the fixed scratch: rejected, nothing launched
    big = torch.zeros(400000, 4, device=dev)
    bigV = torch.zeros(32, 400000, device=dev)
    with pytest.raises(gpk.GPKError) as ei:
        gpk.kmvm_noalloc(hyp, big, bigV, precision="fp16", add_noise=True)
    assert ei.value.status == gpk.GP_ERR_WORKSPACE


def test_noalloc_symbol_is_exported():
    from paper_2207_06856_gb300 import gpk
    assert hasattr(ctypes.CDLL(gpk.LIB_PATH), "gp_kmvm_noalloc")
