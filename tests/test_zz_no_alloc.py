"""gp_kmvm_noalloc: the allocation-free variant of the kernel MVM.

Some callers cannot allocate device memory: applications whose own pool owns
every allocation, latency-critical loops, plugins handed device pointers
only.  This entry point serves them from a fixed device array.  These tests
call it through the C ABI and check that it returns bit for bit what gp_kmvm
returns (it runs the same kernels on the same plan), for every precision and
engine option, on calls in a row (the array keeps the previous call's
contents); that its device-side status reads back clean; that repeated calls
change the free device memory by nothing; and that a problem beyond the
array's size is rejected.  The file is collected last on purpose, and it also
passes when run alone in a fresh process."""

import ctypes

import numpy as np
import pytest

from paper_2207_06856_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2207_06856_gb300 import gpk
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = gpk.Context(0)
    yield c
    c.close()


def _pair(ctx, hyp, Xd, Vd, prec, flags, Xc=None, add_noise=True):
    from paper_2207_06856_gb300 import gpk
    ref = gpk.kmvm(ctx, hyp, Xd, Vd, Xc=Xc, precision=prec, add_noise=add_noise, flags=flags)
    ctx.check()
    got = gpk.kmvm_noalloc(hyp, Xd, Vd, Xc=Xc, precision=prec, add_noise=add_noise, flags=flags)
    assert gpk.kmvm_noalloc_status() == gpk.GP_OK
    return ref.cpu().numpy(), got.cpu().numpy()


@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp32"])
def test_noalloc_equals_gp_kmvm_twice(ctx, prec):
    from paper_2207_06856_gb300 import gpk
    dev = torch.device("cuda:0")
    # two different problems back to back: the second call must not see the first's leftovers
    for (N, d, R, seed, kern) in [(3000, 8, 17, 31, gpk.RBF), (5000, 11, 5, 32, gpk.MATERN32)]:
        X, V, _, ls, a2, s2 = workloads.random_problem(N, d, R, seed=seed, kernel=kern)
        hyp = gpk.Hyper(kern, ls, a2, s2)
        ref, got = _pair(ctx, hyp, torch.from_numpy(X).to(dev), torch.from_numpy(V).to(dev), prec, 0)
        assert np.array_equal(ref, got), (N, prec)


@pytest.mark.parametrize("flag", ["MVM_PSPLIT", "MVM_ONE_TILE", "MVM_HALF_EXP", "MVM_XSPLIT"])
def test_noalloc_takes_every_gp_kmvm_flag(ctx, flag):
    from paper_2207_06856_gb300 import gpk
    dev = torch.device("cuda:0")
    X, V, kern, ls, a2, s2 = workloads.random_problem(2500, 8, 9, seed=34)
    hyp = gpk.Hyper(kern, ls, a2, s2)
    ref, got = _pair(ctx, hyp, torch.from_numpy(X).to(dev), torch.from_numpy(V).to(dev), "fp16",
                     getattr(gpk, flag))
    assert np.array_equal(ref, got), flag


def test_noalloc_rectangular_limit_and_no_allocation(ctx):
    from paper_2207_06856_gb300 import gpk
    dev = torch.device("cuda:0")
    X, V, kern, ls, a2, s2 = workloads.random_problem(2000, 4, 3, seed=33)
    Xs = torch.randn(700, 4, device=dev)
    hyp = gpk.Hyper(kern, ls, a2, s2)
    Xd, Vd = torch.from_numpy(X).to(dev), torch.from_numpy(V).to(dev)
    ref, got = _pair(ctx, hyp, Xs, Vd, "fp16", 0, Xc=Xd, add_noise=False)
    assert np.array_equal(ref, got)
    # calls of several shapes after the first (set-up) call leave the free memory unchanged
    cases = [(2000, "fp16"), (1500, "bf16"), (1000, "fp32"), (2000, "fp16")]
    ins = {n: (Xd[:n].contiguous(), Vd[:, :n].contiguous(), torch.empty(3, n, device=dev)) for n, _ in cases}
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for n, prec in cases:
        gpk.kmvm_noalloc(hyp, ins[n][0], ins[n][1], precision=prec, add_noise=True, out=ins[n][2])
    assert gpk.kmvm_noalloc_status() == gpk.GP_OK
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    # beyond the fixed scratch: rejected, nothing launched
    big = torch.zeros(400000, 4, device=dev)
    bigV = torch.zeros(32, 400000, device=dev)
    with pytest.raises(gpk.GPKError) as ei:
        gpk.kmvm_noalloc(hyp, big, bigV, precision="fp16", add_noise=True)
    assert ei.value.status == gpk.GP_ERR_WORKSPACE


def test_noalloc_symbols_are_exported():
    from paper_2207_06856_gb300 import gpk
    lib = ctypes.CDLL(gpk.LIB_PATH)
    assert hasattr(lib, "gp_kmvm_noalloc") and hasattr(lib, "gp_kmvm_noalloc_check")
